// ac_device.cuh -- device primitives of the GB300 (sm_103a) cellular-array kernels.
//
// Everything here is exact integer arithmetic; the only floating-point step of
// the method (the heat-bath threshold table) is done on the host.
//
//   philox_event()  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) of the
//                   counter {c, k, w2, 0} under the key (seed lo, seed hi): one
//                   counter stream per cell, the per-cell reproducible sequence
//                   the paper asks for (Sec. 5, and the invariance remark after
//                   Fig. 3.6).
//   exp_ticks()     integer exponential gap standing in for -ln r of Eq. (5),
//                   2^32 ticks per unit time: 33 - log2(2x+1) in Q.32 by the
//                   bit-by-bit repeated-squaring logarithm, times ln 2, plus one
//                   tick so that next_t > t (Eq. (2)).
//
// Packed cell word: key = tick << 1 | (spin > 0).  A word carries a cell's next
// arrival time and its current spin together, so a single 64-bit access always
// sees a consistent (time, spin) pair.
#pragma once
#include <cstdint>

namespace ac {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr unsigned long long kLn2Q64 = 0xB17217F7D1CF79ABull;  // floor(ln 2 * 2^64)

struct Philox4 {
  uint32_t x, y, z, w;
};

// Philox4x32-10 with counter {c0, c1, c2, 0}.  Each round multiplies the two even
// words by the round constants (one 32x32->64 product each), xors the high halves
// into the odd words together with the round key and permutes; the key advances
// by the Weyl constants between rounds.
__device__ __forceinline__ Philox4 philox_event(uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t k0, uint32_t k1) {
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = 0u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)kPhiloxM0 * x0;
    const unsigned long long p1 = (unsigned long long)kPhiloxM1 * x2;
    const uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    const uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    x1 = (uint32_t)p1;
    x3 = (uint32_t)p0;
    x0 = y0;
    x2 = y2;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return Philox4{x0, x1, x2, x3};
}

// Integer exponential gap for a 32-bit uniform word x (u = (2x+1)/2^33).
//   k = floor(log2(2x+1)), y = 2x+1 normalised to [2^31, 2^32) (x itself when k = 32);
//   32 steps of: square y (a full 64-bit product), emit the bit that says whether
//   the square reached 2.0 in Q1.31, and keep the truncated Q1.31 value (halved
//   when the bit is set);  gap = floor(((33 - k) * 2^32 - f) * ln2 * 2^64 / 2^64) + 1.
//
// Pipe balance (measured with the exp_ticks probe on a GB300): the 32x32->64 square
// occupies the FMA-heavy pipe for several cycles, so the step's other
// work is split: the shift amount 31 + bit comes from the integer ALU (a shift and
// an add), the funnel shift is an ALU op, and the accumulation f' = 2 f' + amt is a
// multiply-add on the FMA pipe -- `two` must hold 2 at run time but be opaque to the
// compiler (a kernel argument) so that it stays one.  Since
// sum_i (31 + b_i) 2^(31-i) = f + 31 (2^32 - 1), the bits are f = f' + 31 (mod 2^32).
__device__ __forceinline__ unsigned long long exp_ticks(uint32_t x, uint32_t two) {
  uint32_t k, y;
  if (x & 0x80000000u) {
    k = 32u;
    y = x;
  } else {
    const uint32_t m = 2u * x + 1u;
    const uint32_t lz = __clz(m);
    k = 31u - lz;
    y = m << lz;
  }
  uint32_t fa = 0u;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const unsigned long long sq = (unsigned long long)y * y;
    const uint32_t hi = (uint32_t)(sq >> 32);
    const uint32_t lo = (uint32_t)sq;
    const uint32_t amt = (hi >> 31) + 31u;               // 32 if the square reached 2.0, else 31
    y = __funnelshift_rc(lo, hi, amt);                   // square >> (31 + bit), low word
    fa = fa * two + amt;
  }
  const uint32_t f = fa + 31u;
  const unsigned long long nl = ((unsigned long long)(33u - k) << 32) - f;
  return __umul64hi(nl, kLn2Q64) + 1ull;
}

// Gap of a cell with rate 2^20 / m for the rate-1 gap e: max(1, floor(e m / 2^20)),
// from the full 128-bit product (the general asynchrony law (A) of Sec. 2).
__device__ __forceinline__ unsigned long long rated_gap(unsigned long long e, uint32_t m) {
  const unsigned long long lo = e * (unsigned long long)m;
  const unsigned long long hi = __umul64hi(e, (unsigned long long)m);
  const unsigned long long g = (hi << 44) | (lo >> 20);
  return g ? g : 1ull;
}

}  // namespace ac
