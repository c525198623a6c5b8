// ac_time.cu -- the time-only round model of Sec. 4 on the GPU.
//
// Sec. 4 assesses the synchronous round algorithm (Fig. 3.2) with a model that
// keeps only the cells' local times: in a round a cell advances iff its key
// (t, index) is below the keys of all its neighbours and t < t_end, and then draws
// its next increment.  The paper runs it on an n-cell circle, an n x n torus and an
// n x n x n periodic array, with exponential and uniform increments (and r^(1/8)),
// and reports the limiting fraction of cells that advance per round.
//
// The neighbourhood is the 2 dims nearest cells, or the q-th degree neighbourhood of
// Sec. 3 (every cell within Manhattan distance q).
//
// One launch per round, ping-pong time buffers (a cell's decision reads its
// neighbours' times before any of them advances), per-cell counts in place (only
// the owner touches them), and a per-round count of advancing cells.  Increments
// (from the word x of Philox block {c, k, 0, 0}, k = the cell's advance number):
//   law 0  exp_ticks(x)                                  (exponential, Eq. (5))
//   law 1  x + 1                                         (uniform on (0, 1])
//   law 2  three nested integer square roots of (2x+1) 2^31, each step rescaled
//          by 2^32: floor-exact r^(1/8) 2^32 up to the truncation of each step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ac.h"
#include "ac_device.cuh"
#include "ac_internal.h"

namespace ac {
namespace {

// floor(sqrt(v)) for any 64-bit v: a binary64 estimate (off by at most one for
// v < 2^64) corrected with exact integer products; the root is < 2^32, so r * r
// never overflows, and (r + 1)^2 is only formed while r + 1 < 2^32.
__device__ __forceinline__ unsigned long long isqrt_u64(unsigned long long v) {
  unsigned long long r = (unsigned long long)sqrt((double)v);
  if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
  while (r * r > v) --r;
  while (r < 0xFFFFFFFFull && (r + 1) * (r + 1) <= v) ++r;
  return r;
}

__device__ __forceinline__ unsigned long long law_gap(int law, uint32_t x, uint32_t two) {
  if (law == 0) return exp_ticks(x, two);
  if (law == 1) return (unsigned long long)x + 1ull;
  const unsigned long long s1 = isqrt_u64((2ull * x + 1ull) << 31);
  const unsigned long long s2 = isqrt_u64(s1 << 32);
  return isqrt_u64(s2 << 32);
}

struct TimeDesc {
  long long* t_in;
  long long* t_out;
  unsigned* cnt;
  unsigned long long* hist;   // advancing cells per round
  unsigned n, N;
  int law;
  int q;                      // neighbourhood: every cell within Manhattan distance q
  unsigned seed_lo, seed_hi, two;
  long long t_end;
};

__global__ void time_init_kernel(TimeDesc D) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < D.N;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned c = (unsigned)i;
    const Philox4 b = philox_event(c, 0u, 0u, D.seed_lo, D.seed_hi);
    D.t_in[c] = (long long)law_gap(D.law, b.x, D.two);
    D.cnt[c] = 0u;
  }
}

// key (tc, c) below (tn, nb): the (tick, index) order
__device__ __forceinline__ bool key_below(long long tc, unsigned c, long long tn, unsigned nb) {
  return (tc < tn) || (tc == tn && c < nb) || nb == c;
}

template <int DIMS>
__global__ void __launch_bounds__(256) time_round_kernel(TimeDesc D, int round) {
  // uniform early exit once a round advanced nothing (the state is then final)
  if (round > 0 && *(volatile unsigned long long*)&D.hist[round - 1] == 0ull) return;
  unsigned adv = 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < D.N;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned c = (unsigned)i;
    const long long tc = D.t_in[c];
    bool ok = tc < D.t_end;
    unsigned co[3] = {0u, 0u, 0u};
    {
      unsigned rest = c;
#pragma unroll
      for (int a = 0; a < DIMS; ++a) {
        co[a] = rest % D.n;
        rest /= D.n;
      }
    }
    if (D.q == 1) {
      unsigned stride = 1;
#pragma unroll
      for (int a = 0; a < DIMS; ++a) {
        const unsigned x = co[a];
        const unsigned lo = c - x * stride + ((x == 0 ? D.n : x) - 1) * stride;
        const unsigned hi = c - x * stride + ((x + 1 == D.n) ? 0u : x + 1) * stride;
        ok &= key_below(tc, c, D.t_in[lo], lo);
        ok &= key_below(tc, c, D.t_in[hi], hi);
        stride *= D.n;
      }
    } else {
      // the q-th degree neighbourhood (Sec. 3): all offsets with 0 < |dx|+|dy|+|dz| <= q
      const int q = D.q;
      const long long n = (long long)D.n;
      const int qy = DIMS > 1 ? q : 0, qz = DIMS > 2 ? q : 0;
      for (int dz = -qz; dz <= qz && ok; ++dz)
        for (int dy = -qy; dy <= qy && ok; ++dy) {
          const int rem = q - (dz < 0 ? -dz : dz) - (dy < 0 ? -dy : dy);
          if (rem < 0) continue;
          const unsigned zz = DIMS > 2 ? (unsigned)(((long long)co[2] + dz + n) % n) : 0u;
          const unsigned yy = DIMS > 1 ? (unsigned)(((long long)co[1] + dy + n) % n) : 0u;
          const unsigned rowbase = (zz * D.n + yy) * D.n;
          for (int dx = -rem; dx <= rem; ++dx) {
            if (dx == 0 && dy == 0 && dz == 0) continue;
            const unsigned nb = rowbase + (unsigned)(((long long)co[0] + dx + n) % n);
            ok &= key_below(tc, c, D.t_in[nb], nb);
          }
        }
    }
    long long tn = tc;
    if (ok) {
      const unsigned k = D.cnt[c] + 1u;
      const Philox4 b = philox_event(c, k, 0u, D.seed_lo, D.seed_hi);
      tn = tc + (long long)law_gap(D.law, b.x, D.two);
      D.cnt[c] = k;
      ++adv;
    }
    D.t_out[c] = tn;
  }
  for (int o = 16; o > 0; o >>= 1) adv += __shfl_down_sync(0xffffffffu, adv, o);
  if ((threadIdx.x & 31) == 0 && adv) atomicAdd(&D.hist[round], (unsigned long long)adv);
}

ac_status time_fail(ac_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace
}  // namespace ac

extern "C" ac_status ac_time_model(int32_t dims, int64_t n, int32_t q, int32_t law, uint64_t seed, int64_t t_end,
                                   int32_t max_rounds, uint64_t* enabled, int32_t* rounds_out, int64_t* t_out,
                                   uint32_t* n_out, double* device_ms) {
  using namespace ac;
  if (dims < 1 || dims > 3) return time_fail(AC_ERR_ARG, "dims must be 1, 2 or 3");
  if (n < 2) return time_fail(AC_ERR_ARG, "n must be >= 2");
  if (q < 1 || q > 8 || (q > 1 && n < 2 * q + 1)) return time_fail(AC_ERR_ARG, "q must be in 1..8 with n >= 2q+1");
  if (law < AC_LAW_EXP || law > AC_LAW_ROOT8) return time_fail(AC_ERR_ARG, "law must be 0, 1 or 2");
  if (max_rounds < 1 || !enabled || !rounds_out) return time_fail(AC_ERR_ARG, "max_rounds >= 1, enabled and rounds_out are required");
  if (t_end < 0) return time_fail(AC_ERR_ARG, "t_end must be >= 0");
  double Nd = 1.0;
  for (int a = 0; a < dims; ++a) Nd *= (double)n;
  if (Nd >= 4294967296.0) return time_fail(AC_ERR_ARG, "n^dims must be < 2^32 (the Philox cell counter)");
  const unsigned N = (unsigned)Nd;

  TimeDesc D{};
  long long *ta = nullptr, *tb = nullptr;
  unsigned* cnt = nullptr;
  unsigned long long* hist = nullptr;
  auto release = [&]() {
    cudaFree(ta);
    cudaFree(tb);
    cudaFree(cnt);
    cudaFree(hist);
  };
  if (cudaMalloc(&ta, (size_t)N * 8) != cudaSuccess || cudaMalloc(&tb, (size_t)N * 8) != cudaSuccess ||
      cudaMalloc(&cnt, (size_t)N * 4) != cudaSuccess || cudaMalloc(&hist, (size_t)max_rounds * 8) != cudaSuccess) {
    cudaGetLastError();
    release();
    return time_fail(AC_ERR_OOM, "time model: device allocation failed");
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ac_status status = AC_OK;
  do {
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
      status = time_fail(AC_ERR_CUDA, "time model: stream or event creation failed");
      break;
    }
    D.t_in = ta;
    D.t_out = tb;
    D.cnt = cnt;
    D.hist = hist;
    D.n = (unsigned)n;
    D.N = N;
    D.law = law;
    D.q = q;
    D.seed_lo = (unsigned)(seed & 0xffffffffu);
    D.seed_hi = (unsigned)(seed >> 32);
    D.two = 2u;
    D.t_end = t_end;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<long long>(((long long)N + 255) / 256, (long long)sms * 8);
    if (cudaMemsetAsync(hist, 0, (size_t)max_rounds * 8, st) != cudaSuccess) {
      status = time_fail(AC_ERR_CUDA, "time model: memset failed");
      break;
    }
    time_init_kernel<<<grid, 256, 0, st>>>(D);
    cudaEventRecord(e0, st);
    int rounds = 0;
    bool done = false;
    std::vector<unsigned long long> h;
    for (int r0 = 0; r0 < max_rounds && !done; r0 += 64) {
      const int r1 = std::min(max_rounds, r0 + 64);
      for (int r = r0; r < r1; ++r) {
        TimeDesc Dr = D;
        if (r & 1) std::swap(Dr.t_in, Dr.t_out);
        switch (dims) {
          case 1: time_round_kernel<1><<<grid, 256, 0, st>>>(Dr, r); break;
          case 2: time_round_kernel<2><<<grid, 256, 0, st>>>(Dr, r); break;
          default: time_round_kernel<3><<<grid, 256, 0, st>>>(Dr, r); break;
        }
      }
      h.resize((size_t)(r1 - r0));
      if (cudaMemcpyAsync(h.data(), hist + r0, h.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        status = time_fail(AC_ERR_CUDA, "time model: round launch failed");
        break;
      }
      for (size_t i = 0; i < h.size(); ++i) {
        if (h[i] == 0) {
          done = true;
          break;
        }
        enabled[rounds++] = h[i];
      }
    }
    if (status != AC_OK) break;
    cudaEventRecord(e1, st);
    // the last launched round (productive or the first empty one) wrote the final state
    const int last = (rounds < max_rounds) ? rounds : max_rounds - 1;
    const long long* fin = (last & 1) ? ta : tb;
    if (t_out && cudaMemcpyAsync(t_out, fin, (size_t)N * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      status = time_fail(AC_ERR_CUDA, "time model: copy-out failed");
      break;
    }
    if (n_out && cudaMemcpyAsync(n_out, cnt, (size_t)N * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      status = time_fail(AC_ERR_CUDA, "time model: copy-out failed");
      break;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      status = time_fail(AC_ERR_CUDA, "time model: kernel failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (device_ms) *device_ms = ms;
    *rounds_out = rounds;
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  release();
  return status;
}
