// ac_kernels.cu -- sm_103a kernels of the exact parallel simulator of the
// Poisson-asynchronous Glauber (continuous-time Ising) cellular array.
//
// Paper: Lubachevsky, "Efficient Parallel Simulations of Asynchronous Cellular
// Arrays".  A cell may commit its next arrival once its (tick, index) key is
// below the keys of all its neighbours (Fig. 3.1 with the tie rule that the
// smaller row-major index goes first); the result is the unique trajectory of
// the standard serial procedure (Sec. 1) whatever the execution schedule.
//
// Kernels: the round kernel (a), one synchronous round per launch or, with
// temporal blocking, R rounds per launch (the path the throughput figures use);
// the blocked persistent kernel (b); the initialisation, statistics and
// state-transfer kernels; the frame fill; device-primitive probes.  The
// temporal-blocked kernel also runs the Life-like automaton (Moore neighbourhood)
// and writes snapshot frames (Fig. 3.7) when they are open.
//
// Shared-memory tile engine (used by the one-round and blocked kernels).  A CTA holds one tile of at
// most LB x LB cells: the packed keys with a one-cell halo ring, the event
// counts and a compacted work list.  One tile round is
//   scan    every thread walks a column segment and tests its cells against
//           the four neighbours (the enable test of Fig. 3.2, step 2); enabled
//           cells are appended to the work list (warp prefix + one shared
//           atomic per warp);
//   commit  after a barrier, all threads take list entries: neighbour spin
//           sum, one Philox4x32-10 block, flip decision against the threshold
//           table (Eq. (1)) and the next arrival (Eq. (5)); enabled cells form
//           an independent set, so they are updated in place; a barrier ends
//           the round (Fig. 3.2's two synchronisations).
// The enable test works on packed words: with key = tick<<1 | up,
//   tick_c <  tick_n  <=>  (key_c | 1)  <  key_n    (neighbour with smaller index)
//   tick_c <= tick_n  <=>  (key_c & ~1) <= key_n    (neighbour with larger index)
// Inside a tile the up/left neighbours have smaller and the down/right
// neighbours larger indices; at the torus wrap the order flips, which the halo
// absorbs by storing key + 2 (turns "<" into "<=") or key - 2 (turns "<=" into
// "<").  Halo cells never commit.
//
// (a) round kernel: one launch per R tile rounds; halos are frozen copies of the
//     neighbour tiles' edge words of the previous launch (ping-pong), so R = 1 is
//     exactly the synchronous one-cell-per-PE algorithm of Fig. 3.2 run over the
//     whole lattice.
// (b) blocked persistent kernel: the aggregated algorithm of Fig. 3.4 with one
//     CTA per PE and a tile per subarray.  A CTA owns a fixed set of tiles and
//     visits them in turn; boundary commits are published at once as edge words
//     in HBM and neighbours refresh their halos from them.  A published word only
//     grows, so a stale halo value is a lower bound of the neighbour's key and can
//     only delay a commit, never admit a wrong one (the argument of Sec. 3 that a
//     neighbour's state cannot change in (T1, T5)).  Blocked tiles poll a bounded
//     number of times and are then left for the CTA's next tile; a
//     %globaltimer watchdog turns a stall into an error code.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ac_device.cuh"
#include "ac_internal.h"

namespace ac {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- bounds-checked build (-DAC_CHECK, libac_check.so): the kernels check the indices they
// compute -- region cells, order-plane words, work-list entries, table entries, lattice cells,
// bulk-copy ranges, epoch words, frame slots -- and record the first violation, (site << 40)
// | index, in g_check_word; the index is then replaced by 0 so that no access leaves its
// array.  The host turns a recorded violation into AC_ERR_STATE.  Without AC_CHECK both
// macros are empty and the kernels are unchanged.
#ifdef AC_CHECK
__device__ unsigned long long g_check_word = 0ull;
__device__ __forceinline__ long long ac_check_index(long long i, long long n, int site) {
  if (i >= 0 && i < n) return i;
  atomicCAS(&g_check_word, 0ull, ((unsigned long long)site << 40) | ((unsigned long long)i & 0xFFFFFFFFFFull));
  return 0;
}
#define ACI(i, n, site) ac_check_index((long long)(i), (long long)(n), (site))
#define ACK(cond, site, idx)                                                                               \
  do {                                                                                                     \
    if (!(cond))                                                                                           \
      atomicCAS(&g_check_word, 0ull, ((unsigned long long)(site) << 40) | ((unsigned long long)(idx) & 0xFFFFFFFFFFull)); \
  } while (0)
#else
#define ACI(i, n, site) (i)
#define ACK(cond, site, idx) \
  do {                       \
  } while (0)
#endif

// Snapshot frames (Fig. 3.7).  Frame K holds every cell's spin after all of its
// arrivals with tick <= K dt (the figure stores the image before it processes the
// first event later than K dt).  The commit of an arrival at tick ta, whose next
// arrival is at tick tn, is therefore the last one <= T for every frame tick T in
// [ta, tn): it writes the new spin there.  The open frames are evenly spaced.
struct FrameView {
  signed char* frames;
  unsigned long long t0, dt, t_last;   // ticks of the first and the last open frame
  unsigned long long N;                // cells per frame slot
  float inv_dt;
  int open, slot0, B;
};

__device__ __forceinline__ FrameView frame_view(const LatDesc& L) {
  FrameView F;
  F.frames = L.frames;
  F.t0 = (unsigned long long)L.f_t0;
  F.dt = (unsigned long long)L.f_dt;
  F.t_last = F.t0 + (unsigned long long)(L.f_open - 1) * F.dt;
  F.N = (unsigned long long)L.rows * (unsigned long long)L.cols;
  F.inv_dt = 1.0f / (float)F.dt;
  F.open = L.f_open;
  F.slot0 = L.f_slot0;
  F.B = L.f_B;
  return F;
}

__device__ __forceinline__ void write_frames(const FrameView& F, size_t gi, unsigned long long ta,
                                             unsigned long long tn, unsigned up) {
  if (tn <= F.t0 || ta > F.t_last) return;        // no open frame tick in [ta, tn)
  unsigned f = 0;
  if (ta > F.t0) {
    // first frame with t0 + f dt >= ta: a float estimate (f <= 64), then exact steps
    const unsigned long long d = ta - F.t0;
    f = (unsigned)((float)d * F.inv_dt);
    while ((unsigned long long)f * F.dt < d) ++f;
    while (f > 0 && (unsigned long long)(f - 1) * F.dt >= d) --f;
  }
  unsigned long long T = F.t0 + (unsigned long long)f * F.dt;
  int slot = F.slot0 + (int)f;
  if (slot >= F.B) slot -= F.B;
  for (; (int)f < F.open && T < tn; ++f) {
    F.frames[ACI((size_t)slot * F.N + gi, (long long)F.B * (long long)F.N, 15)] = up ? (signed char)1 : (signed char)-1;
    T += F.dt;
    if (++slot == F.B) slot = 0;
  }
}

struct Geom {
  int ti, tj, r0, h, c0, w;
};

__device__ __forceinline__ Geom tile_geom(const LatDesc& L, int t) {
  Geom g;
  g.ti = t / L.tc;
  g.tj = t - g.ti * L.tc;
  const int rn = L.srows ? L.srows : L.rows;   // a row slab tiles only its own rows
  int q = rn / L.tr, rm = rn - q * L.tr;
  g.r0 = L.srow0 + g.ti * q + min(g.ti, rm);
  g.h = q + (g.ti < rm);
  const int cu = L.cpair ? 2 : 1;      // column unit: pairs keep every start and width even
  const int cn = L.cols / cu;
  q = cn / L.tc;
  rm = cn - q * L.tc;
  g.c0 = cu * (g.tj * q + min(g.tj, rm));
  g.w = cu * (q + (g.tj < rm));
  return g;
}

// Lattice owning global tile `tile` (tile_base ascending).
__device__ __forceinline__ int find_lattice(const LatDesc* lats, int nlat, int tile) {
  int lo = 0, hi = nlat - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&lats[mid].tile_base) <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int LB>
struct TileShape {
  static constexpr int P = LB + 2;                 // key row pitch (words), halo ring included
  static constexpr int NT = 4 * LB;                // threads: LB columns x 4 row groups
  static constexpr int LIST = LB * LB / 2 + LB;    // enabled cells form an independent set
  static constexpr size_t kBytes = size_t(P) * P * 8;
  static constexpr size_t cBytes = size_t(LB) * LB * 4;
  static constexpr size_t lBytes = ((size_t(LIST) * 2 + 15) / 16) * 16;
  static constexpr size_t mBytes = 64;             // n_en[2], thr[10]
  static constexpr size_t bytes = kBytes + cBytes + lBytes + mBytes;
};

template <int LB>
struct Smem {
  unsigned long long* K;
  unsigned int* C;
  unsigned short* list;
  unsigned int* n_en;   // [2]
  unsigned int* thr;    // [10]
  __device__ __forceinline__ explicit Smem(unsigned char* base) {
    using S = TileShape<LB>;
    K = reinterpret_cast<unsigned long long*>(base);
    C = reinterpret_cast<unsigned int*>(base + S::kBytes);
    list = reinterpret_cast<unsigned short*>(base + S::kBytes + S::cBytes);
    n_en = reinterpret_cast<unsigned int*>(base + S::kBytes + S::cBytes + S::lBytes);
    thr = n_en + 2;
  }
};

// Per-thread halo slot: thread tid handles edge e = tid / LB, position p = tid % LB.
struct HaloSlot {
  const unsigned long long* src;   // neighbour tile's edge word (nullptr: none / self-wrap)
  long long adj;                   // +2 / -2 at the torus wrap, else 0
  int slot;                        // index into K (-1: unused)
  int mirror;                      // self-wrap: index into K of the mirrored own cell (-1: none)
};

template <int LB>
__device__ __forceinline__ HaloSlot halo_slot(const LatDesc& L, const Geom& g,
                                              const unsigned long long* pub) {
  constexpr int P = TileShape<LB>::P;
  const int e = threadIdx.x / LB, p = threadIdx.x % LB;
  HaloSlot s{nullptr, 0, -1, -1};
  const bool row_edge = e < 2;
  if (row_edge ? (p >= g.w) : (p >= g.h)) return s;
  switch (e) {
    case 0: s.slot = p + 1; s.adj = (g.ti == 0) ? 2 : 0; break;                 // top halo
    case 1: s.slot = (g.h + 1) * P + p + 1; s.adj = (g.ti == L.tr - 1) ? -2 : 0; break;
    case 2: s.slot = (p + 1) * P; s.adj = (g.tj == 0) ? 2 : 0; break;            // left halo
    default: s.slot = (p + 1) * P + g.w + 1; s.adj = (g.tj == L.tc - 1) ? -2 : 0; break;
  }
  const bool self = row_edge ? (L.tr == 1) : (L.tc == 1);
  if (self) {
    switch (e) {
      case 0: s.mirror = g.h * P + p + 1; break;          // own row h-1
      case 1: s.mirror = 1 * P + p + 1; break;            // own row 0
      case 2: s.mirror = (p + 1) * P + g.w; break;        // own column w-1
      default: s.mirror = (p + 1) * P + 1; break;         // own column 0
    }
    return s;
  }
  int nti = g.ti, ntj = g.tj, ne;
  switch (e) {
    case 0: nti = (g.ti + L.tr - 1) % L.tr; ne = 1; break;
    case 1: nti = (g.ti + 1) % L.tr; ne = 0; break;
    case 2: ntj = (g.tj + L.tc - 1) % L.tc; ne = 3; break;
    default: ntj = (g.tj + 1) % L.tc; ne = 2; break;
  }
  s.src = pub + ACI(((size_t)(nti * L.tc + ntj) * 4 + ne) * LB + p, (long long)L.tr * L.tc * 4 * LB, 27);
  return s;
}

// Load the tile's interior keys (and counts) from HBM into shared memory.
template <int LB, bool COUNTS>
__device__ __forceinline__ void load_interior(const Smem<LB>& sm, const LatDesc& L, const Geom& g) {
  constexpr int P = TileShape<LB>::P;
  const int c = threadIdx.x % LB;
  if (c >= g.w) return;
  for (int r = threadIdx.x / LB; r < g.h; r += 4) {
    const size_t gi = ACI((size_t)(g.r0 + r) * L.cols + g.c0 + c, (long long)L.rows * L.cols, 21);
    ACK(g.h <= LB && g.w <= LB, 22, g.h);
    sm.K[(r + 1) * P + c + 1] = L.key[gi];
    if (COUNTS) sm.C[r * LB + c] = L.cnt[gi];
  }
}

template <int LB, bool COUNTS>
__device__ __forceinline__ bool store_interior(const Smem<LB>& sm, const LatDesc& L, const Geom& g) {
  constexpr int P = TileShape<LB>::P;
  const int c = threadIdx.x % LB;
  bool unfinished = false;
  if (c >= g.w) return false;
  for (int r = threadIdx.x / LB; r < g.h; r += 4) {
    const size_t gi = ACI((size_t)(g.r0 + r) * L.cols + g.c0 + c, (long long)L.rows * L.cols, 23);
    const unsigned long long k = sm.K[(r + 1) * P + c + 1];
    L.key[gi] = k;
    if (COUNTS) L.cnt[gi] = sm.C[r * LB + c];
    unfinished |= k < L.t2;
  }
  return unfinished;
}

// Enable test over the thread's column segment; appends enabled cells to the list.
// Returns whether any of the thread's cells still has an arrival before t_end.
template <int LB>
__device__ __forceinline__ bool scan_tile(const Smem<LB>& sm, const Geom& g, unsigned long long t2,
                                          unsigned int* n_slot, unsigned long long& scanned) {
  constexpr int P = TileShape<LB>::P;
  const int c = threadIdx.x % LB;
  const int grp = threadIdx.x / LB;
  const int rpg = (g.h + 3) >> 2;
  const int rb = grp * rpg;
  const int re = min(g.h, rb + rpg);
  unsigned mask = 0;
  bool live_any = false;
  if (c < g.w && rb < re) {
    const unsigned long long* col = sm.K + (rb + 1) * P + (c + 1);
    unsigned long long up = col[-P];
    unsigned long long cur = col[0];
#pragma unroll 4
    for (int r = rb; r < re; ++r) {
      const unsigned long long down = col[P];
      const unsigned long long left = col[-1];
      const unsigned long long right = col[1];
      const unsigned long long hi = cur | 1ull, lo = cur & ~1ull;
      const bool live = cur < t2;
      const bool en = live & (hi < up) & (hi < left) & (lo <= right) & (lo <= down);
      live_any |= live;
      mask |= (unsigned)en << (r - rb);
      up = cur;
      cur = down;
      col += P;
    }
    scanned += (unsigned long long)(re - rb);
  }
  // warp-level compaction: inclusive prefix of per-thread counts, one atomic per warp
  const int lane = threadIdx.x & 31;
  const int cnt = __popc(mask);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  int base = 0;
  if (lane == 31 && incl) base = (int)atomicAdd(n_slot, (unsigned)incl);
  base = __shfl_sync(kFull, base, 31);
  int off = base + incl - cnt;
  while (mask) {
    const int b = __ffs(mask) - 1;
    mask &= mask - 1;
    sm.list[ACI(off++, TileShape<LB>::LIST, 24)] = (unsigned short)(((rb + b) << 8) | c);
  }
  return live_any;
}

// Commit the listed cells.  DIRECT: counts and keys are read from / written to HBM
// (single exact round per launch); PUBLISH: boundary commits are published as
// edge words (blocked kernel).
template <int LB, bool DIRECT, bool PUBLISH>
__device__ __forceinline__ void commit_tile(const Smem<LB>& sm, const LatDesc& L, const Geom& g,
                                            unsigned long long* pub_tile, int n) {
  constexpr int P = TileShape<LB>::P;
  constexpr int NT = TileShape<LB>::NT;
  for (int i = threadIdx.x; i < n; i += NT) {
    const unsigned e = sm.list[ACI(i, TileShape<LB>::LIST, 24)];
    const int r = (int)(e >> 8), c = (int)(e & 255u);
    ACK(r >= 0 && r < g.h && c >= 0 && c < g.w, 25, e);
    unsigned long long* kp = sm.K + (r + 1) * P + (c + 1);
    const unsigned long long key = *kp;
    const unsigned j = ((unsigned)kp[-P] & 1u) + ((unsigned)kp[P] & 1u) +
                       ((unsigned)kp[-1] & 1u) + ((unsigned)kp[1] & 1u);
    const unsigned sp = (unsigned)key & 1u;
    const uint32_t gidx = (uint32_t)ACI((uint32_t)(g.r0 + r) * (uint32_t)L.cols + (uint32_t)(g.c0 + c),
                                        (long long)L.rows * L.cols, 26);
    const unsigned n_old = DIRECT ? L.cnt[gidx] : sm.C[r * LB + c];
    const Philox4 b = philox_event(gidx, n_old + 1u, 0u, L.seed_lo, L.seed_hi);
    const unsigned flip = b.y < sm.thr[ACI(j + 5u * sp, 10, 9)] ? 1u : 0u;
    unsigned long long gap = exp_ticks(b.x, L.two);
    if (L.rates) gap = rated_gap(gap, L.rates[gidx]);
    const unsigned long long nk = (key & ~1ull) + (gap << 1) + (sp ^ flip);
    *kp = nk;
    if (L.f_open) write_frames(frame_view(L), gidx, key >> 1, nk >> 1, (unsigned)nk & 1u);
    if (DIRECT) {
      L.key[gidx] = nk;
      L.cnt[gidx] = n_old + 1u;
    } else {
      sm.C[r * LB + c] = n_old + 1u;
    }
    if (L.tr == 1) {                    // vertical self-wrap: keep the mirrored halo rows live
      if (r == 0) sm.K[(g.h + 1) * P + c + 1] = nk - 2ull;
      if (r == g.h - 1) sm.K[c + 1] = nk + 2ull;
    } else if (PUBLISH && !L.drop_publish) {
      if (r == 0) st_relaxed(pub_tile + c, nk);
      if (r == g.h - 1) st_relaxed(pub_tile + LB + c, nk);
    }
    if (L.tc == 1) {
      if (c == 0) sm.K[(r + 1) * P + g.w + 1] = nk - 2ull;
      if (c == g.w - 1) sm.K[(r + 1) * P] = nk + 2ull;
    } else if (PUBLISH && !L.drop_publish) {
      if (c == 0) st_relaxed(pub_tile + 2 * LB + r, nk);
      if (c == g.w - 1) st_relaxed(pub_tile + 3 * LB + r, nk);
    }
  }
}

// Fill the halo ring: neighbour edge words (+adj) or the mirrored own cells.
template <int LB, bool RELAXED>
__device__ __forceinline__ void fill_halo(const Smem<LB>& sm, const HaloSlot& hs) {
  if (hs.slot < 0) return;
  if (hs.mirror >= 0) {
    sm.K[hs.slot] = sm.K[hs.mirror] + (unsigned long long)hs.adj;
  } else {
    const unsigned long long v = RELAXED ? ld_relaxed(hs.src) : __ldg(hs.src);
    sm.K[hs.slot] = v + (unsigned long long)hs.adj;
  }
}

// Write the tile's boundary cells to its edge words (after a round-kernel launch).
template <int LB>
__device__ __forceinline__ void write_edges(const Smem<LB>& sm, const Geom& g,
                                            unsigned long long* pub_tile) {
  constexpr int P = TileShape<LB>::P;
  const int e = threadIdx.x / LB, p = threadIdx.x % LB;
  if (e < 2) {
    if (p < g.w) pub_tile[e * LB + p] = sm.K[(e == 0 ? 1 : g.h) * P + p + 1];
  } else {
    if (p < g.h) pub_tile[e * LB + p] = sm.K[(p + 1) * P + (e == 2 ? 1 : g.w)];
  }
}

// ------------------------------------------------------------------- kernels

__global__ void init_kernel(LatDesc L, int init_mode) {
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const Philox4 b0 = philox_event((uint32_t)c, 0u, 0u, L.seed_lo, L.seed_hi);
    unsigned up;
    if (init_mode == 1) up = 1u;
    else if (init_mode == 2) up = 0u;
    else {
      const uint32_t x = philox_event((uint32_t)c, 0u, 1u, L.seed_lo, L.seed_hi).x;
      up = (L.model == 1) ? (x < L.life_density ? 1u : 0u) : (x & 1u);   // Life: alive with the given density
    }
    unsigned long long t0 = exp_ticks(b0.x, L.two);
    if (L.rates) t0 = rated_gap(t0, L.rates[c]);
    L.key[c] = (t0 << 1) | up;
    L.cnt[c] = 0u;
  }
}

// Copy every tile's boundary cells from key[] into its edge words.
template <int LB>
__global__ void __launch_bounds__(4 * LB) publish_kernel(const LatDesc* __restrict__ lats, int nlat,
                                                         int to_pub2) {
  const int tile = blockIdx.x;
  const LatDesc& L = lats[find_lattice(lats, nlat, tile)];
  const int t = tile - L.tile_base;
  const Geom g = tile_geom(L, t);
  const int e = threadIdx.x / LB, p = threadIdx.x % LB;
  int r, c;
  if (e < 2) {
    if (p >= g.w) return;
    r = (e == 0) ? 0 : g.h - 1;
    c = p;
  } else {
    if (p >= g.h) return;
    r = p;
    c = (e == 2) ? 0 : g.w - 1;
  }
  unsigned long long* pub = to_pub2 ? L.pub2 : L.pub;
  pub[((size_t)t * 4 + e) * LB + p] = L.key[(size_t)(g.r0 + r) * L.cols + g.c0 + c];
}

// (a) Round kernel: R tile rounds per launch against frozen halos (edge words of
// the previous launch); R = 1 is one global synchronous round of Fig. 3.2.
template <int LB>
__global__ void __launch_bounds__(4 * LB) round_kernel(const LatDesc* __restrict__ lats, int nlat,
                                                       int R, int parity, int launch_idx,
                                                       DevCounters* ctr, unsigned long long* hist,
                                                       int hist_len, int round_idx) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Smem<LB> sm(smem_raw);
  if (launch_idx > 0) {
    if (*(volatile unsigned*)&ctr->active[(launch_idx + 2) % 3] == 0u) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr->active[(launch_idx + 1) % 3] = 0u;
    atomicAdd(&ctr->launched, 1u);
  }

  const int tile = blockIdx.x;
  const LatDesc& L = lats[find_lattice(lats, nlat, tile)];
  const int t = tile - L.tile_base;
  const Geom g = tile_geom(L, t);
  const unsigned long long* pub_in = parity ? L.pub2 : L.pub;
  unsigned long long* pub_out = (parity ? L.pub : L.pub2) + (size_t)t * 4 * LB;
  const unsigned long long t2 = L.t2;
  const bool direct = (R == 1);

  if (direct) load_interior<LB, false>(sm, L, g);
  else load_interior<LB, true>(sm, L, g);
  if (threadIdx.x < 10) sm.thr[threadIdx.x] = L.thr[threadIdx.x];
  if (threadIdx.x == 0) { sm.n_en[0] = 0u; sm.n_en[1] = 0u; }
  const HaloSlot hs = halo_slot<LB>(L, g, pub_in);
  __syncthreads();
  fill_halo<LB, false>(sm, hs);
  __syncthreads();

  unsigned long long scanned = 0, events = 0, rounds = 0, enabled = 0;
  int cur = 0;
  for (int rr = 0; rr < R; ++rr) {
    const bool live = scan_tile<LB>(sm, g, t2, &sm.n_en[cur], scanned);
    const int any_live = __syncthreads_or(live);
    const int n = (int)sm.n_en[cur];
    if (rr == 0 && threadIdx.x == 0 && hist != nullptr && round_idx < hist_len && n > 0)
      atomicAdd(&hist[round_idx], (unsigned long long)n);
    if (n == 0 || !any_live) break;
    if (direct) commit_tile<LB, true, false>(sm, L, g, nullptr, n);
    else commit_tile<LB, false, false>(sm, L, g, nullptr, n);
    if (threadIdx.x == 0) sm.n_en[cur ^ 1] = 0u;
    events += (unsigned long long)n;
    enabled += (unsigned long long)n;
    ++rounds;
    __syncthreads();
    cur ^= 1;
  }
  bool unfinished;
  if (direct) {
    unfinished = false;
    const int c = threadIdx.x % LB;
    if (c < g.w)
      for (int r = threadIdx.x / LB; r < g.h; r += 4)
        unfinished |= sm.K[(r + 1) * TileShape<LB>::P + c + 1] < t2;
  } else {
    unfinished = store_interior<LB, true>(sm, L, g);
  }
  write_edges<LB>(sm, g, pub_out);
  const int any_unfinished = __syncthreads_or(unfinished);
  // reduce the scanned counter over the block (only thread-local so far)
  for (int o = 16; o > 0; o >>= 1) scanned += __shfl_down_sync(kFull, scanned, o);
  if ((threadIdx.x & 31) == 0 && scanned) atomicAdd(&ctr->scanned, scanned);
  if (threadIdx.x == 0) {
    if (any_unfinished) atomicAdd(&ctr->active[launch_idx % 3], 1u);
    if (events) {
      atomicAdd(&ctr->events, events);
      atomicAdd(L.events, events);
    }
    if (enabled) atomicAdd(&ctr->enabled, enabled);
    if (rounds) atomicAdd(&ctr->rounds, rounds);
  }
}

// ---- early commits of certain rejections (the idea behind BKL, Sec. 3 "The BKL algorithm":
// at low temperature most arrivals change nothing).  A pending arrival whose flip decision is
// a rejection for every neighbour configuration still possible at its time may be committed
// before the neighbours that precede it: its spin does not change, so no neighbour's
// decision depends on whether it came first, and its new tick only lets neighbours that now
// precede it go ahead.  The neighbours that do not precede the cell keep their spins until
// after its arrival; those that precede it may still change, so the number j of up
// neighbours at the arrival lies in [fixed up, fixed up + preceding].  fmask[c] holds the j
// for which the cell's pending arrival would flip (bit j: u < thr[j + 5 (s > 0)], u the
// pending acceptance uniform): the arrival is a certain rejection iff no bit of that range
// is set.  Early commits can be adjacent to each other and to local minima, so the work list
// holds every cell; no order planes are kept (one synchronous round per launch).

// flip mask of the pending arrival of a cell with spin bit `up` and count n (block n + 1)
__device__ __forceinline__ unsigned flip_mask(uint32_t c, unsigned n, unsigned up, const unsigned* thr,
                                              uint32_t seed_lo, uint32_t seed_hi) {
  const uint32_t u = philox_event(c, n + 1u, 0u, seed_lo, seed_hi).y;
  unsigned m = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j) m |= (u < thr[j + 5 * up] ? 1u : 0u) << j;
  return m;
}

__global__ void fmask_kernel(LatDesc L) {
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x)
    L.fmask[c] = (unsigned char)flip_mask((uint32_t)c, L.cnt[c], (unsigned)L.key[c] & 1u, L.thr, L.seed_lo, L.seed_hi);
}

template <int LB>
struct TileShapeER {   // TileShape with a work list for every cell of the tile
  static constexpr int LIST = LB * LB;
  static constexpr size_t kBytes = TileShape<LB>::kBytes, cBytes = TileShape<LB>::cBytes;
  static constexpr size_t lBytes = ((size_t(LIST) * 2 + 15) / 16) * 16;
  static constexpr size_t bytes = kBytes + cBytes + lBytes + TileShape<LB>::mBytes;
};

// Enable test with early commits over the thread's column segment; list entries carry bit 15
// for an early commit (a certain rejection).  Returns whether any cell is still live.
template <int LB>
__device__ __forceinline__ bool scan_tile_er(unsigned long long* K, unsigned short* list, const LatDesc& L,
                                             const Geom& g, unsigned long long t2, unsigned int* n_slot,
                                             unsigned long long& scanned, unsigned long long& early) {
  constexpr int P = TileShape<LB>::P;
  const int c = threadIdx.x % LB;
  const int grp = threadIdx.x / LB;
  const int rpg = (g.h + 3) >> 2;
  const int rb = grp * rpg;
  const int re = min(g.h, rb + rpg);
  unsigned mask = 0, emask = 0;
  bool live_any = false;
  if (c < g.w && rb < re) {
    const unsigned long long* col = K + (rb + 1) * P + (c + 1);
    unsigned long long up = col[-P];
    unsigned long long cur = col[0];
    for (int r = rb; r < re; ++r) {
      const unsigned long long down = col[P];
      const unsigned long long left = col[-1];
      const unsigned long long right = col[1];
      const unsigned long long hi = cur | 1ull, lo = cur & ~1ull;
      const bool live = cur < t2;
      // the cell precedes each neighbour (the enable test of Fig. 3.2, term by term)
      const bool cu = hi < up, cl = hi < left, cr = lo <= right, cd = lo <= down;
      const bool en = live & cu & cl & cr & cd;
      bool er = false;
      if (live && !en) {
        const unsigned upfix = (cu ? (unsigned)up & 1u : 0u) + (cl ? (unsigned)left & 1u : 0u) +
                               (cr ? (unsigned)right & 1u : 0u) + (cd ? (unsigned)down & 1u : 0u);
        const unsigned unk = (cu ? 0u : 1u) + (cl ? 0u : 1u) + (cr ? 0u : 1u) + (cd ? 0u : 1u);
        const unsigned range = ((2u << unk) - 1u) << upfix;
        const size_t gi = ACI((size_t)(g.r0 + r) * L.cols + g.c0 + c, (long long)L.rows * L.cols, 28);
        er = (L.fmask[gi] & range) == 0u;
      }
      live_any |= live;
      mask |= (unsigned)(en | er) << (r - rb);
      emask |= (unsigned)er << (r - rb);
      up = cur;
      cur = down;
      col += P;
    }
    scanned += (unsigned long long)(re - rb);
    early += (unsigned long long)__popc(emask);
  }
  const int lane = threadIdx.x & 31;
  const int cnt = __popc(mask);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  int base = 0;
  if (lane == 31 && incl) base = (int)atomicAdd(n_slot, (unsigned)incl);
  base = __shfl_sync(kFull, base, 31);
  int off = base + incl - cnt;
  while (mask) {
    const int b = __ffs(mask) - 1;
    mask &= mask - 1;
    list[ACI(off++, TileShapeER<LB>::LIST, 29)] =
        (unsigned short)(((rb + b) << 8) | c | (((emask >> b) & 1u) << 15));
  }
  return live_any;
}

// One synchronous round of Fig. 3.2 per launch with early commits of certain rejections
// (keys and counts read from and written to HBM; halos from the previous launch's edge
// words).  Each commit also writes the flip mask of the cell's next pending arrival.
template <int LB>
__global__ void __launch_bounds__(4 * LB) round_er_kernel(const LatDesc* __restrict__ lats, int nlat, int parity,
                                                          int launch_idx, DevCounters* ctr) {
  using S = TileShapeER<LB>;
  constexpr int P = TileShape<LB>::P;
  constexpr int NT = TileShape<LB>::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* K = reinterpret_cast<unsigned long long*>(smem_raw);
  unsigned short* list = reinterpret_cast<unsigned short*>(smem_raw + S::kBytes + S::cBytes);
  unsigned int* n_en = reinterpret_cast<unsigned int*>(smem_raw + S::kBytes + S::cBytes + S::lBytes);
  unsigned int* thr = n_en + 2;
  if (launch_idx > 0) {
    if (*(volatile unsigned*)&ctr->active[(launch_idx + 2) % 3] == 0u) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctr->active[(launch_idx + 1) % 3] = 0u;
    atomicAdd(&ctr->launched, 1u);
  }
  const int tile = blockIdx.x;
  const LatDesc& L = lats[find_lattice(lats, nlat, tile)];
  const int t = tile - L.tile_base;
  const Geom g = tile_geom(L, t);
  const unsigned long long* pub_in = parity ? L.pub2 : L.pub;
  unsigned long long* pub_out = (parity ? L.pub : L.pub2) + (size_t)t * 4 * LB;
  const unsigned long long t2 = L.t2;
  {
    const int c = threadIdx.x % LB;
    if (c < g.w)
      for (int r = threadIdx.x / LB; r < g.h; r += 4)
        K[(r + 1) * P + c + 1] = L.key[ACI((size_t)(g.r0 + r) * L.cols + g.c0 + c, (long long)L.rows * L.cols, 21)];
  }
  if (threadIdx.x < 10) thr[threadIdx.x] = L.thr[threadIdx.x];
  if (threadIdx.x == 0) n_en[0] = 0u;
  const Smem<LB> sm(smem_raw);   // K and the halo layout of the tile engine
  const HaloSlot hs = halo_slot<LB>(L, g, pub_in);
  __syncthreads();
  fill_halo<LB, false>(sm, hs);
  __syncthreads();

  unsigned long long scanned = 0, early = 0;
  const bool live = scan_tile_er<LB>(K, list, L, g, t2, &n_en[0], scanned, early);
  const int any_live = __syncthreads_or(live);
  const int n = (int)n_en[0];
  if (n > 0 && any_live) {
    for (int i = threadIdx.x; i < n; i += NT) {
      const unsigned e = list[ACI(i, S::LIST, 29)];
      const bool er = (e >> 15) & 1u;
      const int r = (int)((e >> 8) & 127u), c = (int)(e & 255u);
      ACK(r < g.h && c < g.w, 25, e);
      unsigned long long* kp = K + (r + 1) * P + (c + 1);
      const unsigned long long key = *kp;
      const unsigned sp = (unsigned)key & 1u;
      const uint32_t gidx = (uint32_t)ACI((uint32_t)(g.r0 + r) * (uint32_t)L.cols + (uint32_t)(g.c0 + c),
                                          (long long)L.rows * L.cols, 26);
      const unsigned n_old = L.cnt[gidx];
      const Philox4 b = philox_event(gidx, n_old + 1u, 0u, L.seed_lo, L.seed_hi);
      unsigned flip = 0u;
      if (!er) {   // a local minimum: the heat-bath decision on the neighbours' spins
        const unsigned j = ((unsigned)kp[-P] & 1u) + ((unsigned)kp[P] & 1u) + ((unsigned)kp[-1] & 1u) +
                           ((unsigned)kp[1] & 1u);
        flip = b.y < thr[ACI(j + 5u * sp, 10, 9)] ? 1u : 0u;
      }
      unsigned long long gap = exp_ticks(b.x, L.two);
      if (L.rates) gap = rated_gap(gap, L.rates[gidx]);
      const unsigned ns = sp ^ flip;
      const unsigned long long nk = (key & ~1ull) + (gap << 1) + ns;
      *kp = nk;
      if (L.f_open) write_frames(frame_view(L), gidx, key >> 1, nk >> 1, ns);
      L.key[gidx] = nk;
      L.cnt[gidx] = n_old + 1u;
      L.fmask[gidx] = (unsigned char)flip_mask(gidx, n_old + 1u, ns, thr, L.seed_lo, L.seed_hi);
      if (L.tr == 1) {                    // vertical self-wrap: keep the mirrored halo rows live
        if (r == 0) K[(g.h + 1) * P + c + 1] = nk - 2ull;
        if (r == g.h - 1) K[c + 1] = nk + 2ull;
      }
      if (L.tc == 1) {
        if (c == 0) K[(r + 1) * P + g.w + 1] = nk - 2ull;
        if (c == g.w - 1) K[(r + 1) * P] = nk + 2ull;
      }
    }
    __syncthreads();
  }
  bool unfinished = false;
  {
    const int c = threadIdx.x % LB;
    if (c < g.w)
      for (int r = threadIdx.x / LB; r < g.h; r += 4) unfinished |= K[(r + 1) * P + c + 1] < t2;
  }
  write_edges<LB>(sm, g, pub_out);
  const int any_unfinished = __syncthreads_or(unfinished);
  for (int o = 16; o > 0; o >>= 1) {
    scanned += __shfl_down_sync(kFull, scanned, o);
    early += __shfl_down_sync(kFull, early, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (scanned) atomicAdd(&ctr->scanned, scanned);
    if (early) atomicAdd(&ctr->early, early);
  }
  if (threadIdx.x == 0) {
    if (any_unfinished) atomicAdd(&ctr->active[launch_idx % 3], 1u);
    if (n > 0 && any_live) {
      atomicAdd(&ctr->events, (unsigned long long)n);
      atomicAdd(L.events, (unsigned long long)n);
      atomicAdd(&ctr->enabled, (unsigned long long)n);
      atomicAdd(&ctr->rounds, 1ull);
    }
  }
}

// (b) Blocked persistent kernel (cooperative launch: all CTAs co-resident).
template <int LB>
__global__ void __launch_bounds__(4 * LB) blocked_kernel(const LatDesc* __restrict__ lats, int nlat,
                                                         int total_tiles, int polls, int refresh,
                                                         int max_rounds, long long watchdog_ns,
                                                         unsigned int* tile_done, DevCounters* ctr) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Smem<LB> sm(smem_raw);
  unsigned long long scanned = 0, events = 0, rounds = 0, visits = 0, npolls = 0;
  unsigned long long last_progress = global_ns();
  bool failed = false;

  for (;;) {
    bool any_left = false, progressed = false;
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      if (*(volatile unsigned*)&tile_done[tile]) continue;
      any_left = true;
      const LatDesc& L = lats[find_lattice(lats, nlat, tile)];
      const int t = tile - L.tile_base;
      const Geom g = tile_geom(L, t);
      const unsigned long long t2 = L.t2;
      unsigned long long* pub_tile = L.pub + (size_t)t * 4 * LB;

      load_interior<LB, true>(sm, L, g);
      if (threadIdx.x < 10) sm.thr[threadIdx.x] = L.thr[threadIdx.x];
      if (threadIdx.x == 0) { sm.n_en[0] = 0u; sm.n_en[1] = 0u; }
      const HaloSlot hs = halo_slot<LB>(L, g, L.pub);
      __syncthreads();
      fill_halo<LB, true>(sm, hs);
      __syncthreads();
      ++visits;

      int cur = 0, stuck = 0, vrounds = 0;
      bool done = false;
      unsigned long long vevents = 0;
      for (;;) {
        const bool live = scan_tile<LB>(sm, g, t2, &sm.n_en[cur], scanned);
        const int any_live = __syncthreads_or(live);
        const int n = (int)sm.n_en[cur];
        if (n == 0) {
          if (!any_live) { done = true; break; }
          // blocked on the halo: poll the neighbours' edge words and rescan only
          // once one of them has moved (a rescan with an unchanged halo finds nothing)
          bool moved = false;
          for (;;) {
            if (stuck >= polls) break;
            ++stuck;
            ++npolls;
            __nanosleep(256u << min(stuck, 4));
            bool mine = false;
            if (hs.src) {
              const unsigned long long v = ld_relaxed(hs.src) + (unsigned long long)hs.adj;
              if (v != sm.K[hs.slot]) {
                sm.K[hs.slot] = v;
                mine = true;
              }
            }
            if (__syncthreads_or(mine)) {
              moved = true;
              break;
            }
          }
          if (!moved) break;
          continue;
        }
        stuck = 0;
        const bool do_refresh = (refresh > 0) && ((vrounds + 1) % refresh == 0) && hs.src;
        unsigned long long fresh = 0;
        if (do_refresh) fresh = ld_relaxed(hs.src);        // latency hidden by the commit phase
        commit_tile<LB, false, true>(sm, L, g, pub_tile, n);
        if (threadIdx.x == 0) sm.n_en[cur ^ 1] = 0u;
        vevents += (unsigned long long)n;
        ++vrounds;
        __syncthreads();
        cur ^= 1;
        if (refresh > 0 && (vrounds % refresh) == 0) {
          if (do_refresh) sm.K[hs.slot] = fresh + (unsigned long long)hs.adj;
          __syncthreads();
        }
        if (max_rounds > 0 && vrounds >= max_rounds) break;
      }
      store_interior<LB, true>(sm, L, g);
      if (threadIdx.x == 0) {
        if (done) tile_done[tile] = 1u;
        if (vevents) atomicAdd(L.events, vevents);
      }
      events += vevents;
      rounds += (unsigned long long)vrounds;
      if (vevents) progressed = true;
      // one barrier both ends the visit and makes the error decision uniform
      if (__syncthreads_or(threadIdx.x == 0 && *(volatile int*)&ctr->error != 0)) {
        failed = true;
        break;
      }
    }
    if (failed || !any_left) break;
    int stall = 0;
    if (threadIdx.x == 0) {
      const unsigned long long now = global_ns();
      if (progressed) {
        last_progress = now;
      } else if ((long long)(now - last_progress) > watchdog_ns) {
        if (atomicCAS(&ctr->error, 0, 4 /* AC_ERR_STALL */) == 0) ctr->err_block = (int)blockIdx.x;
        stall = 1;
      }
    }
    if (__syncthreads_or(stall)) break;
  }
  for (int o = 16; o > 0; o >>= 1) scanned += __shfl_down_sync(kFull, scanned, o);
  if ((threadIdx.x & 31) == 0 && scanned) atomicAdd(&ctr->scanned, scanned);
  if (threadIdx.x == 0) {
    atomicAdd(&ctr->events, events);
    atomicAdd(&ctr->enabled, events);
    atomicAdd(&ctr->rounds, rounds);
    atomicAdd(&ctr->visits, visits);
    atomicAdd(&ctr->polls, npolls);
  }
}


// ----------------------------------------------------------------------------
// (a) Temporal-blocked round kernel.  A CTA loads an RW x RW region (RW = 96, two
// CTAs per SM, or 128, one) -- its tile of side at most RW - 2D plus a halo of depth
// D around it, wrapped on the torus -- from the input state buffer, runs R <= D
// synchronous rounds in shared memory and writes the tile to the output buffer
// (ping-pong, so every launch reads one consistent state).  Round k scans the
// region minus its outer k rings: a cell at distance d from the region's edge
// follows the global synchronous schedule for d rounds, so after R rounds the tile
// is exactly where R global rounds of Fig. 3.2 would put it, while the halo's
// commits (redundant with the neighbouring tiles) are discarded.  In a region that
// wraps, halo cells from across the torus seam carry key + 2 (seam above / left of
// the tile) or key - 2 (below / right): comparisons between two cells on the same
// side are unchanged, and between the sides they give the (tick, index) order of
// the seam (the Life variant compares lattice indices there instead).  Counts are
// held as 16-bit offsets from the tile centre's count.  Requires rows, cols >= 4D
// (the region never overlaps itself).  Every model tests enablement on order planes
// (one bit per lattice edge): see order_update (4-neighbour array), moore_order_update
// (Life automaton, q = 2 diamond) and q3_order_update (q = 3 diamond, 128-wide only).
template <int RW>
struct TbCfg {
  static constexpr int NT = 4 * RW;               // 384 or 512 threads
  static constexpr int LSTRIDE = NT / RW;         // load / store mapping: rows per column sweep
  // enabled cells form an independent set of the scanned rectangle (at most
  // (RW-2) x (RW-2) cells): the list holds every one of them, so a round always
  // commits all enabled cells and every tile advances exactly R synchronous rounds
  static constexpr int LIST = ((RW - 2) * (RW - 2) + 1) / 2 + 32;
  static constexpr int MIN_CTAS = (RW <= 96) ? 2 : 1;
  // keys with one guard row above and two below (the unrolled scan reads neighbours of
  // masked-out rows), 16-bit counts relative to a per-region base, work list, tables
  static constexpr size_t kBytes = size_t(RW + 3) * RW * 8;
  static constexpr size_t cBytes = size_t(RW) * RW * 2;
  static constexpr size_t lBytes = size_t(LIST) * 2;
  static constexpr size_t gBytes = size_t(RW) * 4 * 2;
  static constexpr size_t mBytes = (4 + kThrMax) * 4;   // n_en[2], overflow flag, thresholds
  // order planes: 32 cells per word, one word row per region row; H, V, LV for the
  // 4-neighbour array, the two diagonals as well for the Moore neighbourhood, and the
  // two edges of length 2 as well for the q = 2 diamond (7 planes); the q = 3 diamond
  // (12 edge directions and LV, 13 planes) runs on the 128-wide region only
  static constexpr int W = RW / 32;
  static constexpr int PLANES = (RW == 128) ? 13 : 7;
  static constexpr size_t pOff = kBytes + cBytes + lBytes + gBytes + mBytes;
  static constexpr size_t pBytes = size_t(PLANES) * RW * W * 4;
  static constexpr size_t fBytes = 64;            // snapshot-frame view (frame variant), 16-byte aligned
  static constexpr size_t fOff = (pOff + pBytes + 15) / 16 * 16;
  static constexpr size_t bytes = fOff + fBytes;
  static_assert(RW % 32 == 0 && pOff % 4 == 0, "order-plane layout");
};

// Order planes of the 4-neighbour array (one bit per lattice edge, packed 32 cells to a
// word): H bit (i, j) says cell (i, j) is live (its tick below the commit bound) and
// precedes its right neighbour in (tick, index) order, V bit (i, j) that it is live and
// precedes the cell below.  Cell (i, j) is enabled (Fig. 3.2) iff H(i, j) and V(i, j)
// are set and H(i, j-1), V(i-1, j) are clear, so a round's enable test is a few word
// operations per 32 cells.  Folding liveness into the planes changes no decision: a cell
// past the bound precedes no live cell, so clearing its bits never frees a live
// neighbour, and its own clear bits keep it from being enabled.  An edge's bit changes
// only when one of its two cells commits (a cell's liveness changes only with its own
// key), and the cells committed in one round are pairwise non-adjacent, so every bit has
// at most one writer per round.  A committed cell's old bits are known (it was enabled),
// so it updates them with xor masks.  (LV is unused here; the other models keep it.)
__device__ __forceinline__ void order_update(unsigned* H, unsigned* V, unsigned* LV, int W, int r, int c,
                                             unsigned long long nk, unsigned long long kl, unsigned long long kr,
                                             unsigned long long ku, unsigned long long kd, unsigned long long t2) {
  const unsigned long long lo = nk & ~1ull;
  const bool live = nk < t2;
  const unsigned bit = 1u << (c & 31);
  const int wc = r * W + (c >> 5);
  const unsigned hc = (live && lo <= kr) ? 0u : bit;   // no longer (live and) before the right neighbour
  const bool hl = (kl & ~1ull) <= nk && kl < t2;       // the (live) left neighbour now precedes it
  if (c & 31) {
    const unsigned m = hc | (hl ? (bit >> 1) : 0u);
    if (m) atomicXor(&H[wc], m);
  } else {                                             // the left edge's bit is in the previous word
    if (hc) atomicXor(&H[wc], hc);
    if (hl) atomicXor(&H[wc - 1], 0x80000000u);
  }
  if (!(live && lo <= kd)) atomicXor(&V[wc], bit);
  if ((ku & ~1ull) <= nk && ku < t2) atomicXor(&V[wc - W], bit);
}

// (tick, lattice index) order of two cells from their keys and indices: the exact order
// in a region that wraps across the torus seam, where region order is not index order.
__device__ __forceinline__ bool precedes_exact(unsigned long long ka, unsigned ga, unsigned long long kb, unsigned gb) {
  const unsigned long long ta = ka >> 1, tb = kb >> 1;
  return ta < tb || (ta == tb && ga < gb);
}

__device__ __forceinline__ void plane_flip(unsigned* P, int W, int r, int c, bool flip) {
  if (flip) atomicXor(&P[r * W + (c >> 5)], 1u << (c & 31));
}

// Order planes of the Moore neighbourhood (Life-like automaton): besides H (right) and V
// (below), SE bit (i, j) says cell (i, j) precedes (i+1, j+1) and SW bit (i, j) that it
// precedes (i+1, j-1).  Cell (i, j) is enabled iff its own H, V, SE, SW and LV bits are
// set and H(i, j-1), V(i-1, j), SE(i-1, j-1), SW(i-1, j+1) are clear.  Enabled cells
// are at Chebyshev distance >= 2, so each edge bit has at most one writer per round; a
// committed cell flips those of its 8 edges whose order changed (its own four were set,
// the four towards earlier cells clear).  With exact = false the region does not wrap
// and region order is index order, so a key compare with the index tie rule decides.
// FAR adds the q = 2 diamond's edges of length 2: H2 bit (i, j) says the cell precedes
// (i, j+2), V2 bit (i, j) that it precedes (i+2, j) (12 edges per cell; enabled cells
// of the diamond are more than 2 apart, so again one writer per edge and round).
template <int RW, bool FAR>
__device__ __forceinline__ void moore_order_update(unsigned* OH, unsigned* OV, unsigned* OL, unsigned* OSE,
                                                   unsigned* OSW, unsigned* OH2, unsigned* OV2, int r, int c,
                                                   unsigned long long nk, unsigned gc, const unsigned long long* kp,
                                                   bool exact, const unsigned* rowoff, const unsigned* colg,
                                                   unsigned long long t2) {
  constexpr int W = RW / 32;
  if (FAR) {
    const unsigned long long kl2 = kp[-2], kr2 = kp[2], ku2 = kp[-2 * RW], kd2 = kp[2 * RW];
    bool h2_c, h2_l, v2_c, v2_u;
    if (exact) {
      const unsigned r1 = rowoff[r], c1 = colg[c];
      h2_c = precedes_exact(nk, gc, kr2, r1 + colg[c + 2]);
      h2_l = precedes_exact(kl2, r1 + colg[c - 2], nk, gc);
      v2_c = precedes_exact(nk, gc, kd2, rowoff[r + 2] + c1);
      v2_u = precedes_exact(ku2, rowoff[r - 2] + c1, nk, gc);
    } else {
      const unsigned long long lo = nk & ~1ull;
      h2_c = lo <= kr2;
      h2_l = (kl2 & ~1ull) <= nk;
      v2_c = lo <= kd2;
      v2_u = (ku2 & ~1ull) <= nk;
    }
    plane_flip(OH2, W, r, c, !h2_c);
    plane_flip(OH2, W, r, c - 2, h2_l);
    plane_flip(OV2, W, r, c, !v2_c);
    plane_flip(OV2, W, r - 2, c, v2_u);
  }
  const unsigned long long kl = kp[-1], kr = kp[1], ku = kp[-RW], kd = kp[RW];
  const unsigned long long kul = kp[-RW - 1], kur = kp[-RW + 1], kdl = kp[RW - 1], kdr = kp[RW + 1];
  bool e_c, e_l, s_c, s_u, se_c, se_ul, sw_c, sw_ur;
  if (exact) {
    const unsigned r0 = rowoff[r - 1], r1 = rowoff[r], r2 = rowoff[r + 1];
    const unsigned c0 = colg[c - 1], c1 = colg[c], c2 = colg[c + 1];
    e_c = precedes_exact(nk, gc, kr, r1 + c2);
    e_l = precedes_exact(kl, r1 + c0, nk, gc);
    s_c = precedes_exact(nk, gc, kd, r2 + c1);
    s_u = precedes_exact(ku, r0 + c1, nk, gc);
    se_c = precedes_exact(nk, gc, kdr, r2 + c2);
    se_ul = precedes_exact(kul, r0 + c0, nk, gc);
    sw_c = precedes_exact(nk, gc, kdl, r2 + c0);
    sw_ur = precedes_exact(kur, r0 + c2, nk, gc);
  } else {
    const unsigned long long lo = nk & ~1ull;
    e_c = lo <= kr;
    e_l = (kl & ~1ull) <= nk;
    s_c = lo <= kd;
    s_u = (ku & ~1ull) <= nk;
    se_c = lo <= kdr;
    se_ul = (kul & ~1ull) <= nk;
    sw_c = lo <= kdl;
    sw_ur = (kur & ~1ull) <= nk;
  }
  plane_flip(OH, W, r, c, !e_c);
  plane_flip(OH, W, r, c - 1, e_l);
  plane_flip(OV, W, r, c, !s_c);
  plane_flip(OV, W, r - 1, c, s_u);
  plane_flip(OSE, W, r, c, !se_c);
  plane_flip(OSE, W, r - 1, c - 1, se_ul);
  plane_flip(OSW, W, r, c, !sw_c);
  plane_flip(OSW, W, r - 1, c + 1, sw_ur);
  if (nk >= t2) atomicAnd(&OL[r * W + (c >> 5)], ~(1u << (c & 31)));
}

// The q = 3 diamond's 12 forward edge directions (dr, dc): the neighbours within
// Manhattan distance 3 that come later in region order.  Plane d holds, for each cell,
// whether it precedes its neighbour at (i + dr, j + dc); plane 12 is LV.
__device__ __forceinline__ constexpr int q3_dr(int d) { return d < 3 ? 0 : (d < 8 ? 1 : (d < 11 ? 2 : 3)); }
__device__ __forceinline__ constexpr int q3_dc(int d) { return d < 3 ? d + 1 : (d < 8 ? d - 5 : (d < 11 ? d - 9 : 0)); }

// Order planes of the q = 3 diamond (128-wide region): a cell is enabled iff its 12 own
// bits and LV are set and, for every direction d, the bit of the cell at (i - dr, j - dc)
// is clear.  Enabled cells are more than 3 apart, so each edge has at most one writer
// per round; a committed cell flips the changed bits of its 24 edges.
template <int RW>
__device__ __forceinline__ void q3_order_update(unsigned* OQ, int r, int c, unsigned long long nk, unsigned gc,
                                                const unsigned long long* kp, bool exact, const unsigned* rowoff,
                                                const unsigned* colg, unsigned long long t2) {
  constexpr int W = RW / 32;
#pragma unroll
  for (int d = 0; d < 12; ++d) {
    const int dr = q3_dr(d), dc = q3_dc(d);
    unsigned* P = OQ + d * RW * W;
    const unsigned long long kf = kp[dr * RW + dc], kb = kp[-dr * RW - dc];
    bool own, back;
    if (exact) {
      own = precedes_exact(nk, gc, kf, rowoff[r + dr] + colg[c + dc]);
      back = precedes_exact(kb, rowoff[r - dr] + colg[c - dc], nk, gc);
    } else {
      own = (nk & ~1ull) <= kf;
      back = (kb & ~1ull) <= nk;
    }
    plane_flip(P, W, r, c, !own);
    plane_flip(P, W, r - dr, c - dc, back);
  }
  if (nk >= t2) atomicAnd(&OQ[12 * RW * W + r * W + (c >> 5)], ~(1u << (c & 31)));
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---- epoch kernel: bulk asynchronous copies (the TMA unit) completing on an mbarrier,
// and the release / acquire words that order tiles across CTAs.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// global -> shared, the box at element (x, y) of a 2D tensor map (a 128-byte map in global
// memory); x times the element size a multiple of 16 bytes, the destination 128-byte aligned
__device__ __forceinline__ void tensor_box_load(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
// orders this thread's earlier generic-proxy accesses before its later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int wrap_index(int x, int n, int& shift, int up_shift) {
  // x in [-n, 2n): wrapped index; shift = +up_shift if x came from below 0, -up_shift if >= n
  if (x < 0) {
    shift = up_shift;
    return x + n;
  }
  if (x >= n) {
    shift = -up_shift;
    return x - n;
  }
  shift = 0;
  return x;
}

// Bulk copies of the region's key rows [i0, i1) into K, issued by the 32 lanes of one
// warp: one copy per row, two where the row crosses the torus seam (columns x0 .. Lcols-1,
// then 0 .. RC-n1-1).  Region row i is torus row r0D + i (wrapped).
template <int RW>
__device__ __forceinline__ void bulk_key_rows(unsigned long long* K, const unsigned long long* key_in, int i0, int i1,
                                              int r0D, int Lrows, int Lcols, int x0, int n1, int RC, size_t Ncells,
                                              unsigned long long* bar, int lane) {
  for (int i = i0 + lane; i < i1; i += 32) {
    int shr;
    const int gr = wrap_index(r0D + i, Lrows, shr, 2);
    const unsigned long long* src = key_in + (size_t)gr * (size_t)Lcols;
    ACK((size_t)gr * Lcols + x0 + n1 <= Ncells && (x0 & 1) == 0 && (n1 & 1) == 0 && (Lcols & 1) == 0, 4, i);
    ACK(i * RW + RC <= (RW + 2) * RW, 5, i);
    bulk_load(&K[i * RW], src + x0, (unsigned)n1 * 8u, bar);
    if (n1 < RC) bulk_load(&K[i * RW + n1], src, (unsigned)(RC - n1) * 8u, bar);
  }
}

// Bounded wait for the mbarrier phase of `parity`; true if it gave up (2 s).
__device__ __forceinline__ bool bulk_wait(unsigned long long* bar, unsigned parity) {
  unsigned long long t0 = 0;
  for (unsigned n = 0; !mbar_try_wait(bar, parity); ++n) {
    if ((n & 1023u) != 1023u) continue;
    const unsigned long long now = global_ns();
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > 2000000000ull) {
      return true;
    }
  }
  return false;
}

// ---- Life-like automaton on the Moore neighbourhood (the deterministic update of
// Sec. 3, e.g. Conway's Game of Life): a cell may commit once its key is below the
// keys of all 8 Moore neighbours (its update reads all of them), so enabled cells
// are pairwise at Chebyshev distance >= 2 and the same shrinking-region argument as
// for the 4-neighbour array holds.  The enable test reads order planes (see
// moore_order_update).

// live cells among the 8 Moore neighbours of the region cell at kp
template <int RW>
__device__ __forceinline__ unsigned moore_live(const unsigned long long* kp) {
  return ((unsigned)kp[-RW - 1] & 1u) + ((unsigned)kp[-RW] & 1u) + ((unsigned)kp[-RW + 1] & 1u) +
         ((unsigned)kp[-1] & 1u) + ((unsigned)kp[1] & 1u) + ((unsigned)kp[RW - 1] & 1u) +
         ((unsigned)kp[RW] & 1u) + ((unsigned)kp[RW + 1] & 1u);
}

// ---- Ising array on the q-th degree neighbourhood (Sec. 3): every cell within
// Manhattan distance q is a neighbour; a cell may commit once its key is below all of
// theirs.  Enabled cells are then more than q apart, so commits never read each other.

// up spins among the diamond of radius q around the region cell at kp
template <int RW>
__device__ __forceinline__ unsigned q_up(const unsigned long long* kp, int q) {
  unsigned j = 0;
  for (int dr = -q; dr <= q; ++dr) {
    const int rem = q - (dr < 0 ? -dr : dr);
    for (int dx = -rem; dx <= rem; ++dx)
      if (dr != 0 || dx != 0) j += (unsigned)kp[dr * RW + dx] & 1u;
  }
  return j;
}

// ---- epoch kernel control (one thread claims and publishes; nine threads check the
// nine dependencies of an item)

// tile of work item k: epoch k / total, position k % total in the work list, rotated
// by half the list on odd epochs
__device__ __forceinline__ int ep_tile(unsigned k, int total, int* epoch) {
  const int e = (int)(k / (unsigned)total);
  const int j = (int)(k - (unsigned)e * (unsigned)total);
  *epoch = e;
  return (e & 1) ? (j + total / 2) % total : j;
}

// done word of dependency n (0..8: the tile and its 8 neighbours on the torus of
// tiles) of item k, and the epoch it must have reached; nullptr for epoch 0
__device__ __forceinline__ const unsigned* ep_dep(const LatDesc* lats, int nlat, int total, const EpArgs& ep,
                                                  unsigned k, int n, unsigned* need) {
  int epoch;
  const int tile = ep_tile(k, total, &epoch);
  *need = (unsigned)epoch;
  if (epoch == 0) return nullptr;
  const LatDesc& L = lats[find_lattice(lats, nlat, tile)];
  const int t = tile - L.tile_base;
  int ti = t / L.tc + n / 3 - 1, tj = t % L.tc + n % 3 - 1;
  ti = ti < 0 ? ti + L.tr : (ti >= L.tr ? ti - L.tr : ti);
  tj = tj < 0 ? tj + L.tc : (tj >= L.tc ? tj - L.tc : tj);
  ACK(L.tile_base + ti * L.tc + tj < total, 14, tile);
  return ep.done + L.tile_base + ti * L.tc + tj;
}

// the claim word: next item (low half), stop epoch (high half)
__device__ __forceinline__ unsigned long long* ep_claim_word(DevCounters* ctr) {
  return reinterpret_cast<unsigned long long*>(&ctr->next_item);
}

// claim the next item (~0: none left, an error was reported, or the run has finished)
__device__ __forceinline__ unsigned ep_claim(DevCounters* ctr, const EpArgs& ep, int total) {
  if (*(volatile int*)&ctr->error != 0) return ~0u;
  const unsigned long long w = atomicAdd(ep_claim_word(ctr), 1ull);
  const unsigned k = (unsigned)w, e = k / (unsigned)total;
  return (e >= (unsigned)ep.max_epochs || e >= (unsigned)(w >> 32)) ? ~0u : k;
}

// stop epoch = min(stop epoch, s) in the claim word's high half (claims change only the low
// half; a bounded compare-and-swap loop -- a stop epoch that is not set only costs identity
// epochs up to the launch's epoch budget)
__device__ __forceinline__ void ep_set_stop(DevCounters* ctr, unsigned s) {
  unsigned long long* cw = ep_claim_word(ctr);
  unsigned long long old = *(volatile unsigned long long*)cw;
  for (int it = 0; it < 4096 && (unsigned)(old >> 32) > s; ++it) {
    const unsigned long long seen = atomicCAS(cw, old, ((unsigned long long)s << 32) | (old & 0xFFFFFFFFull));
    if (seen == old) break;
    old = seen;
  }
}

// Publish item kp (~0: none) and claim the next item, their global-memory round trips in
// flight together.  Publishing: its tile has completed epoch e + 1 (the CTA's stores
// precede this call on its barrier; fence, then release the done word), and one atomic
// adds the tile to epoch e's count and, if live, to its live count; the tile that
// completes the epoch sees every other tile's live flag in the value it gets back and
// ends the run if none has an arrival before t_end left.  Claiming: as ep_claim (an item
// claimed while an error is reported is dropped).
__device__ __forceinline__ unsigned ep_publish_claim(const LatDesc* lats, int nlat, int total, const EpArgs& ep,
                                                     DevCounters* ctr, unsigned kp, bool live, bool claim,
                                                     bool fenced = false) {
  unsigned long long old = 0;
  int pe = -1;
  if (kp != ~0u) {
    const int tile = ep_tile(kp, total, &pe);
    // (fenced: the caller's fence after the CTA's barrier already orders the tile's stores,
    // and a relaxed store completes the release)
    if (!fenced) __threadfence();
    // (the verification hook that suppresses edge publication also withholds the epoch
    // words, so that the neighbours' bounded waits and the watchdog end the run)
    ACK(tile >= 0 && tile < total && pe < ep.max_epochs, 13, tile);
    if (!lats[find_lattice(lats, nlat, tile)].drop_publish) {
      if (fenced)
        st_relaxed_u32(&ep.done[tile], (unsigned)pe + 1u);
      else
        st_release_u32(&ep.done[tile], (unsigned)pe + 1u);
    }
    old = atomicAdd(&ep.ep_count[pe], (1ull << 32) | (live ? 1ull : 0ull));
  }
  int err = 0;
  unsigned long long w = ~0ull;
  if (claim) {
    err = *(volatile int*)&ctr->error;
    w = atomicAdd(ep_claim_word(ctr), 1ull);
  }
  if (pe >= 0 && (unsigned)(old >> 32) == (unsigned)total - 1u && (unsigned)old + (live ? 1u : 0u) == 0u)
    ep_set_stop(ctr, (unsigned)pe + 1u);
  if (!claim) return ~0u;
  // refused only by the stop epoch the claim itself returned: a later claim sees the same
  // or a smaller stop epoch, so every accepted item's dependencies (claimed earlier) were
  // accepted too, and none waits on an item nobody runs
  const unsigned k = (unsigned)w, e = k / (unsigned)total;
  return (err != 0 || e >= (unsigned)ep.max_epochs || e >= (unsigned)(w >> 32)) ? ~0u : k;
}

// publish item k (see ep_publish_claim)
__device__ __forceinline__ void ep_publish(const LatDesc* lats, int nlat, int total, const EpArgs& ep,
                                           DevCounters* ctr, unsigned k, bool live) {
  ep_publish_claim(lats, nlat, total, ep, ctr, k, live, false);
}

// threads 0..8: wait until dependency `tid` of item k is met -- bounded polls, then sleeps,
// a %globaltimer watchdog, and an early exit when another CTA has reported an error.
// Returns true if the wait gave up.
__device__ __forceinline__ bool ep_wait(const LatDesc* lats, int nlat, int total, const EpArgs& ep, DevCounters* ctr,
                                     unsigned k, int tid) {
  unsigned need;
  const unsigned* f = ep_dep(lats, nlat, total, ep, k, tid, &need);
  if (f == nullptr) return false;
  unsigned long long t0 = 0;
  unsigned n = 0;
  bool gave_up = false;
  for (; ld_acquire_u32(f) < need; ++n) {
    if (n < 32) continue;
    __nanosleep(n < 256 ? 64 : 512);
    if (*(volatile int*)&ctr->error != 0) {
      gave_up = true;
      break;
    }
    const unsigned long long now = global_ns();
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > (unsigned long long)ep.watchdog_ns) {
      atomicCAS(&ctr->error, 0, 4 /* AC_ERR_STALL */);
      atomicExch(&ctr->err_block, (int)blockIdx.x);
      gave_up = true;
      break;
    }
  }
  if (n) atomicAdd(&ctr->polls, (unsigned long long)n);
  return gave_up;
}

// FR: snapshot frames are open (write_frames for the tile's own cells).
// MODEL: 0 the Ising heat bath; 1 the Life-like automaton (Moore neighbourhood, birth /
// survival masks in thr[0] / thr[1]); 2 the Ising heat bath on the q-th degree
// neighbourhood (radius L.q; the region shrinks by q rings per round).
// EP: the epoch kernel.  Instead of one pass over the tiles per launch, a persistent
// grid claims (epoch, tile) work items in increasing order from ctr->next_item.  Item
// (e, t) advances tile t from the state of epoch e (buffer e & 1) to that of epoch
// e + 1 (the other buffer), exactly what launch e of the launch variant does for it.
// Its region covers the tile and parts of its 8 neighbour tiles, so it waits until
// all 9 have published done >= e (acquire), and publishes done = e + 1 (release) after
// its stores.  This is the aggregated algorithm of Fig. 3.4 with a tile per subarray
// and a tile's completed epoch as the local time its neighbours wait on.  Every item
// waits only on items claimed before it, so the schedule cannot deadlock, whatever
// the number of resident CTAs.  Within an epoch, items go in work-list order, rotated
// by half the list on odd epochs, so that an item's dependencies were claimed about
// half an epoch earlier.  Region keys arrive by the TMA unit (one 2D tensor copy for a
// region inside the lattice, row copies across the torus seam; through L2, never a stale
// L1 line); counts are read with ld.global.cg.  A CTA holds its claims one visit ahead,
// and the control work overlaps the region load: while the copy and the count loads are
// in flight, warp 1 publishes the CTA's previous item and claims the item after the next
// one, and warp 2 checks the next item's nine dependencies once; only if that check fails
// does the CTA, at the top of its next visit, publish at once and wait (so it never waits
// on itself).
// RATES: some lattice of the launch has per-cell rates (otherwise the commits skip the
// rate test).
template <int RW, bool FR, int MODEL, bool EP, bool RATES = true>
__global__ void __launch_bounds__(TbCfg<RW>::NT, TbCfg<RW>::MIN_CTAS)
    tb_kernel(const LatDesc* __restrict__ lats, int nlat, int total_tiles, int D, int R, DevCounters* ctr,
              EpArgs ep) {
  static_assert(!(EP && FR), "the epoch kernel does not write snapshot frames");
  using Cfg = TbCfg<RW>;
  constexpr int NT = Cfg::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* K = reinterpret_cast<unsigned long long*>(smem_raw) + RW;   // row 0
  unsigned short* C = reinterpret_cast<unsigned short*>(smem_raw + Cfg::kBytes);
  unsigned short* list = reinterpret_cast<unsigned short*>(smem_raw + Cfg::kBytes + Cfg::cBytes);
  unsigned int* rowoff = reinterpret_cast<unsigned int*>(smem_raw + Cfg::kBytes + Cfg::cBytes + Cfg::lBytes);
  unsigned int* colg = rowoff + RW;
  unsigned int* misc = colg + RW;
  unsigned int* n_en = misc;          // [2]
  unsigned int* s_over = misc + 2;    // count window overflow in this region
  unsigned int* thr = misc + 4;       // [kThrMax]
  unsigned int* OH = reinterpret_cast<unsigned int*>(smem_raw + Cfg::pOff);   // order planes
  unsigned int* OV = OH + RW * Cfg::W;
  unsigned int* OL = OV + RW * Cfg::W;
  unsigned int* OSE = OL + RW * Cfg::W;
  unsigned int* OSW = OSE + RW * Cfg::W;
  unsigned int* OH2 = OSW + RW * Cfg::W;
  unsigned int* OV2 = OH2 + RW * Cfg::W;
  FrameView* fv = reinterpret_cast<FrameView*>(smem_raw + Cfg::fOff);
  static_assert(sizeof(FrameView) <= Cfg::fBytes, "frame view does not fit");
  // the epoch kernel keeps its mbarrier and the claimed item where the frame view sits
  unsigned long long* ep_bar = reinterpret_cast<unsigned long long*>(smem_raw + Cfg::fOff);
  unsigned int* ep_ctl = reinterpret_cast<unsigned int*>(smem_raw + Cfg::fOff + 8);
  // ep_ctl: [0] next item, [1] its dependencies were met at the early check,
  //         [2] current item, [3] previous item not yet published, [4] its live flag,
  //         [5] 0x10 | phase of a region load whose wait timed out (0: none),
  //         [6] the item after the next one, [7] the one claimed during this visit's load
  //         (a CTA holds its claims in claim order and runs them in that order, so the
  //         smallest unfinished claimed item is always at the head of its CTA's queue)

  const int tid = threadIdx.x;
  // this launch's number, advanced by the last CTA of the previous launch
  unsigned launch_idx = 0;
  int parity = 0;
  if constexpr (!EP) {
    launch_idx = *(volatile unsigned*)&ctr->seq;
    parity = (int)(launch_idx & 1u);
    if (launch_idx > 0) {
      // nothing left, or an earlier launch of this call hit the count window (its output
      // is not a consistent state, so no later launch may build on it): uniform exit
      if (*(volatile unsigned*)&ctr->active[(launch_idx + 2) % 3] == 0u || *(volatile int*)&ctr->error != 0)
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctr->active[(launch_idx + 1) % 3] = 0u;
      if (FR) ctr->kmin[(launch_idx + 1) % 3] = ~0ull;
      atomicAdd(&ctr->launched, 1u);
    }
  } else {
    // the count check of the call: every lattice's count range must fit the 16-bit window
    // (a refused launch claims no item: the work loop below then ends at once)
    bool wide = false;
    for (int i = tid; i < ep.nrange; i += NT) wide |= ep.range[2 * i + 1] - ep.range[2 * i] >= ep.limit;
    wide = __syncthreads_or(wide) != 0;
    if (tid == 0) {
      mbar_init(ep_bar);
      if (wide && blockIdx.x == 0) atomicCAS(&ctr->error, 0, kEpWindow);
      ep_ctl[0] = wide ? ~0u : ep_claim(ctr, ep, total_tiles);
      ep_ctl[6] = ep_ctl[0] == ~0u ? ~0u : ep_claim(ctr, ep, total_tiles);
      ep_ctl[7] = ~0u;
      ep_ctl[1] = 0u;
      ep_ctl[3] = ~0u;
      ep_ctl[5] = 0u;
    }
    __syncthreads();
  }
  const int lane = tid & 31;
  const int lj = tid % RW, li0 = tid / RW;                 // load / store mapping: column, first row
  unsigned ep_phase = 0;                                   // epoch kernel: mbarrier phase of the next load

  for (int tile_it = blockIdx.x;; tile_it += gridDim.x) {
    int tile = tile_it;
    if constexpr (EP) {
      // the item claimed during the previous visit (or before the first one)
      const unsigned k = ep_ctl[0];
      if (k == ~0u) break;
      if (!ep_ctl[1]) {
        // its dependencies were not all met at the early check: publish the previous
        // item first (it may be one of them), then wait
        if (tid == 0 && ep_ctl[3] != ~0u) {
          ep_publish(lats, nlat, total_tiles, ep, ctr, ep_ctl[3], ep_ctl[4] != 0u);
          ep_ctl[3] = ~0u;
        }
        // a wait that gives up has reported the error: the visit still runs (on a state
        // that is undefined from now on), and the next claim finds the error and ends the loop
        if (tid < 9) ep_wait(lats, nlat, total_tiles, ep, ctr, k, tid);
        __syncthreads();
      }
      int epoch;
      tile = ep_tile(k, total_tiles, &epoch);
      parity = epoch & 1;
      if (tid == 0) ep_ctl[2] = k;
    } else {
      if (tile >= total_tiles) break;
    }
    const LatDesc& L = lats[find_lattice(lats, nlat, tile)];
    const Geom g = tile_geom(L, tile - L.tile_base);
    // in registers: the copies below are asm statements that clobber memory
    const int Lrows = L.rows, Lcols = L.cols;
    const unsigned long long* key_in = parity ? L.key2 : L.key;
    const unsigned int* cnt_in = parity ? L.cnt2 : L.cnt;
    const int RH = g.h + 2 * D, RC = g.w + 2 * D;
    ACK(RH <= RW && RC <= RW && g.h >= 1 && g.w >= 1, 1, tile);
    ACK(RH <= Lrows && RC <= Lcols, 2, tile);   // the region never overlaps itself
    // lattice index of region cell (0, 0) when the region does not wrap (unused otherwise)
    const uint32_t g00 = (uint32_t)(g.r0 - D) * (uint32_t)Lcols + (uint32_t)(g.c0 - D);
    // the region wraps across the torus seam (small tiles of interior positions can too)
    const bool edge = (g.r0 < D) || (g.r0 + g.h + D > Lrows) || (g.c0 < D) || (g.c0 + g.w + D > Lcols);
    // the tile centre (its count starts the region's 16-bit count window)
    const size_t ci = (size_t)(g.r0 + g.h / 2) * Lcols + g.c0 + g.w / 2;
    const size_t Ncells = (size_t)Lrows * (size_t)Lcols;
    const unsigned cap = 65535u - (unsigned)R;

    // ---- load the region: keys by asynchronous copies, counts through registers
    if (tid == 0) {
      n_en[0] = 0u;
      n_en[1] = 0u;
      s_over[0] = 0u;
      if (FR) *fv = frame_view(L);
    }
    int shc;
    const int gc = wrap_index(g.c0 - D + lj, Lcols, shc, 2);
    bool over = false;
    __syncthreads();
    if constexpr (EP) {
      if (!edge && L.tmap != nullptr && ((g.c0 - D) & 1) == 0) {
        // a region inside the lattice: one 2D tensor copy of the RW x RW box at its first
        // cell (the box's rows and columns past the region arrive too, zeros past the
        // lattice's edge, and are never read)
        if (tid == 0) {
          mbar_expect_tx(ep_bar, (unsigned)(RW * RW) * 8u);
          fence_proxy_async();
          tensor_box_load(K, static_cast<const unsigned char*>(L.tmap) + ((RW == 128 ? 2 : 0) + parity) * kTmapBytes,
                          g.c0 - D, g.r0 - D, ep_bar);
        }
      } else if (tid < 32) {
        // a region across the torus seam: one warp issues its rows as bulk copies, one per
        // row, two where the row crosses the seam (even cols, an even region start and an
        // even width keep every source, destination and size a multiple of 16 bytes)
        if (tid == 0) mbar_expect_tx(ep_bar, (unsigned)(RH * RC) * 8u);
        __syncwarp();
        fence_proxy_async();
        int shx;
        const int x0 = wrap_index(g.c0 - D, Lcols, shx, 2);
        bulk_key_rows<RW>(K, key_in, 0, RH, g.r0 - D, Lrows, Lcols, x0, min(RC, Lcols - x0), RC, Ncells, ep_bar, tid);
      }
      // the next warp's first lane fences before its count loads (the tile's stores of
      // the previous visit are then visible), publishes the previous item once the loads
      // are in flight, and claims the item after the next one (claimed a visit ahead)
      if (tid == 32 && ep_ctl[3] != ~0u) __threadfence();
    }
    // counts are kept as 16-bit offsets from a window start taken at the tile centre; the
    // thread's own-tile cells' offsets at load are summed (against the sum at the
    // write-back, it gives the tile's committed arrivals)
    const bool own_col = lj >= D && lj < D + g.w;
    unsigned base = 0, own_before = 0;
    {
      // the centre count (every thread loads it) and the thread's counts: one batch of
      // loads in flight together (the launch kernel's key copies too)
      const unsigned ccen = EP ? __ldcg(&cnt_in[ACI(ci, Ncells, 3)]) : __ldg(&cnt_in[ACI(ci, Ncells, 3)]);
      base = ccen > 32768u ? ccen - 32768u : 0u;
      if constexpr (EP) {
        // the epoch kernel loads two adjacent counts per thread (8-byte loads: the region's
        // first column, its width and the lattice's columns are even, so a pair never
        // crosses the torus seam): thread (pj, pi0) takes columns 2 pj, 2 pj + 1 of rows
        // pi0 + PSTRIDE m
        constexpr int PW = RW / 2, PSTRIDE = NT / PW, PROWS = RW / PSTRIDE;
        const int pj = tid % PW, pi0 = tid / PW, cj = 2 * pj;
        uint2 cv2[PROWS];
        if (cj < RC) {
          int shp;
          const int gcp = wrap_index(g.c0 - D + cj, Lcols, shp, 2);
          int shr0;
          int gr = wrap_index(g.r0 - D + pi0, Lrows, shr0, 2);
#pragma unroll
          for (int m = 0; m < PROWS; ++m) {
            const int i = pi0 + PSTRIDE * m;
            if (i < RH) {
              const uint32_t gi = (uint32_t)ACI((uint32_t)gr * (uint32_t)Lcols + (uint32_t)gcp, Ncells - 1, 3);
              cv2[m] = __ldcg(reinterpret_cast<const uint2*>(&cnt_in[gi]));
            }
            gr += PSTRIDE;
            if (gr >= Lrows) gr -= Lrows;
          }
        }
        if (tid == 32) {
          ep_ctl[7] = ep_publish_claim(lats, nlat, total_tiles, ep, ctr, ep_ctl[3], ep_ctl[4] != 0u, ep_ctl[6] != ~0u,
                                       true);
          ep_ctl[3] = ~0u;
        }
        if (tid >= 64 && tid < 96) {
          // with its counts in flight, warp 2 checks the next item's dependencies once
          // (acquire loads: they order only what follows them)
          const int lw = tid - 64;
          const unsigned kn = ep_ctl[6];
          bool met = true;
          if (kn != ~0u && lw < 9) {
            unsigned need;
            const unsigned* f = ep_dep(lats, nlat, total_tiles, ep, kn, lw, &need);
            met = (f == nullptr) || ld_acquire_u32(f) >= need;
          }
          met = __all_sync(kFull, met);
          if (lw == 0) ep_ctl[1] = met ? 1u : 0u;
        }
        if (cj < RC) {
          const bool own_p = cj >= D && cj < D + g.w;   // both columns or neither (D, w even)
#pragma unroll
          for (int m = 0; m < PROWS; ++m) {
            const int i = pi0 + PSTRIDE * m;
            if (i < RH) {
              const unsigned a = cv2[m].x - base, b = cv2[m].y - base;
              over |= (a > cap) | (b > cap);
              *reinterpret_cast<unsigned*>(&C[i * RW + cj]) = (a & 0xFFFFu) | (b << 16);
              if (own_p && i >= D && i < D + g.h) own_before += a + b;
            }
          }
        }
      } else if (lj < RC) {
        constexpr int MROWS = RW / Cfg::LSTRIDE;
        unsigned cvs[MROWS];
        int shr0;
        int gr = wrap_index(g.r0 - D + li0, Lrows, shr0, 2);   // the wrapped lattice row, stepped
#pragma unroll
        for (int m = 0; m < MROWS; ++m) {
          const int i = li0 + Cfg::LSTRIDE * m;
          if (i < RH) {
            const uint32_t gi = (uint32_t)ACI((uint32_t)gr * (uint32_t)Lcols + (uint32_t)gc, Ncells, 3);
            if constexpr (!EP) cp_async8(&K[i * RW + lj], &key_in[gi]);
            cvs[m] = EP ? __ldcg(&cnt_in[gi]) : cnt_in[gi];
          }
          gr += Cfg::LSTRIDE;
          if (gr >= Lrows) gr -= Lrows;
        }
#pragma unroll
        for (int m = 0; m < MROWS; ++m) {
          const int i = li0 + Cfg::LSTRIDE * m;
          if (i < RH) {
            const unsigned cv = cvs[m] - base;
            over |= cv > cap;
            C[i * RW + lj] = (unsigned short)cv;
            if (own_col && i >= D && i < D + g.h) own_before += cv;
          }
        }
      }
    }
    if (tid < RW) {
      int sh;
      rowoff[tid] = (unsigned)wrap_index(min(g.r0 - D + tid, 2 * Lrows - 1), Lrows, sh, 2) * (unsigned)Lcols;
      colg[tid] = (unsigned)wrap_index(min(g.c0 - D + tid, 2 * Lcols - 1), Lcols, sh, 2);
    } else if (tid < RW + kThrMax) {
      thr[tid - RW] = L.thr[tid - RW];
    }
    if (over) atomicOr(s_over, 1u);
    if constexpr (EP) {
      // the region's bulk copies: bounded wait on the mbarrier phase of this load
      if (bulk_wait(ep_bar, ep_phase)) {   // reported; its copies are waited on again before the CTA exits
        atomicCAS(&ctr->error, 0, 4 /* AC_ERR_STALL */);
        ep_ctl[5] = 0x10u | ep_phase;
      }
      ep_phase ^= 1u;
      __syncthreads();
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    if (edge && MODEL == 0) {   // halo cells from across the torus seam: key +-2 (one tick of tie order)
      if (lj < RC) {
        for (int i = li0; i < RH; i += Cfg::LSTRIDE) {
          int shr;
          wrap_index(g.r0 - D + i, Lrows, shr, 2);
          if (shr + shc) K[i * RW + lj] += (unsigned long long)(long long)(shr + shc);
        }
      }
      __syncthreads();
    }
    if constexpr (EP) {
      // the claimed items move up (every reader of these slots is behind a barrier)
      if (tid == 0) {
        ep_ctl[0] = ep_ctl[6];
        ep_ctl[6] = ep_ctl[7];
      }
    }
    if (s_over[0]) {
      // the counts of this region do not fit the 16-bit window (the host checks the
      // lattice's count range first, so this is a safety net): flag the launch; the
      // host then discards its output and keeps the launch's input state
      if (tid == 0) atomicCAS(&ctr->error, 0, 5 /* AC_ERR_STATE */);
      __syncthreads();
      continue;
    }

    // ---- R synchronous rounds over the shrinking region
    // (the visit's statistics are added to the counters at its end: 32-bit accumulators)
    unsigned scanned = 0, enabled = 0, rounds_done = 0;
    const unsigned long long t2 = L.t2;
    const uint32_t two = L.two, seed_lo = L.seed_lo, seed_hi = L.seed_hi;
    // (the per-cell rate array is read through the descriptor at each commit: a pointer kept
    // in registers across the commit loop costs spills)
    constexpr int W = Cfg::W;
    const int qn = (MODEL == 2) ? L.q : 1;     // rings lost per round
    // the q = 3 diamond has its own 13 planes and runs on the 128-wide region only (the
    // host routes it there); a 96-wide launch of it is refused, uniformly per CTA
    const bool q3 = MODEL == 2 && qn == 3;
    if (q3 && RW != 128) {
      if (tid == 0) atomicCAS(&ctr->error, 0, 1 /* AC_ERR_ARG */);
      break;
    }
    unsigned* OQ = OH;   // plane d of the q = 3 diamond at OQ + d * RW * W, LV at d = 12
    if (q3) {
      for (int i = li0; i < RW; i += Cfg::LSTRIDE) {
        const unsigned long long kc = K[i * RW + lj];
        const unsigned gc = edge ? rowoff[i] + colg[lj] : 0u;
#pragma unroll
        for (int d = 0; d < 12; ++d) {
          const int dr = q3_dr(d), dc = q3_dc(d);
          const unsigned long long kn = K[(i + dr) * RW + lj + dc];
          const bool pr = edge ? precedes_exact(kc, gc, kn, rowoff[i + dr] + colg[lj + dc]) : (kc & ~1ull) <= kn;
          const unsigned b = __ballot_sync(kFull, pr);
          if (lane == 0) OQ[d * RW * W + i * W + (lj >> 5)] = b;
        }
        const unsigned lb = __ballot_sync(kFull, kc < t2);
        if (lane == 0) OQ[12 * RW * W + i * W + (lj >> 5)] = lb;
      }
      __syncthreads();
    } else {
      // order planes of the loaded region; a warp covers 32 consecutive columns of one
      // row, and a thread RW / LSTRIDE consecutive rows (the key below a row is the next
      // row's own key).  Relations with cells outside the loaded rectangle are never read
      // (the reads past the region's last row and column stay inside shared memory).
      constexpr int RPT = RW / Cfg::LSTRIDE;
      unsigned long long kcarry = K[li0 * RPT * RW + lj];
      for (int i = li0 * RPT; i < (li0 + 1) * RPT; ++i) {
        const unsigned long long kc = kcarry;
        const unsigned long long kr = K[i * RW + lj + 1];
        const unsigned long long kd = K[(i + 1) * RW + lj];
        kcarry = kd;
        bool ph, pv, pse = false, psw = false, ph2 = false, pv2 = false;
        if (MODEL != 0 && edge) {   // wider neighbourhoods across the seam: exact order
          const unsigned gc = rowoff[i] + colg[lj], gd = rowoff[i + 1];
          ph = precedes_exact(kc, gc, kr, rowoff[i] + colg[lj + 1]);
          pv = precedes_exact(kc, gc, kd, gd + colg[lj]);
          pse = precedes_exact(kc, gc, K[(i + 1) * RW + lj + 1], gd + colg[lj + 1]);
          psw = precedes_exact(kc, gc, K[(i + 1) * RW + lj - 1], gd + colg[lj - 1]);
          if (MODEL == 2) {
            ph2 = precedes_exact(kc, gc, K[i * RW + lj + 2], rowoff[i] + colg[lj + 2]);
            pv2 = precedes_exact(kc, gc, K[(i + 2) * RW + lj], rowoff[i + 2] + colg[lj]);
          }
        } else {
          const unsigned long long lo = kc & ~1ull;
          ph = lo <= kr;
          pv = lo <= kd;
          if (MODEL != 0) {
            pse = lo <= K[(i + 1) * RW + lj + 1];
            psw = lo <= K[(i + 1) * RW + lj - 1];
          }
          if (MODEL == 2) {
            ph2 = lo <= K[i * RW + lj + 2];
            pv2 = lo <= K[(i + 2) * RW + lj];
          }
        }
        // the 4-neighbour array folds the bound into its two planes (a cell at or past the
        // bound precedes nobody): H and V bits of a cell are set only while it is live
        const bool lv = kc < t2;
        const unsigned hb = __ballot_sync(kFull, MODEL == 0 ? (ph && lv) : ph);
        const unsigned vb = __ballot_sync(kFull, MODEL == 0 ? (pv && lv) : pv);
        const unsigned lb = MODEL == 0 ? 0u : __ballot_sync(kFull, lv);
        unsigned seb = 0u, swb = 0u, h2b = 0u, v2b = 0u;
        if (MODEL != 0) {
          seb = __ballot_sync(kFull, pse);
          swb = __ballot_sync(kFull, psw);
        }
        if (MODEL == 2) {
          h2b = __ballot_sync(kFull, ph2);
          v2b = __ballot_sync(kFull, pv2);
        }
        if (lane == 0) {
          const int wi = i * W + (lj >> 5);
          OH[wi] = hb;
          OV[wi] = vb;
          if (MODEL != 0) OL[wi] = lb;
          if (MODEL != 0) {
            OSE[wi] = seb;
            OSW[wi] = swb;
          }
          if (MODEL == 2) {
            OH2[wi] = h2b;
            OV2[wi] = v2b;
          }
        }
      }
      __syncthreads();
    }
    int cur = 0;
    for (int k = 1; k <= R; ++k) {
      const int kk = k * qn;
      unsigned mask = 0;
      // the word scanned by this thread (4-neighbour array): row oi, columns 32 ow ...
      const int oi = tid / W, ow = tid % W;
      {
        if (oi < RW && oi >= kk && oi < RH - kk) {
          const int lo = max(kk - 32 * ow, 0), hi = min(RC - kk - 32 * ow, 32);
          if (hi > lo) {
            const unsigned cm = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
            const int wi = oi * W + ow, wu = wi - W;
            ACK(wi >= qn * W && wi < RW * W, 7, wi);   // the words qn rows up exist
            const unsigned h = OH[wi];
            const unsigned hl = (h << 1) | (ow > 0 ? (OH[wi - 1] >> 31) : 0u);
            unsigned m = h & ~hl & OV[wi] & ~OV[wu] & cm;
            if (MODEL != 0) m &= OL[wi];
            if (MODEL != 0) {   // the diagonals: SE of the up-left cell, SW of the up-right cell
              const unsigned seu = (OSE[wu] << 1) | (ow > 0 ? (OSE[wu - 1] >> 31) : 0u);
              const unsigned swu = (OSW[wu] >> 1) | (ow + 1 < W ? (OSW[wu + 1] << 31) : 0u);
              m &= OSE[wi] & OSW[wi] & ~seu & ~swu;
            }
            if (MODEL == 2 && !q3) {   // q = 2: H2 of the cell two to the left, V2 of the cell two above
              const unsigned h2 = OH2[wi];
              const unsigned h2l = (h2 << 2) | (ow > 0 ? (OH2[wi - 1] >> 30) : 0u);
              m &= h2 & ~h2l & OV2[wi] & ~OV2[wu - W];
            }
            if (q3) {   // the q = 3 diamond: its own planes, each against the cell d back
              m = OQ[12 * RW * W + wi] & cm;
#pragma unroll
              for (int d = 0; d < 12; ++d) {
                const int dr = q3_dr(d), dc = q3_dc(d);
                const unsigned* P = OQ + d * RW * W;
                const int wb = wi - dr * W;
                unsigned back = P[wb];
                if (dc > 0) back = (back << dc) | (ow > 0 ? (P[wb - 1] >> (32 - dc)) : 0u);
                if (dc < 0) back = (back >> -dc) | (ow + 1 < W ? (P[wb + 1] << (32 + dc)) : 0u);
                m &= P[wi] & ~back;
              }
            }
            mask = m;
            scanned += (unsigned)__popc(cm);
          }
        }
      }
      // exclusive prefix of the per-lane counts by an inclusive warp scan
      const int cnt = __popc(mask);
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      const int excl = incl - cnt;
      int wbase = 0;
      if (lane == 0 && total) wbase = (int)atomicAdd(&n_en[cur], (unsigned)total);
      wbase = __shfl_sync(kFull, wbase, 0);
      // the lane's entries, two per iteration (the list holds every enabled cell: they
      // form an independent set of the scanned rectangle)
      int off = wbase + excl;
      const unsigned ebase = (unsigned)((oi << 8) | (32 * ow));
      while (mask) {
        const unsigned m2 = mask & (mask - 1);
        list[ACI(off, Cfg::LIST, 6)] = (unsigned short)(ebase + (unsigned)__ffs(mask) - 1u);
        if (m2) list[ACI(off + 1, Cfg::LIST, 6)] = (unsigned short)(ebase + (unsigned)__ffs(m2) - 1u);
        mask = m2 & (m2 - 1);
        off += 2;
      }
      __syncthreads();
      const int n = min((int)n_en[cur], Cfg::LIST);
      if (n == 0) break;
      // two commits per iteration: all shared-memory reads first, then two independent
      // Philox / exp_ticks chains the compiler can interleave, then the writes
      // (listed cells are pairwise non-adjacent, so the two never touch each other)
      int e_i = tid;
      for (; e_i + NT < n; e_i += 2 * NT) {
        const unsigned ea = list[ACI(e_i, Cfg::LIST, 6)], eb = list[ACI(e_i + NT, Cfg::LIST, 6)];
        const int ra = (int)(ea >> 8), ca = (int)(ea & 255u), rb = (int)(eb >> 8), cb = (int)(eb & 255u);
        ACK(ra >= kk && ra < RH - kk && ca >= kk && ca < RC - kk, 8, ea);
        ACK(rb >= kk && rb < RH - kk && cb >= kk && cb < RC - kk, 8, eb);
        unsigned long long* kpa = K + ra * RW + ca;
        unsigned long long* kpb = K + rb * RW + cb;
        const unsigned long long keya = *kpa, keyb = *kpb;
        const unsigned spa = (unsigned)keya & 1u, spb = (unsigned)keyb & 1u;
        uint32_t gia, gib;
        if (edge) {
          gia = rowoff[ra] + colg[ca];
          gib = rowoff[rb] + colg[cb];
        } else {   // the region does not wrap: lattice index from the region's first cell
          gia = g00 + (uint32_t)(ra * Lcols + ca);
          gib = g00 + (uint32_t)(rb * Lcols + cb);
        }
        const unsigned c16a = C[ra * RW + ca], c16b = C[rb * RW + cb];
        // the 4-neighbour array's neighbour keys, read once for the heat-bath sum and the
        // order planes (no commit of this round writes a neighbour of a listed cell)
        unsigned long long nua = 0, nda = 0, nla = 0, nra = 0, nub = 0, ndb = 0, nlb = 0, nrb = 0;
        if (MODEL == 0) {
          nua = kpa[-RW];
          nda = kpa[RW];
          nla = kpa[-1];
          nra = kpa[1];
          nub = kpb[-RW];
          ndb = kpb[RW];
          nlb = kpb[-1];
          nrb = kpb[1];
        }
        unsigned tha, thb;
        if (MODEL == 1) {   // rule mask of the current state; the new state is its bit k
          tha = thr[spa];
          thb = thr[spb];
        } else if (MODEL == 2) {
          const unsigned M1 = 2u * qn * (qn + 1) + 1u;
          tha = thr[ACI(q_up<RW>(kpa, qn) + M1 * spa, kThrMax, 9)];
          thb = thr[ACI(q_up<RW>(kpb, qn) + M1 * spb, kThrMax, 9)];
        } else {
          tha = thr[ACI(((unsigned)nua & 1u) + ((unsigned)nda & 1u) + ((unsigned)nla & 1u) + ((unsigned)nra & 1u) + 5u * spa, 10, 9)];
          thb = thr[ACI(((unsigned)nub & 1u) + ((unsigned)ndb & 1u) + ((unsigned)nlb & 1u) + ((unsigned)nrb & 1u) + 5u * spb, 10, 9)];
        }
        ACK(gia < Ncells && gib < Ncells, 10, gia);
        const Philox4 pa = philox_event(gia, base + c16a + 1u, 0u, seed_lo, seed_hi);
        const Philox4 pb = philox_event(gib, base + c16b + 1u, 0u, seed_lo, seed_hi);
        unsigned long long gapa = exp_ticks(pa.x, two), gapb = exp_ticks(pb.x, two);
        if (RATES && L.rates) {
          gapa = rated_gap(gapa, L.rates[gia]);
          gapb = rated_gap(gapb, L.rates[gib]);
        }
        const unsigned nsa = MODEL == 1 ? (tha >> moore_live<RW>(kpa)) & 1u : spa ^ (pa.y < tha ? 1u : 0u);
        const unsigned nsb = MODEL == 1 ? (thb >> moore_live<RW>(kpb)) & 1u : spb ^ (pb.y < thb ? 1u : 0u);
        const unsigned long long nka = (keya & ~1ull) + (gapa << 1) + nsa;
        const unsigned long long nkb = (keyb & ~1ull) + (gapb << 1) + nsb;
        *kpa = nka;
        *kpb = nkb;
        C[ra * RW + ca] = (unsigned short)(c16a + 1u);
        C[rb * RW + cb] = (unsigned short)(c16b + 1u);
        if (MODEL == 0) {
          order_update(OH, OV, OL, W, ra, ca, nka, nla, nra, nua, nda, t2);
          order_update(OH, OV, OL, W, rb, cb, nkb, nlb, nrb, nub, ndb, t2);
        } else if (MODEL == 1) {
          moore_order_update<RW, false>(OH, OV, OL, OSE, OSW, OH2, OV2, ra, ca, nka, gia, kpa, edge, rowoff, colg, t2);
          moore_order_update<RW, false>(OH, OV, OL, OSE, OSW, OH2, OV2, rb, cb, nkb, gib, kpb, edge, rowoff, colg, t2);
        } else if (q3) {
          q3_order_update<RW>(OQ, ra, ca, nka, gia, kpa, edge, rowoff, colg, t2);
          q3_order_update<RW>(OQ, rb, cb, nkb, gib, kpb, edge, rowoff, colg, t2);
        } else {   // the q = 2 diamond
          moore_order_update<RW, true>(OH, OV, OL, OSE, OSW, OH2, OV2, ra, ca, nka, gia, kpa, edge, rowoff, colg, t2);
          moore_order_update<RW, true>(OH, OV, OL, OSE, OSW, OH2, OV2, rb, cb, nkb, gib, kpb, edge, rowoff, colg, t2);
        }
        if (FR) {   // own cells only: halo commits are repeated by the owning tile
          if (ra >= D && ra < D + g.h && ca >= D && ca < D + g.w)
            write_frames(*fv, gia, keya >> 1, nka >> 1, (unsigned)nka & 1u);
          if (rb >= D && rb < D + g.h && cb >= D && cb < D + g.w)
            write_frames(*fv, gib, keyb >> 1, nkb >> 1, (unsigned)nkb & 1u);
        }
      }
      if (e_i < n) {
        const unsigned e = list[ACI(e_i, Cfg::LIST, 6)];
        const int r = (int)(e >> 8), cc = (int)(e & 255u);
        ACK(r >= kk && r < RH - kk && cc >= kk && cc < RC - kk, 8, e);
        unsigned long long* kp = K + r * RW + cc;
        const unsigned long long key = *kp;
        const unsigned sp = (unsigned)key & 1u;
        const uint32_t gidx = rowoff[r] + colg[cc];
        ACK(gidx < Ncells, 10, gidx);
        const unsigned c16 = C[r * RW + cc];
        const Philox4 b = philox_event(gidx, base + c16 + 1u, 0u, seed_lo, seed_hi);
        unsigned ns;
        unsigned long long nu = 0, nd = 0, nl = 0, nr = 0;   // neighbour keys, read once
        if (MODEL == 1) {
          ns = (thr[sp] >> moore_live<RW>(kp)) & 1u;
        } else if (MODEL == 2) {
          const unsigned M1 = 2u * qn * (qn + 1) + 1u;
          ns = sp ^ (b.y < thr[ACI(q_up<RW>(kp, qn) + M1 * sp, kThrMax, 9)] ? 1u : 0u);
        } else {
          nu = kp[-RW];
          nd = kp[RW];
          nl = kp[-1];
          nr = kp[1];
          const unsigned j = ((unsigned)nu & 1u) + ((unsigned)nd & 1u) + ((unsigned)nl & 1u) + ((unsigned)nr & 1u);
          ns = sp ^ (b.y < thr[ACI(j + 5u * sp, 10, 9)] ? 1u : 0u);
        }
        unsigned long long gap = exp_ticks(b.x, two);
        if (RATES && L.rates) gap = rated_gap(gap, L.rates[gidx]);
        const unsigned long long nk = (key & ~1ull) + (gap << 1) + ns;
        *kp = nk;
        C[r * RW + cc] = (unsigned short)(c16 + 1u);
        if (MODEL == 0) order_update(OH, OV, OL, W, r, cc, nk, nl, nr, nu, nd, t2);
        if (MODEL == 1)
          moore_order_update<RW, false>(OH, OV, OL, OSE, OSW, OH2, OV2, r, cc, nk, gidx, kp, edge, rowoff, colg, t2);
        else if (MODEL == 2 && q3)
          q3_order_update<RW>(OQ, r, cc, nk, gidx, kp, edge, rowoff, colg, t2);
        else if (MODEL == 2)
          moore_order_update<RW, true>(OH, OV, OL, OSE, OSW, OH2, OV2, r, cc, nk, gidx, kp, edge, rowoff, colg, t2);
        if (FR && r >= D && r < D + g.h && cc >= D && cc < D + g.w)
          write_frames(*fv, gidx, key >> 1, nk >> 1, (unsigned)nk & 1u);
      }
      enabled += (unsigned)n;
      ++rounds_done;
      if (tid == 0) n_en[cur ^ 1] = 0u;
      __syncthreads();
      cur ^= 1;
    }

    // ---- write the tile back; count its arrivals; is anything left before t_end?
    bool live = false;
    unsigned long long ev = 0, kmin = ~0ull;
    unsigned own_after = 0;
    if constexpr (EP) {
      // the epoch kernel writes own cells in column pairs: 16-byte key and 8-byte count
      // stores (the tile's first column and width are even)
      constexpr int PW = RW / 2, PSTRIDE = NT / PW;
      const int pj = tid % PW, pi0 = tid / PW, cj = 2 * pj;
      if (cj >= D && cj < D + g.w) {
        unsigned long long* key_out = parity ? L.key : L.key2;
        unsigned int* cnt_out = parity ? L.cnt : L.cnt2;
        for (int ri = pi0; ri < D + g.h; ri += PSTRIDE) {
          if (ri < D) continue;
          const int si = ri * RW + cj;
          const uint32_t gi = (uint32_t)ACI((uint32_t)(g.r0 + ri - D) * (uint32_t)Lcols + (uint32_t)(g.c0 + cj - D), Ncells - 1, 11);
          const ulonglong2 kk = *reinterpret_cast<const ulonglong2*>(&K[si]);
          const unsigned c2 = *reinterpret_cast<const unsigned*>(&C[si]);
          const unsigned ca = c2 & 0xFFFFu, cb = c2 >> 16;
          own_after += ca + cb;
          *reinterpret_cast<ulonglong2*>(&key_out[gi]) = kk;
          *reinterpret_cast<uint2*>(&cnt_out[gi]) = make_uint2(base + ca, base + cb);
          live |= (kk.x < t2) | (kk.y < t2);
        }
      }
    } else if (own_col) {
      // own rows i = li0 + 4m - D for region rows li0 + 4m in [D, D + h)
      unsigned long long* key_out = parity ? L.key : L.key2;
      unsigned int* cnt_out = parity ? L.cnt : L.cnt2;
      for (int ri = li0; ri < D + g.h; ri += Cfg::LSTRIDE) {
        if (ri < D) continue;
        const int i = ri - D;
        const int si = ri * RW + lj;
        const uint32_t gi = (uint32_t)ACI((uint32_t)(g.r0 + i) * (uint32_t)Lcols + (uint32_t)(g.c0 + lj - D), Ncells, 11);
        ACK(si < RW * RW, 12, si);
        const unsigned long long kk = K[si];
        const unsigned c16 = C[si];
        own_after += c16;
        key_out[gi] = kk;
        cnt_out[gi] = base + c16;
        live |= kk < t2;
        if (FR) kmin = min(kmin, kk);
      }
    }
    // the tile's committed arrivals: summed over the CTA, the own cells' offsets at the
    // write-back less those at load (signed per thread: the epoch kernel loads counts in
    // column pairs, so a thread's cells at load and at the write-back differ)
    ev = (unsigned long long)((long long)own_after - (long long)own_before);
    if (FR) {   // the launch's smallest output key: frames below its tick are complete
      for (int o = 16; o > 0; o >>= 1) kmin = min(kmin, __shfl_down_sync(kFull, kmin, o));
      if (lane == 0 && kmin != ~0ull) atomicMin(&ctr->kmin[launch_idx % 3], kmin);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ev += __shfl_down_sync(kFull, ev, o);
      scanned += __shfl_down_sync(kFull, scanned, o);
    }
    if (lane == 0) {
      if (ev) {
        atomicAdd(L.events, ev);
        atomicAdd(&ctr->events, ev);
      }
      if (scanned) atomicAdd(&ctr->scanned, (unsigned long long)scanned);
    }
    if (tid == 0) {
      atomicAdd(&ctr->enabled, (unsigned long long)enabled);
      atomicAdd(&ctr->rounds, (unsigned long long)rounds_done);
    }
    const int any_live = __syncthreads_or(live);
    if constexpr (EP) {
      // the tile's stores are done (the barrier above); its epoch is published during the
      // next visit's load, or before the CTA waits or exits
      if (tid == 0) {
        ep_ctl[3] = ep_ctl[2];
        ep_ctl[4] = any_live ? 1u : 0u;
      }
    } else {
      if (tid == 0 && any_live) atomicAdd(&ctr->active[launch_idx % 3], 1u);
    }
  }
  __syncthreads();
  if (tid == 0) {
    if constexpr (EP) {
      if (ep_ctl[3] != ~0u) ep_publish(lats, nlat, total_tiles, ep, ctr, ep_ctl[3], ep_ctl[4] != 0u);
      if (ep_ctl[5]) {   // a region load timed out: wait once more (bounded) for its copies
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(ep_bar, ep_ctl[5] & 1u) && global_ns() - t0 < 2000000000ull) {
        }
      }
    } else {
      // the last CTA of this launch advances the launch number for the next one
      __threadfence();
      if (atomicAdd(&ctr->blocks_done, 1u) == gridDim.x - 1u) {
        ctr->blocks_done = 0u;
        __threadfence();
        atomicExch(&ctr->seq, launch_idx + 1u);
      }
    }
  }
}

// ---- observables, packing, device-primitive probes ---------------------------

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// out[0] = sum of spins, out[1] = sum over right and down bonds of s s',
// out[2] = state fingerprint sum_c mix(mix(mix(c) ^ t) ^ (2n + up)), out[3] = sum of counts.
__global__ void reduce_kernel(LatDesc L, unsigned long long* out) {
  const size_t N = (size_t)L.rows * L.cols;
  long long ms = 0, bonds = 0;
  unsigned long long fp = 0, ev = 0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const size_t r = c / L.cols, q = c - r * L.cols;
    const unsigned long long k = L.key[c];
    const int s = (k & 1ull) ? 1 : -1;
    const int sr = (L.key[r * L.cols + (q + 1 == (size_t)L.cols ? 0 : q + 1)] & 1ull) ? 1 : -1;
    const int sd = (L.key[(r + 1 == (size_t)L.rows ? 0 : r + 1) * L.cols + q] & 1ull) ? 1 : -1;
    const unsigned n = L.cnt[c];
    ms += s;
    bonds += s * sr + s * sd;
    unsigned long long z = mix64((unsigned long long)c);
    z = mix64(z ^ (k >> 1));
    z = mix64(z ^ (((unsigned long long)n << 1) | (k & 1ull)));
    fp += z;
    ev += n;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ms += __shfl_down_sync(kFull, ms, o);
    bonds += __shfl_down_sync(kFull, bonds, o);
    fp += __shfl_down_sync(kFull, fp, o);
    ev += __shfl_down_sync(kFull, ev, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], (unsigned long long)ms);
    atomicAdd(&out[1], (unsigned long long)bonds);
    atomicAdd(&out[2], fp);
    atomicAdd(&out[3], ev);
  }
}

// out[0] = min count, out[1] = max count (out initialised to {~0, 0} by the caller)
// BKL classes (Sec. 3): cells counted by spin and number j of up neighbours, index
// j + 5 (s > 0) as in the threshold table; block counters in shared memory.
__global__ void class_count_kernel(LatDesc L, unsigned long long* out) {
  __shared__ unsigned long long sc[10];
  if (threadIdx.x < 10) sc[threadIdx.x] = 0ull;
  __syncthreads();
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const size_t r = c / L.cols, q = c - r * L.cols;
    const size_t up = (r == 0 ? L.rows - 1 : r - 1) * L.cols + q, dn = (r + 1 == (size_t)L.rows ? 0 : r + 1) * L.cols + q;
    const size_t lf = r * L.cols + (q == 0 ? L.cols - 1 : q - 1), rt = r * L.cols + (q + 1 == (size_t)L.cols ? 0 : q + 1);
    const unsigned j = (unsigned)(L.key[up] & 1ull) + (unsigned)(L.key[dn] & 1ull) + (unsigned)(L.key[lf] & 1ull) +
                       (unsigned)(L.key[rt] & 1ull);
    atomicAdd(&sc[j + 5u * (unsigned)(L.key[c] & 1ull)], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 10 && sc[threadIdx.x]) atomicAdd(&out[threadIdx.x], sc[threadIdx.x]);
}

__global__ void count_range_kernel(LatDesc L, unsigned* out) {
  const size_t N = (size_t)L.rows * L.cols;
  unsigned mn = 0xFFFFFFFFu, mx = 0u;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const unsigned v = L.cnt[c];
    mn = min(mn, v);
    mx = max(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_down_sync(kFull, mn, o));
    mx = max(mx, __shfl_down_sync(kFull, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&out[0], mn);
    atomicMax(&out[1], mx);
  }
}

// out[2i] = min count, out[2i+1] = max count of lattice i (initialised to {~0, 0});
// blockIdx.y = lattice, blockIdx.x strides over its cells
__global__ void count_range_batch_kernel(const LatDesc* __restrict__ lats, unsigned* out) {
  const LatDesc& L = lats[blockIdx.y];
  const size_t N = (size_t)L.rows * L.cols;
  unsigned mn = 0xFFFFFFFFu, mx = 0u;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const unsigned v = L.cnt[c];
    mn = min(mn, v);
    mx = max(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_down_sync(kFull, mn, o));
    mx = max(mx, __shfl_down_sync(kFull, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&out[2 * blockIdx.y], mn);
    atomicMax(&out[2 * blockIdx.y + 1], mx);
  }
}

__global__ void unpack_kernel(LatDesc L, int8_t* s, long long* t, unsigned* n) {
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long k = L.key[c];
    if (s) s[c] = (k & 1ull) ? (int8_t)1 : (int8_t)-1;
    if (t) t[c] = (long long)(k >> 1);
    if (n) n[c] = L.cnt[c];
  }
}

__global__ void pack_kernel(LatDesc L, const int8_t* s, const long long* t, const unsigned* n) {
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    L.key[c] = ((unsigned long long)t[c] << 1) | (s[c] > 0 ? 1ull : 0ull);
    L.cnt[c] = n[c];
  }
}

// pack_kernel behind a device-side check: nothing is written unless *bad is still ~0 (the
// validation of the staged state, asynchronous loads)
__global__ void pack_checked_kernel(LatDesc L, const int8_t* s, const long long* t, const unsigned* n,
                                    const unsigned long long* bad) {
  if (*(volatile const unsigned long long*)bad != ~0ull) return;
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    L.key[c] = ((unsigned long long)t[c] << 1) | (s[c] > 0 ? 1ull : 0ull);
    L.cnt[c] = n[c];
  }
}

// first cell (lowest index) whose spin is not +-1 or whose tick is outside [tmin, tmax)
__global__ void validate_kernel(const int8_t* s, const long long* t, size_t N, long long tmin, long long tmax,
                                unsigned long long* first_bad) {
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const bool ok = (s[c] == 1 || s[c] == -1) && t[c] >= tmin && t[c] < tmax;
    if (!ok) atomicMin(first_bad, (unsigned long long)c);
  }
}

__global__ void exp_ticks_kernel(const uint32_t* x, unsigned long long* out, long long n, uint32_t two) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = exp_ticks(x[i], two);
}

__global__ void philox_kernel(unsigned long long seed, const uint32_t* c, const uint32_t* k,
                              uint32_t w2, uint32_t* out4, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const Philox4 b = philox_event(c[i], k[i], w2, (uint32_t)seed, (uint32_t)(seed >> 32));
    out4[4 * i + 0] = b.x;
    out4[4 * i + 1] = b.y;
    out4[4 * i + 2] = b.z;
    out4[4 * i + 3] = b.w;
  }
}

int grid_for(size_t n, int block) {
  size_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

template <int LB>
cudaError_t set_smem_attrs() {
  static bool done = false;   // per process; attributes are per-function
  if (done) return cudaSuccess;
  const int bytes = (int)TileShape<LB>::bytes;
  cudaError_t e = cudaFuncSetAttribute(round_kernel<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(blocked_kernel<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  done = true;
  return cudaSuccess;
}

template <int LB>
cudaError_t round_launch(const LatDesc* d, int nlat, int total, const LaunchCfg& cfg, int parity,
                         int launch_idx, DevCounters* ctr, unsigned long long* hist, int hist_len,
                         int round_idx, cudaStream_t s) {
  cudaError_t e = set_smem_attrs<LB>();
  if (e != cudaSuccess) return e;
  round_kernel<LB><<<total, 4 * LB, TileShape<LB>::bytes, s>>>(d, nlat, cfg.rounds, parity, launch_idx,
                                                               ctr, hist, hist_len, round_idx);
  return cudaGetLastError();
}

template <int LB>
int blocked_resident(int* per_sm) {
  if (set_smem_attrs<LB>() != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, blocked_kernel<LB>, 4 * LB,
                                                    TileShape<LB>::bytes) != cudaSuccess)
    return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm) *per_sm = nb;
  return nb * sms;
}

template <int LB>
cudaError_t blocked_launch(const LatDesc* d, int nlat, int total, const LaunchCfg& cfg, int grid,
                           unsigned* tile_done, DevCounters* ctr, cudaStream_t s) {
  cudaError_t e = set_smem_attrs<LB>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid);
  lc.blockDim = dim3(4 * LB);
  lc.dynamicSmemBytes = TileShape<LB>::bytes;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, blocked_kernel<LB>, d, nlat, total, cfg.polls, cfg.refresh,
                            cfg.max_rounds, cfg.watchdog_ns, tile_done, ctr);
}

}  // namespace

size_t tile_smem_bytes(int lb) {
  switch (lb) {
    case 32: return TileShape<32>::bytes;
    case 64: return TileShape<64>::bytes;
    case 128: return TileShape<128>::bytes;
    default: return 0;
  }
}

int blocked_max_ctas(int lb, int* per_sm) {
  switch (lb) {
    case 32: return blocked_resident<32>(per_sm);
    case 64: return blocked_resident<64>(per_sm);
    case 128: return blocked_resident<128>(per_sm);
    default: return 0;
  }
}

template <int LB>
cudaError_t round_er_launch(const LatDesc* d, int nlat, int total, int parity, int launch_idx, DevCounters* ctr,
                            cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(round_er_kernel<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TileShapeER<LB>::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  round_er_kernel<LB><<<total, 4 * LB, TileShapeER<LB>::bytes, s>>>(d, nlat, parity, launch_idx, ctr);
  return cudaGetLastError();
}

cudaError_t launch_round_er(const LatDesc* d, int nlat, int total, int lb, int parity, int launch_idx,
                            DevCounters* ctr, cudaStream_t s) {
  switch (lb) {
    case 32: return round_er_launch<32>(d, nlat, total, parity, launch_idx, ctr, s);
    case 64: return round_er_launch<64>(d, nlat, total, parity, launch_idx, ctr, s);
    case 128: return round_er_launch<128>(d, nlat, total, parity, launch_idx, ctr, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fmask(const LatDesc* h, cudaStream_t s) {
  const size_t N = (size_t)h->rows * h->cols;
  fmask_kernel<<<grid_for(N, 256), 256, 0, s>>>(*h);
  return cudaGetLastError();
}

cudaError_t launch_init(const LatDesc* h, int init_mode, cudaStream_t s) {
  const size_t N = (size_t)h->rows * h->cols;
  init_kernel<<<grid_for(N, 256), 256, 0, s>>>(*h, init_mode);
  return cudaGetLastError();
}

cudaError_t launch_publish(const LatDesc* d, int nlat, int total, int lb, int to_pub2, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  switch (lb) {
    case 32: publish_kernel<32><<<total, 128, 0, s>>>(d, nlat, to_pub2); break;
    case 64: publish_kernel<64><<<total, 256, 0, s>>>(d, nlat, to_pub2); break;
    case 128: publish_kernel<128><<<total, 512, 0, s>>>(d, nlat, to_pub2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_round(const LatDesc* d, int nlat, int total, const LaunchCfg& cfg, int parity,
                         int launch_idx, DevCounters* ctr, unsigned long long* hist, int hist_len,
                         int round_idx, cudaStream_t s) {
  switch (cfg.lb) {
    case 32: return round_launch<32>(d, nlat, total, cfg, parity, launch_idx, ctr, hist, hist_len, round_idx, s);
    case 64: return round_launch<64>(d, nlat, total, cfg, parity, launch_idx, ctr, hist, hist_len, round_idx, s);
    case 128: return round_launch<128>(d, nlat, total, cfg, parity, launch_idx, ctr, hist, hist_len, round_idx, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_blocked(const LatDesc* d, int nlat, int total, const LaunchCfg& cfg, int grid,
                           unsigned* tile_done, DevCounters* ctr, cudaStream_t s) {
  switch (cfg.lb) {
    case 32: return blocked_launch<32>(d, nlat, total, cfg, grid, tile_done, ctr, s);
    case 64: return blocked_launch<64>(d, nlat, total, cfg, grid, tile_done, ctr, s);
    case 128: return blocked_launch<128>(d, nlat, total, cfg, grid, tile_done, ctr, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reduce(const LatDesc* h, unsigned long long* d_out4, cudaStream_t s) {
  const size_t N = (size_t)h->rows * h->cols;
  reduce_kernel<<<grid_for(N, 256), 256, 0, s>>>(*h, d_out4);
  return cudaGetLastError();
}

cudaError_t launch_count_range(const LatDesc* h, unsigned* d_out2, cudaStream_t st) {
  const size_t N = (size_t)h->rows * h->cols;
  count_range_kernel<<<grid_for(N, 256), 256, 0, st>>>(*h, d_out2);
  return cudaGetLastError();
}

cudaError_t launch_class_counts(const LatDesc* h, unsigned long long* d_out10, cudaStream_t st) {
  const size_t N = (size_t)h->rows * h->cols;
  class_count_kernel<<<grid_for(N, 256), 256, 0, st>>>(*h, d_out10);
  return cudaGetLastError();
}

cudaError_t launch_count_range_batch(const LatDesc* d, int nlat, size_t max_cells, unsigned* d_out2n,
                                     cudaStream_t st) {
  if (nlat <= 0) return cudaSuccess;
  // about 32 cells per thread for the largest lattice
  const size_t bx = std::min<size_t>(1024, std::max<size_t>(1, (max_cells + 256 * 32 - 1) / (256 * 32)));
  count_range_batch_kernel<<<dim3((unsigned)bx, (unsigned)nlat), 256, 0, st>>>(d, d_out2n);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const LatDesc* h, int8_t* so, long long* to, unsigned* no, cudaStream_t st,
                          int max_blocks) {
  const size_t N = (size_t)h->rows * h->cols;
  const int g = max_blocks > 0 ? std::min(grid_for(N, 256), max_blocks) : grid_for(N, 256);
  unpack_kernel<<<g, 256, 0, st>>>(*h, so, to, no);
  return cudaGetLastError();
}

cudaError_t launch_pack(const LatDesc* h, const int8_t* si, const long long* ti, const unsigned* ni,
                        cudaStream_t st) {
  const size_t N = (size_t)h->rows * h->cols;
  pack_kernel<<<grid_for(N, 256), 256, 0, st>>>(*h, si, ti, ni);
  return cudaGetLastError();
}


template <int RW, bool FR, int MODEL, bool RATES = true>
cudaError_t tb_launch_rw(const LatDesc* d, int nlat, int total, int halo, int rounds, DevCounters* ctr,
                         cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tb_kernel<RW, FR, MODEL, false, RATES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TbCfg<RW>::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = std::min(total, tb_grid(RW));
  tb_kernel<RW, FR, MODEL, false, RATES><<<grid, TbCfg<RW>::NT, TbCfg<RW>::bytes, s>>>(d, nlat, total, halo, rounds,
                                                                                       ctr, EpArgs{});
  return cudaGetLastError();
}

template <int RW, int MODEL, bool RATES>
cudaError_t ep_launch_rw(const LatDesc* d, int nlat, int total, int halo, int rounds, DevCounters* ctr,
                         const EpArgs& ep, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tb_kernel<RW, false, MODEL, true, RATES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TbCfg<RW>::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = std::min(total * ep.max_epochs, tb_grid(RW));
  tb_kernel<RW, false, MODEL, true, RATES><<<grid, TbCfg<RW>::NT, TbCfg<RW>::bytes, s>>>(d, nlat, total, halo,
                                                                                         rounds, ctr, ep);
  return cudaGetLastError();
}

template <int RW, int MODEL>
cudaError_t tb_launch_frames(const LatDesc* d, int nlat, int total, int halo, int rounds, DevCounters* ctr,
                             cudaStream_t s, bool frames, bool rates) {
  if constexpr (MODEL == 0) {   // the Ising array without frames or rates: the rate-free kernel
    if (!frames && !rates) return tb_launch_rw<RW, false, 0, false>(d, nlat, total, halo, rounds, ctr, s);
  }
  return frames ? tb_launch_rw<RW, true, MODEL>(d, nlat, total, halo, rounds, ctr, s)
                : tb_launch_rw<RW, false, MODEL>(d, nlat, total, halo, rounds, ctr, s);
}

template <int RW>
cudaError_t tb_launch_model(const LatDesc* d, int nlat, int total, int halo, int rounds, DevCounters* ctr,
                            cudaStream_t s, bool frames, int model, bool rates) {
  switch (model) {
    case 0: return tb_launch_frames<RW, 0>(d, nlat, total, halo, rounds, ctr, s, frames, rates);
    case 1: return tb_launch_frames<RW, 1>(d, nlat, total, halo, rounds, ctr, s, frames, rates);
    case 2: return tb_launch_frames<RW, 2>(d, nlat, total, halo, rounds, ctr, s, frames, rates);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tb(const LatDesc* d, int nlat, int total, int region, int halo, int rounds, DevCounters* ctr,
                      cudaStream_t s, bool frames, int model, bool rates) {
  if (halo < 1 || rounds < 1 || rounds > halo || 4 * halo >= region) return cudaErrorInvalidValue;
  switch (region) {
    case 96: return tb_launch_model<96>(d, nlat, total, halo, rounds, ctr, s, frames, model, rates);
    case 128: return tb_launch_model<128>(d, nlat, total, halo, rounds, ctr, s, frames, model, rates);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t read_check_word(unsigned long long* word) {
#ifdef AC_CHECK
  cudaError_t e = cudaMemcpyFromSymbol(word, g_check_word, sizeof(unsigned long long));
  if (e != cudaSuccess) return e;
  const unsigned long long zero = 0ull;
  return cudaMemcpyToSymbol(g_check_word, &zero, sizeof zero);
#else
  *word = 0ull;
  return cudaSuccess;
#endif
}

__global__ void store_desc_kernel(LatDesc d, LatDesc* out) { *out = d; }

cudaError_t launch_store_desc(const LatDesc& d, LatDesc* out, cudaStream_t s) {
  store_desc_kernel<<<1, 1, 0, s>>>(d, out);
  return cudaGetLastError();
}

cudaError_t launch_ep(const LatDesc* d, int nlat, int total, int region, int halo, int rounds, DevCounters* ctr,
                      const EpArgs& ep, cudaStream_t s, int model, bool rates) {
  if (halo < 2 || (halo & 1) || rounds < 1 || rounds > halo || 4 * halo >= region || total < 1 ||
      ep.max_epochs < 1 || (long long)total * ep.max_epochs >= (1ll << 31) || model != 0)
    return cudaErrorInvalidValue;
  switch (region) {
    case 96:
      return rates ? ep_launch_rw<96, 0, true>(d, nlat, total, halo, rounds, ctr, ep, s)
                   : ep_launch_rw<96, 0, false>(d, nlat, total, halo, rounds, ctr, ep, s);
    case 128:
      return rates ? ep_launch_rw<128, 0, true>(d, nlat, total, halo, rounds, ctr, ep, s)
                   : ep_launch_rw<128, 0, false>(d, nlat, total, halo, rounds, ctr, ep, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void frames_fill_kernel(LatDesc L, long long K, int count) {
  const size_t N = (size_t)L.rows * L.cols;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long k = L.key[c];
    const signed char v = (k & 1ull) ? (signed char)1 : (signed char)-1;
    for (int f = 0; f < count; ++f) {
      const unsigned long long T = (unsigned long long)((K + f) * L.f_dt);
      if (T < (k >> 1)) L.frames[(size_t)((K + f) % L.f_B) * N + c] = v;
    }
  }
}

cudaError_t launch_frames_fill(const LatDesc* h, long long K, int count, cudaStream_t s) {
  const size_t N = (size_t)h->rows * h->cols;
  if (count <= 0) return cudaSuccess;
  frames_fill_kernel<<<grid_for(N, 256), 256, 0, s>>>(*h, K, count);
  return cudaGetLastError();
}

int tb_grid(int region) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  return sms * (region <= 96 ? TbCfg<96>::MIN_CTAS : TbCfg<128>::MIN_CTAS);
}

cudaError_t launch_pack_checked(const LatDesc* h, const int8_t* si, const long long* ti, const unsigned* ni,
                                const unsigned long long* d_bad, cudaStream_t st, int max_blocks) {
  const size_t N = (size_t)h->rows * h->cols;
  const int g = max_blocks > 0 ? std::min(grid_for(N, 256), max_blocks) : grid_for(N, 256);
  pack_checked_kernel<<<g, 256, 0, st>>>(*h, si, ti, ni, d_bad);
  return cudaGetLastError();
}

cudaError_t launch_validate(const int8_t* s_in, const long long* t_in, size_t N, long long tmin, long long tmax,
                            unsigned long long* d_first_bad, cudaStream_t st, int max_blocks) {
  const int g = max_blocks > 0 ? std::min(grid_for(N, 256), max_blocks) : grid_for(N, 256);
  validate_kernel<<<g, 256, 0, st>>>(s_in, t_in, N, tmin, tmax, d_first_bad);
  return cudaGetLastError();
}

cudaError_t launch_exp_ticks(const uint32_t* x, unsigned long long* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  exp_ticks_kernel<<<grid_for((size_t)n, 256), 256, 0, s>>>(x, out, n, 2u);
  return cudaGetLastError();
}

cudaError_t launch_philox(unsigned long long seed, const uint32_t* c, const uint32_t* k, uint32_t w2,
                          uint32_t* out4, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<grid_for((size_t)n, 256), 256, 0, s>>>(seed, c, k, w2, out4, n);
  return cudaGetLastError();
}

}  // namespace ac
