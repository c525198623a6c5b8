// ac_internal.h -- structures shared by the kernels (ac_kernels.cu) and the host
// runtime (ac_api.cu).  Not part of the public C ABI (include/ac.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ac {

// Per-lattice descriptor, resident in device memory for the kernels.
//
// Device state of a rows x cols torus (row-major):
//   key[c] = tick << 1 | (spin > 0)   next-arrival tick and current spin
//   cnt[c] = number of committed arrivals of cell c
// Tiling: tr x tc tiles; tile (i, j) covers rows [r0(i), r0(i)+h(i)) with
// r0(i) = i*(rows/tr) + min(i, rows%tr), h(i) = rows/tr + (i < rows%tr), and the
// same for columns (with cpair = 1, the same in units of two columns: every tile
// column start and width is even); every tile side is <= lb.
// Edge words: pub[(ti*tc + tj)*4*lb + e*lb + p] is the key of the tile's boundary
// cell p on edge e (0 top row, 1 bottom row, 2 left column, 3 right column).
// Threshold table capacity: 10 entries for the 4-neighbour array, 2 (M + 1) for the
// q-th degree neighbourhood with M = 2 q (q + 1) neighbours (q <= 3).
constexpr int kThrMax = 50;

struct LatDesc {
  unsigned long long* key;
  unsigned int* cnt;
  unsigned long long* pub;   // edge words, live (blocked kernel) / round input
  unsigned long long* pub2;  // round kernel output edge words (ping-pong)
  unsigned long long* key2;  // second state buffer (temporal-blocked round kernel, ping-pong)
  unsigned int* cnt2;
  unsigned long long* events;  // per-lattice committed-arrival counter
  int rows, cols;
  int tr, tc;
  int cpair;                 // 1: columns are tiled in pairs (every tile column start and width even)
  int srow0, srows;          // row slab: the tiles cover rows [srow0, srow0 + srows) only (srows = 0: all rows)
  int lb;
  int tile_base;             // first tile of this lattice in the launch's work list
  unsigned int thr[kThrMax]; // flip thresholds, index j + 5*(s > 0) (q-th degree neighbourhood:
                             // j + (M+1)*(s > 0)); the Life automaton keeps its masks in thr[0..1]
  unsigned int seed_lo, seed_hi;
  long long t_end;           // commit arrivals with tick < t_end
  unsigned long long t2;     // 2 * t_end: key < t2  <=>  tick < t_end
  int drop_publish;          // verification hook: suppress edge-word publication
  unsigned int two;          // the constant 2, opaque to the compiler (see exp_ticks)
  // Snapshot frames (Fig. 3.7): f_open frames are open, the f-th at tick f_t0 + f * f_dt
  // in slot (f_slot0 + f) % f_B of `frames` (f_B slots of rows * cols int8 spins).
  // A commit of an arrival at tick ta whose next arrival is at tick tn writes the new
  // spin into every open frame whose tick T satisfies ta <= T < tn.  f_open = 0: off.
  signed char* frames;
  long long f_t0, f_dt;
  int f_open, f_slot0, f_B;
  // model: 0 = Ising heat bath (thr = flip thresholds); 1 = Life-like automaton on the
  // Moore neighbourhood (thr[0] = birth mask, thr[1] = survival mask over the number of
  // live neighbours; a random initial cell is alive iff its init word < life_density);
  // 2 = Ising heat bath on the q-th degree neighbourhood (every cell within Manhattan
  // distance q, 2 <= q <= 3)
  int model;
  int q;
  unsigned life_density;
  // per-cell rates (law (A) of Sec. 2): cell c's gaps are max(1, floor(e * rates[c] / 2^20))
  // for the rate-1 gap e, i.e. rate 2^20 / rates[c]; nullptr = every cell at rate 1
  const unsigned* rates;
  // early commits of certain rejections (one-round kernel): flip mask of each cell's pending
  // arrival, bit j set iff it flips with j up neighbours; nullptr = off
  unsigned char* fmask;
  // epoch kernel: four 128-byte 2D tensor maps (driver CUtensorMap) of the key buffers,
  // RW x RW boxes of uint64: box 96 over key and key2, then box 128 over key and key2;
  // nullptr = region rows by row copies only
  const void* tmap;
};
constexpr int kTmapBytes = 128;

// Device counters of one run call (zeroed by the host before the call).
struct DevCounters {
  unsigned long long events;    // committed arrivals
  unsigned long long rounds;    // tile rounds executed (commit phases)
  unsigned long long scanned;   // cells tested by the enable test
  unsigned long long enabled;   // cells found enabled
  unsigned long long visits;    // tile visits (blocked kernel)
  unsigned long long polls;     // halo polls while a tile was blocked
  int error;                    // AC_ERR_* set by the device watchdog
  int err_block;
  unsigned int active[3];       // round kernel: tiles with pending arrivals (mod-3 ring)
  unsigned int launched;        // round kernel: launches that did work
  unsigned int seq;             // temporal-blocked kernel: launches completed in this call
  unsigned int blocks_done;     // temporal-blocked kernel: CTAs finished in the current launch
  unsigned long long kmin[3];   // temporal-blocked kernel with frames: smallest output key of a
                                // launch (mod-3 ring like active; the host presets all to ~0)
  unsigned long long early;     // one-round kernel: arrivals committed early as certain rejections
  // epoch kernel: the claim word, one 64-bit word (low half first): the next work item to
  // claim, and the epochs after which no arrival before t_end is left (the host presets ~0).
  // A claim is one 64-bit atomic add, so it sees the stop epoch as of its own place in the
  // word's order: refusals are monotone in the item index
  unsigned int next_item;
  unsigned int stop_epoch;
};
static_assert(offsetof(DevCounters, next_item) % 8 == 0 && offsetof(DevCounters, stop_epoch) == offsetof(DevCounters, next_item) + 4,
              "the claim word");

// Epoch kernel (the persistent temporal-blocked kernel): per-tile and per-epoch words.
//   done[tile]        epochs the tile has completed (release / acquire)
//   ep_count[e]       high word: tiles that completed epoch e; low word: those of them with
//                     an arrival before t_end left (one atomic carries both)
// All zero before a launch; ep_count holds max_epochs entries.
// range: nrange (min, max) count pairs from count_range kernels; if any max - min >= limit
// the kernel does no work and reports kEpWindow (the 16-bit count window of a region could
// overflow during the call; the caller falls back to the exact one-round kernel).
struct EpArgs {
  unsigned int* done;
  unsigned long long* ep_count;
  int max_epochs;
  long long watchdog_ns;
  const unsigned int* range;
  int nrange;
  unsigned int limit;
};
constexpr int kEpWindow = 6;   // DevCounters::error of an epoch-kernel launch refused by the count check

enum KernelKind { kKernelRound = 0, kKernelBlocked = 1, kKernelEpoch = 2 };

// Temporal-blocked round kernel: a shared-memory region of side 96 (two CTAs per
// SM) or 128 (one) holds a tile and a halo of depth D around it; tile side = region - 2D.
constexpr int kTbMaxHalo = 16;
// wide = true selects the 128-wide region (512 threads, one CTA per SM) for any halo.
inline int tb_region_for(int halo, bool wide = false) { return (halo <= 12 && !wide) ? 96 : 128; }
// the q = 3 diamond's 13 order planes exist on the 128-wide region only
inline int tb_region_for_model(int halo, int model, int q, bool wide = false) {
  return (model == 2 && q == 3) ? 128 : tb_region_for(halo, wide);
}

struct LaunchCfg {
  int kernel;       // KernelKind
  int lb;           // 32, 64 or 128
  int threads;      // 4 * lb
  int rounds;       // round kernel: rounds per launch (1 = exact synchronous rounds)
  int polls;        // blocked kernel: halo polls before a blocked tile is left
  int refresh;      // blocked kernel: refresh halos every `refresh` rounds
  int max_rounds;   // blocked kernel: cap on rounds per tile visit (0 = none)
  long long watchdog_ns;  // blocked kernel: no-progress limit before AC_ERR_STALL
};

// Sets the thread-local message returned by ac_last_error() (ac_api.cu).
void set_last_error(const char* msg);

// Heat-bath threshold table of the 4-neighbour Ising array (appendix flip
// probabilities; ac_api.cu), shared by every entry point of the library.
void make_thresholds(double beta, double J, double h, uint32_t thr[10]);

// ---- launchers (ac_kernels.cu) -------------------------------------------------
size_t tile_smem_bytes(int lb);
int blocked_max_ctas(int lb, int* per_sm);   // resident CTAs of the blocked kernel
cudaError_t launch_init(const LatDesc* host_desc, int init_mode, cudaStream_t s);
// One synchronous round (Fig. 3.2) over Lb tiles with early commits of certain rejections
// (LatDesc::fmask set; see round_er_kernel), and the pass that fills fmask for every cell.
cudaError_t launch_round_er(const LatDesc* d_desc, int nlat, int total_tiles, int lb, int parity, int launch_idx,
                            DevCounters* ctr, cudaStream_t s);
cudaError_t launch_fmask(const LatDesc* host_desc, cudaStream_t s);
cudaError_t launch_publish(const LatDesc* d_desc, int nlat, int total_tiles, int lb, int to_pub2,
                           cudaStream_t s);
cudaError_t launch_round(const LatDesc* d_desc, int nlat, int total_tiles, const LaunchCfg& cfg,
                         int parity, int launch_idx, DevCounters* ctr, unsigned long long* hist,
                         int hist_len, int round_idx, cudaStream_t s);
cudaError_t launch_blocked(const LatDesc* d_desc, int nlat, int total_tiles, const LaunchCfg& cfg,
                           int grid, unsigned int* tile_done, DevCounters* ctr, cudaStream_t s);
cudaError_t launch_reduce(const LatDesc* host_desc, unsigned long long* d_out4, cudaStream_t s);
cudaError_t launch_count_range(const LatDesc* host_desc, unsigned* d_out2, cudaStream_t s);
cudaError_t launch_class_counts(const LatDesc* host_desc, unsigned long long* d_out10, cudaStream_t s);
// max_blocks > 0 caps the grid (grid-stride loops): the asynchronous transfers run these
// kernels beside another handle's persistent kernel on a few SMs only
cudaError_t launch_unpack(const LatDesc* host_desc, int8_t* s_out, long long* t_out,
                          unsigned int* n_out, cudaStream_t st, int max_blocks = 0);
cudaError_t launch_pack(const LatDesc* host_desc, const int8_t* s_in, const long long* t_in,
                        const unsigned int* n_in, cudaStream_t st);
// Launch of the temporal-blocked round kernel.  The launch number (which fixes the
// ping-pong parity) is kept on the device in ctr->seq, so every launch of a run has
// the same arguments and a sequence of launches can be captured in a CUDA graph.
// frames: the lattices have open snapshot frames (the kernel variant that writes them);
// model: the lattices' model (LatDesc::model; all lattices of a launch share it).
// The q-th degree neighbourhood model shrinks the region by q rings per round:
// halo = q * rounds.
// rates = false: no lattice of the launch has per-cell rates (the 4-neighbour array without
// frames then runs a kernel without the per-commit rate test); captured graphs keep true.
cudaError_t launch_tb(const LatDesc* d_desc, int nlat, int total_tiles, int region, int halo, int rounds,
                      DevCounters* ctr, cudaStream_t s, bool frames = false, int model = 0, bool rates = true);
// One launch of the epoch kernel: the temporal-blocked tile visit of launch_tb run as a
// persistent dataflow over (epoch, tile) work items.  Each item advances one tile by
// `rounds` synchronous rounds; it starts once the tile and its 8 neighbours have
// completed the previous epoch (done words, release / acquire), and the kernel ends
// when an epoch leaves no arrival before t_end (ctr->stop_epoch) or after
// ep.max_epochs epochs.  State of epoch e is in key / cnt for even e, key2 / cnt2 for
// odd e.  Needs even cols, even halo, a cpair tiling whose tile sides are >= halo, and
// 16-byte aligned key buffers (the region rows are loaded by bulk asynchronous copies).
cudaError_t launch_ep(const LatDesc* d_desc, int nlat, int total_tiles, int region, int halo, int rounds,
                      DevCounters* ctr, const EpArgs& ep, cudaStream_t s, int model = 0, bool rates = true);
// Bounds-checked build (-DAC_CHECK): the first index violation the kernels recorded since the
// last call, (site << 40) | index, and clears it; always 0 in the production build.
cudaError_t read_check_word(unsigned long long* word);

// Stores a descriptor into device memory by a one-thread kernel (a launch parameter, no copy
// engine: the copy engines may be busy with other streams' transfers).
cudaError_t launch_store_desc(const LatDesc& d, LatDesc* out, cudaStream_t s);
// Frames [K, K + count) were just opened: write each cell's spin into those whose tick
// lies before the cell's next arrival (later commits write the others).
cudaError_t launch_frames_fill(const LatDesc* host_desc, long long K, int count, cudaStream_t s);
cudaError_t launch_count_range_batch(const LatDesc* d_desc, int nlat, size_t max_cells, unsigned* d_out2n,
                                     cudaStream_t s);
int tb_grid(int region);   // resident CTAs of the temporal-blocked kernel
cudaError_t launch_validate(const int8_t* s_in, const long long* t_in, size_t N, long long tmin, long long tmax,
                            unsigned long long* d_first_bad, cudaStream_t st, int max_blocks = 0);
// launch_pack that writes nothing unless *d_bad == ~0 (device-side validation result)
cudaError_t launch_pack_checked(const LatDesc* host_desc, const int8_t* s_in, const long long* t_in,
                                const unsigned int* n_in, const unsigned long long* d_bad, cudaStream_t st,
                                int max_blocks = 0);
cudaError_t launch_exp_ticks(const uint32_t* x, unsigned long long* out, long long n, cudaStream_t s);
cudaError_t launch_philox(unsigned long long seed, const uint32_t* c, const uint32_t* k, uint32_t w2,
                          uint32_t* out4, long long n, cudaStream_t s);

}  // namespace ac
