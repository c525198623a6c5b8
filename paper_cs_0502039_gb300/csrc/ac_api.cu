// ac_api.cu -- host runtime behind the C ABI of include/ac.h.
//
// Owns device memory and streams, computes the heat-bath threshold table (the
// only floating-point step of the method, appendix flip probabilities, in IEEE
// binary64 on the host), drives the round kernel (one launch per synchronous
// round of Fig. 3.2, checked for completion in chunks) and the blocked
// persistent kernel (one cooperative launch per run call, Fig. 3.4), and
// captures batched runs into CUDA graphs.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is reached through the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ac.h"
#include "ac_internal.h"

namespace {

thread_local std::string g_err;

ac_status fail(ac_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define AC_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(AC_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                     \
  } while (0)

constexpr double kTicksPerUnit = 4294967296.0;
// grid of the state-transfer kernels of the asynchronous loads and reads: they run beside
// another handle's persistent kernel, so they stay on a few SMs
constexpr int kAsyncBlocks = 152;
constexpr long long kTickLimit = 1ll << 61;

int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace

namespace ac {
// Lets other translation units of the library report through ac_last_error().
void set_last_error(const char* msg) { g_err = msg; }

// Heat-bath thresholds: p = 1/(1 + exp(beta dE)), dE = 2 s (J S + h);
// thr = min(floor(p * 2^32), 2^32 - 1), index j + 5*(s > 0), S = 2j - 4.
void make_thresholds(double beta, double J, double h, uint32_t thr[10]) {
  for (int up = 0; up < 2; ++up) {
    const double s = up ? 1.0 : -1.0;
    for (int j = 0; j < 5; ++j) {
      const double S = (double)(2 * j - 4);
      const double dE = 2.0 * s * (J * S + h);
      const double p = 1.0 / (1.0 + std::exp(beta * dE));
      const double v = std::ldexp(p, 32);
      thr[j + 5 * up] = (v < 4294967295.0) ? (uint32_t)std::floor(v) : 0xFFFFFFFFu;
    }
  }
}

}  // namespace ac

struct ac_sim {
  int rows = 0, cols = 0, init = 0;
  double beta = 0, J = 0, h = 0;
  uint64_t seed = 0;
  cudaStream_t stream = nullptr;
  ac::LaunchCfg cfg{};
  uint32_t thr[ac::kThrMax] = {};
  int q = 1;                                // neighbourhood radius (model 2)
  int tr = 0, tc = 0;

  unsigned long long* key = nullptr;
  unsigned int* cnt = nullptr;
  unsigned long long* key2 = nullptr;       // second state buffer (temporal-blocked rounds);
  unsigned int* cnt2 = nullptr;             // between run calls also the staging of state transfers
  int8_t* stage8 = nullptr;                 // spin staging of state transfers
  unsigned long long* pub = nullptr;
  unsigned long long* pub2 = nullptr;
  size_t pub_words = 0;
  unsigned long long* d_events = nullptr;   // per-lattice event counter
  ac::LatDesc* d_desc = nullptr;
  ac::DevCounters* d_ctr = nullptr;
  unsigned int* d_tile_done = nullptr;
  size_t tile_done_cap = 0;
  unsigned long long* d_hist = nullptr;     // enabled counts per synchronous round
  int hist_cap = 0;
  unsigned long long* d_red = nullptr;
  unsigned int* d_ep = nullptr;             // epoch kernel: tile done words, per-epoch counts
  size_t ep_cap = 0;
  unsigned char* d_fmask = nullptr;         // early commits of certain rejections: flip masks
  // epoch kernel: 2D tensor maps of the key buffers (encoded for the pair tmap_a / tmap_b):
  // h_tmap / d_tmap hold [96: a, b; 128: a, b] then the same with a and b exchanged
  CUtensorMap h_tmap[8];
  void* d_tmap = nullptr;
  const void* tmap_a = nullptr;
  const void* tmap_b = nullptr;
  bool tmap_off = false;                    // the encoder is unavailable or refused the maps
  bool early_reject = false;
  int slab_row0 = 0, slab_rows = 0;         // row slab of a partitioned lattice (0 rows: none)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // asynchronous state transfers (ac_load_state_async / ac_read_state_async) on a caller's stream
  cudaEvent_t ev_work = nullptr, ev_load = nullptr, ev_read = nullptr;
  unsigned long long* h_bad = nullptr;      // pinned: validation result of the pending load
  bool load_pending = false, read_pending = false;
  long long load_t_done = 0;

  long long t_done = 0;
  // snapshot frames (Fig. 3.7): f_B slots of ncells() spins; frames [f_K, f_K + f_B) open
  // model: 0 = Ising heat bath, 1 = Life-like automaton (birth / survival masks, density)
  int model = 0;
  uint32_t life_birth = 0, life_survive = 0, life_density = 0;
  unsigned* d_rates = nullptr;              // per-cell rate multipliers (nullptr: all rate 1)
  int8_t* frames = nullptr;
  int8_t* frame_host = nullptr;             // pinned copy handed to host callbacks
  int f_B = 0;
  long long f_dt = 0, f_K = 0;
  // accumulated statistics
  unsigned long long events = 0, rounds = 0, launches = 0, scanned = 0, enabled = 0, visits = 0,
                     polls = 0, global_rounds = 0, enabled_r1 = 0, early = 0;
  double device_ms = 0.0;
  int last_grid = 0, ctas_per_sm = 0;
  int drop_publish = 0;

  size_t ncells() const { return (size_t)rows * (size_t)cols; }
  int tiles() const { return tr * tc; }

  ac::LatDesc host_desc(long long t_end, int tile_base) const {
    ac::LatDesc d{};
    d.key = key;
    d.cnt = cnt;
    d.key2 = key2;
    d.cnt2 = cnt2;
    d.two = 2u;
    d.pub = pub;
    d.pub2 = pub2;
    d.events = d_events;
    d.rows = rows;
    d.cols = cols;
    d.tr = tr;
    d.tc = tc;
    d.lb = cfg.lb;
    d.tile_base = tile_base;
    std::memcpy(d.thr, thr, sizeof thr);
    d.seed_lo = (unsigned)(seed & 0xffffffffu);
    d.seed_hi = (unsigned)(seed >> 32);
    d.t_end = t_end;
    d.t2 = 2ull * (unsigned long long)t_end;
    d.drop_publish = drop_publish;
    d.model = model;
    d.q = q;
    d.life_density = life_density;
    d.rates = d_rates;
    if (model == 1) {
      d.thr[0] = life_birth;
      d.thr[1] = life_survive;
    }
    if (f_B > 0) {
      d.frames = reinterpret_cast<signed char*>(frames);
      d.f_t0 = f_K * f_dt;
      d.f_dt = f_dt;
      d.f_open = f_B;
      d.f_slot0 = (int)(f_K % f_B);
      d.f_B = f_B;
    }
    return d;
  }
};

namespace {

// ---------------------------------------------------------------- batch graphs
struct BatchRunner {
  std::vector<ac_sim*> sims;
  ac::LatDesc* h_desc = nullptr;   // pinned; read by the graph's copy node at replay
  ac::LatDesc* d_desc = nullptr;
  ac::DevCounters* d_ctr = nullptr;
  unsigned int* d_tile_done = nullptr;
  unsigned long long* h_before = nullptr;
  int total_tiles = 0, grid = 0, lb = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  ac::LaunchCfg cfg{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // epoch-kernel batches: tile done words and per-epoch counts
  bool ep = false;
  unsigned int* d_ep = nullptr;
  size_t ep_cap = 0;
  // temporal-blocked batches: per-lattice count ranges, a captured chunk of launches
  bool tb = false;
  int region = 0, halo = 0, calls = 0;
  unsigned* d_range = nullptr;
  cudaGraphExec_t chunk_exec = nullptr;
  cudaGraph_t chunk_graph = nullptr;
};

std::mutex g_batch_mu;
std::map<std::vector<ac_sim*>, BatchRunner*> g_runners;

void free_runner(BatchRunner* r) {
  if (!r) return;
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  if (r->h_desc) cudaFreeHost(r->h_desc);
  if (r->d_desc) cudaFree(r->d_desc);
  if (r->d_ctr) cudaFree(r->d_ctr);
  if (r->d_tile_done) cudaFree(r->d_tile_done);
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
  if (r->own_stream) cudaStreamDestroy(r->own_stream);
  if (r->chunk_exec) cudaGraphExecDestroy(r->chunk_exec);
  if (r->chunk_graph) cudaGraphDestroy(r->chunk_graph);
  if (r->d_range) cudaFree(r->d_range);
  if (r->d_ep) cudaFree(r->d_ep);
  delete r;
}

void drop_runners_of(ac_sim* sim) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto it = g_runners.begin(); it != g_runners.end();) {
    if (std::find(it->first.begin(), it->first.end(), sim) != it->first.end()) {
      free_runner(it->second);
      it = g_runners.erase(it);
    } else {
      ++it;
    }
  }
}

ac_status alloc_edges(ac_sim* s) {
  s->tr = ceil_div(s->rows, s->cfg.lb);
  s->tc = ceil_div(s->cols, s->cfg.lb);
  const size_t words = (size_t)s->tiles() * 4 * s->cfg.lb;
  if (words > s->pub_words) {
    if (s->pub) cudaFree(s->pub);
    if (s->pub2) cudaFree(s->pub2);
    s->pub = s->pub2 = nullptr;
    s->pub_words = 0;
    if (cudaMalloc(&s->pub, words * 8) != cudaSuccess || cudaMalloc(&s->pub2, words * 8) != cudaSuccess)
      return fail(AC_ERR_OOM, "edge words: cudaMalloc of %zu bytes failed", words * 16);
    s->pub_words = words;
  }
  if ((size_t)s->tiles() > s->tile_done_cap) {
    if (s->d_tile_done) cudaFree(s->d_tile_done);
    s->d_tile_done = nullptr;
    if (cudaMalloc(&s->d_tile_done, (size_t)s->tiles() * 4) != cudaSuccess)
      return fail(AC_ERR_OOM, "tile flags: cudaMalloc failed");
    s->tile_done_cap = (size_t)s->tiles();
  }
  return AC_OK;
}

void free_sim(ac_sim* s) {
  if (!s) return;
  // asynchronous transfers still in flight on a caller's stream use the handle's buffers
  if (s->load_pending) cudaEventSynchronize(s->ev_load);
  if (s->read_pending) cudaEventSynchronize(s->ev_read);
  if (s->ev_work) cudaEventDestroy(s->ev_work);
  if (s->ev_load) cudaEventDestroy(s->ev_load);
  if (s->ev_read) cudaEventDestroy(s->ev_read);
  if (s->h_bad) cudaFreeHost(s->h_bad);
  cudaFree(s->key);
  cudaFree(s->cnt);
  cudaFree(s->key2);
  cudaFree(s->cnt2);
  cudaFree(s->stage8);
  cudaFree(s->pub);
  cudaFree(s->pub2);
  cudaFree(s->d_events);
  cudaFree(s->d_desc);
  cudaFree(s->d_ctr);
  cudaFree(s->d_tile_done);
  cudaFree(s->d_hist);
  cudaFree(s->d_red);
  cudaFree(s->d_ep);
  cudaFree(s->d_fmask);
  cudaFree(s->d_tmap);
  cudaFree(s->frames);
  cudaFree(s->d_rates);
  if (s->frame_host) cudaFreeHost(s->frame_host);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  delete s;
}

ac_status check_params(const ac_lattice& lat, double beta, double J, double h) {
  if (lat.rows < 2 || lat.cols < 2)
    return fail(AC_ERR_ARG, "rows and cols must be >= 2 (got %d x %d)", lat.rows, lat.cols);
  if ((unsigned long long)lat.rows * (unsigned long long)lat.cols >= (1ull << 32))
    return fail(AC_ERR_ARG, "rows * cols must be < 2^32");
  if (lat.init < AC_INIT_RANDOM || lat.init > AC_INIT_DOWN)
    return fail(AC_ERR_ARG, "init must be AC_INIT_RANDOM, AC_INIT_UP or AC_INIT_DOWN");
  if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(AC_ERR_ARG, "beta must be finite and >= 0");
  if (!std::isfinite(J) || !std::isfinite(h)) return fail(AC_ERR_ARG, "J and h must be finite");
  return AC_OK;
}

ac_status create_one(ac_lattice lat, double beta, double J, double h, uint64_t seed, ac_sim** out) {
  ac_sim* s = new (std::nothrow) ac_sim();
  if (!s) return fail(AC_ERR_OOM, "host allocation failed");
  s->rows = lat.rows;
  s->cols = lat.cols;
  s->init = lat.init;
  s->beta = beta;
  s->J = J;
  s->h = h;
  s->seed = seed;
  s->cfg.kernel = ac::kKernelBlocked;
  s->cfg.lb = 64;
  s->cfg.threads = 256;
  s->cfg.rounds = 1;
  s->cfg.polls = 8;
  s->cfg.refresh = 1;
  s->cfg.max_rounds = 0;
  s->cfg.watchdog_ns = 5ll * 1000 * 1000 * 1000;
  ac::make_thresholds(beta, J, h, s->thr);
  const size_t N = s->ncells();
  if (cudaMalloc(&s->key, N * 8) != cudaSuccess || cudaMalloc(&s->cnt, N * 4) != cudaSuccess ||
      cudaMalloc(&s->d_events, 8) != cudaSuccess || cudaMalloc(&s->d_desc, sizeof(ac::LatDesc)) != cudaSuccess ||
      cudaMalloc(&s->d_ctr, sizeof(ac::DevCounters)) != cudaSuccess ||
      cudaMalloc(&s->d_red, 16 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    free_sim(s);
    return fail(AC_ERR_OOM, "cudaMalloc of the lattice state (%zu cells) failed", N);
  }
  ac_status st = alloc_edges(s);
  if (st != AC_OK) {
    free_sim(s);
    return st;
  }
  if (cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess) {
    free_sim(s);
    return fail(AC_ERR_CUDA, "cudaEventCreate failed");
  }
  const ac::LatDesc d = s->host_desc(0, 0);
  cudaError_t e = ac::launch_init(&d, lat.init, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    free_sim(s);
    return fail(AC_ERR_CUDA, "init kernel failed: %s", cudaGetErrorString(e));
  }
  *out = s;
  return AC_OK;
}

// Bounds-checked build: AC_ERR_STATE if the kernels recorded an index violation since the
// last check (a no-op in the production build).
ac_status check_bounds() {
#ifdef AC_CHECK
  unsigned long long word = 0;
  AC_CUDA(ac::read_check_word(&word));
  if (word) return fail(AC_ERR_STATE, "bounds check: site %llu, index %llu", word >> 40, word & 0xFFFFFFFFFFull);
#endif
  return AC_OK;
}

ac_status accumulate(ac_sim* s, const ac::DevCounters& c, float ms, bool round_kernel) {
  const ac_status bc = check_bounds();
  if (bc != AC_OK) return bc;
  s->rounds += c.rounds;
  s->scanned += c.scanned;
  s->enabled += c.enabled;
  s->visits += c.visits;
  s->polls += c.polls;
  s->early += c.early;
  s->device_ms += ms;
  if (round_kernel) {
    s->launches += c.launched;
    if (s->cfg.rounds == 1) {
      s->global_rounds += c.launched;
      s->enabled_r1 += c.enabled;
    }
  } else {
    s->launches += 1;
  }
  if (c.error == AC_ERR_STALL) return fail(AC_ERR_STALL, "device watchdog: no progress (block %d)", c.err_block);
  if (c.error == AC_ERR_STATE) return fail(AC_ERR_STATE, "device: event counts left the 16-bit window of a region");
  if (c.error) return fail((ac_status)c.error, "device reported error %d (a q = 3 launch on a 96-wide region)", c.error);
  return AC_OK;
}

// Tile grid of the temporal-blocked round kernel: tiles of side <= 128 - 2D, at
// least 2 per dimension, and a tile count that fills the SMs' waves evenly.
void tb_tiling(int rows, int cols, int region, int halo, int sms, int* tr, int* tc) {
  const int own = region - 2 * halo;
  const int r0 = std::max(2, ceil_div(rows, own)), c0 = std::max(2, ceil_div(cols, own));
  double best = 1e300;
  *tr = r0;
  *tc = c0;
  for (int a = r0; a < r0 + 8 && a <= rows / 2; ++a)
    for (int b = c0; b < c0 + 8 && b <= cols / 2; ++b) {
      const double waves = std::ceil((double)a * b / sms);
      const double region = (std::ceil((double)rows / a) + 2 * halo) * (std::ceil((double)cols / b) + 2 * halo);
      const double cost = waves * region;
      if (cost < best - 1e-9) {
        best = cost;
        *tr = a;
        *tc = b;
      }
    }
}

// Tile grid of a lattice inside a batch: the fewest tiles (side <= region - 2D, at
// least 2 per dimension).  Every tile visit costs a region load, R rounds and a store
// whatever the tile's size, and the whole batch's tile list fills the waves, so the
// tile count, not one lattice's wave balance, sets the time.
void tb_tiling_batch(int rows, int cols, int region, int halo, int* tr, int* tc) {
  const int own = region - 2 * halo;
  *tr = std::max(2, ceil_div(rows, own));
  *tc = std::max(2, ceil_div(cols, own));
}

// Halo depth D and rounds per launch R of the temporal-blocked kernel for the handle's
// model: D = R for the 4-neighbour array and the Life automaton, D = q R for the q-th
// degree neighbourhood (the region loses q rings per round); D <= 16 and rows, cols >= 4D.
void tb_depth(const ac_sim* s, int* D, int* R) {
  const int side = std::min(s->rows, s->cols);
  if (s->model == 0) {
    *R = *D = s->cfg.rounds;
  } else {
    const int q = (s->model == 2) ? s->q : 1;
    *R = std::max(1, std::min({s->cfg.rounds, ac::kTbMaxHalo / q, side / (4 * q)}));
    *D = q * (*R);
  }
}

bool tb_applicable(const ac_sim* s) {
  const int D = s->cfg.rounds;
  return s->cfg.rounds > 1 && D <= ac::kTbMaxHalo && s->rows >= 4 * D && s->cols >= 4 * D;
}

// The temporal-blocked kernel keeps counts as 16-bit offsets within a window of
// +-32768 around each region's centre; it may run only if no region's counts can
// leave that window during the call.
ac_status tb_counts_fit(ac_sim* s, long long t_end, bool* fits) {
  const ac::LatDesc d = s->host_desc(s->t_done, 0);
  unsigned init[2] = {0xFFFFFFFFu, 0u}, r[2] = {0u, 0u};
  unsigned* d_r = reinterpret_cast<unsigned*>(s->d_red);
  AC_CUDA(cudaMemcpyAsync(d_r, init, sizeof init, cudaMemcpyHostToDevice, s->stream));
  AC_CUDA(ac::launch_count_range(&d, d_r, s->stream));
  AC_CUDA(cudaMemcpyAsync(r, d_r, sizeof r, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  const double span = (double)(t_end - s->t_done) / kTicksPerUnit;
  // a cell commits about `span` arrivals (Poisson); allow a wide margin
  *fits = (double)(r[1] - r[0]) + 2.0 * span + 64.0 * std::sqrt(span + 1.0) + 64.0 < 30000.0;
  return AC_OK;
}

ac_status run_tb(ac_sim* s, long long t_end, int D, int R) {
  const size_t N = s->ncells();
  if (!s->key2) {
    if (cudaMalloc(&s->key2, N * 8) != cudaSuccess || cudaMalloc(&s->cnt2, N * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(AC_ERR_OOM, "second state buffer (%zu cells) allocation failed", N);
    }
  }
  const int region = ac::tb_region_for_model(D, s->model, s->q, s->cfg.lb == 128);
  int tr = 0, tc = 0;
  tb_tiling(s->rows, s->cols, region, D, ac::tb_grid(region), &tr, &tc);
  ac::LatDesc d = s->host_desc(t_end, 0);
  d.tr = tr;
  d.tc = tc;
  const int total = tr * tc;
  AC_CUDA(cudaMemcpyAsync(s->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s->stream));
  AC_CUDA(cudaMemsetAsync(s->d_ctr, 0, sizeof(ac::DevCounters), s->stream));
  AC_CUDA(cudaEventRecord(s->ev0, s->stream));
  // about 8.3 synchronous rounds per unit time (Sec. 4), D of them per launch
  const double span = (double)(t_end - s->t_done) / kTicksPerUnit;
  int chunk = (int)std::min(4096.0, (9.0 * std::ceil(span) + 16.0) / D + 2.0);
  int launch_idx = 0;
  for (;;) {
    for (int i = 0; i < chunk; ++i) {
      AC_CUDA(ac::launch_tb(s->d_desc, 1, total, region, D, R, s->d_ctr, s->stream, s->f_B > 0, s->model,
                            s->d_rates != nullptr));
      ++launch_idx;
    }
    ac::DevCounters cc{};
    AC_CUDA(cudaMemcpyAsync(&cc, s->d_ctr, sizeof cc, cudaMemcpyDeviceToHost, s->stream));
    AC_CUDA(cudaStreamSynchronize(s->stream));
    // the last completed launch left nothing, or a later launch found nothing left
    if (cc.seq < (unsigned)launch_idx || cc.error || (cc.seq > 0 && cc.active[(cc.seq + 2) % 3] == 0)) break;
    if ((double)launch_idx * D > 64.0 * (9.0 * std::ceil(span) + 16.0) + 4096.0)
      return fail(AC_ERR_STALL, "round kernel: no completion after %d launches", launch_idx);
    chunk = 4;
  }
  AC_CUDA(cudaEventRecord(s->ev1, s->stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  // c.seq launches completed; launch j wrote the second buffer when j is even.  A launch
  // that hit the count window (safety net, see tb_counts_fit) produced no consistent
  // output: its input is the state to keep.
  const unsigned good = (c.error == AC_ERR_STATE) ? c.seq - 1u : c.seq;
  if (good & 1u) {
    std::swap(s->key, s->key2);
    std::swap(s->cnt, s->cnt2);
  }
  s->last_grid = std::min(total, ac::tb_grid(region));
  return accumulate(s, c, ms, true);
}

// Tile grid of the epoch kernel: as tb_tiling_batch (the fewest tiles of side <=
// region - 2D, at least 2 per dimension), with columns tiled in pairs so that every
// region row starts on an even column.  The sides stay >= D whenever rows, cols >= 4D,
// so a region reaches into the 8 neighbour tiles only.
void ep_tiling(int rows, int cols, int region, int halo, int* tr, int* tc) {
  const int own = region - 2 * halo;
  *tr = std::max(2, ceil_div(rows, own));
  *tc = std::max(2, ceil_div(cols / 2, own / 2));
}

// ---- 2D tensor maps of the key buffers (epoch kernel region copies)

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime (nullptr: none)
EncodeTiledFn tensor_map_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// rows x cols uint64 keys, row-major, boxes of box x box elements, no swizzle, zero fill
bool encode_key_map(CUtensorMap* m, void* buf, int rows, int cols, int box) {
  const EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)cols * 8u};
  const cuuint32_t boxd[2] = {(cuuint32_t)box, (cuuint32_t)box};
  const cuuint32_t es[2] = {1u, 1u};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, buf, dim, stride, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Device address of the four maps [96: key, key2; 128: key, key2] of the handle's current
// buffers, encoded and uploaded (on `stream`) the first time the pair is seen; nullptr when
// the epoch kernel is to copy region rows instead (no encoder, or the maps were refused).
const void* ensure_tmaps(ac_sim* s, cudaStream_t stream) {
  if (s->tmap_off || !s->key2 || (s->cols & 1)) return nullptr;
  const bool known = (s->key == s->tmap_a && s->key2 == s->tmap_b) || (s->key == s->tmap_b && s->key2 == s->tmap_a);
  if (!known) {
    void* a = s->key;
    void* b = s->key2;
    bool ok = encode_key_map(&s->h_tmap[0], a, s->rows, s->cols, 96) &&
              encode_key_map(&s->h_tmap[1], b, s->rows, s->cols, 96) &&
              encode_key_map(&s->h_tmap[2], a, s->rows, s->cols, 128) &&
              encode_key_map(&s->h_tmap[3], b, s->rows, s->cols, 128);
    s->h_tmap[4] = s->h_tmap[1];
    s->h_tmap[5] = s->h_tmap[0];
    s->h_tmap[6] = s->h_tmap[3];
    s->h_tmap[7] = s->h_tmap[2];
    if (ok && !s->d_tmap) ok = cudaMalloc(&s->d_tmap, sizeof s->h_tmap) == cudaSuccess;
    if (ok) ok = cudaMemcpyAsync(s->d_tmap, s->h_tmap, sizeof s->h_tmap, cudaMemcpyHostToDevice, stream) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      s->tmap_off = true;
      return nullptr;
    }
    s->tmap_a = a;
    s->tmap_b = b;
  }
  return static_cast<const char*>(s->d_tmap) + (s->key == s->tmap_a ? 0 : 4) * sizeof(CUtensorMap);
}

// The epoch kernel runs the 4-neighbour Ising array without frames, on even cols with
// an even halo (its bulk row copies need 16-byte alignment) and rows, cols >= 4D.
bool ep_applicable(const ac_sim* s) {
  const int D = s->cfg.rounds;
  return s->model == 0 && s->f_B == 0 && D >= 2 && (D & 1) == 0 && D <= ac::kTbMaxHalo && (s->cols & 1) == 0 &&
         s->rows >= 4 * D && s->cols >= 4 * D;
}

// Epochs to run per launch: about 8.3 synchronous rounds per unit time (Sec. 4), D per
// epoch, with a factor-2 margin; a launch that ends before its last epoch found
// nothing left is followed by another one.
int ep_epochs(double span, int D, int total) {
  const double e = 2.0 * (9.0 * std::ceil(span) + 16.0) / D + 8.0;
  const int cap = (int)std::min<long long>(4096, ((1ll << 31) - 1) / std::max(1, total) - 1);
  return std::max(1, std::min(cap, (int)e));
}

// Epoch-kernel words: the tiles' done words, then (8-byte aligned) one 64-bit count per epoch.
size_t ep_words(int total, int E) { return (((size_t)total + 1) & ~(size_t)1) + 2 * (size_t)E; }
unsigned long long* ep_counts(unsigned* d_ep, int total) {
  return reinterpret_cast<unsigned long long*>(d_ep + (((size_t)total + 1) & ~(size_t)1));
}

ac_status ensure_ep_words(unsigned int** buf, size_t* cap, size_t words) {
  if (words <= *cap) return AC_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, words * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(AC_ERR_OOM, "epoch kernel words: cudaMalloc of %zu bytes failed", words * 4);
  }
  *cap = words;
  return AC_OK;
}

// Count margin of the 16-bit window for a call of `span` time units: a cell commits about
// `span` arrivals (Poisson), with a wide margin (the same test as tb_counts_fit).
unsigned count_window_limit(double span) {
  const double margin = 2.0 * span + 64.0 * std::sqrt(span + 1.0) + 64.0;
  return margin >= 30000.0 ? 0u : (unsigned)(30000.0 - margin);
}

// Zero the counters of an epoch-kernel launch and mark no epoch as the last (device-side
// writes only: nothing waits for a copy engine that other streams' transfers may occupy).
ac_status reset_ep_counters(ac::DevCounters* d_ctr, unsigned* d_ep, size_t ep_words, cudaStream_t st) {
  AC_CUDA(cudaMemsetAsync(d_ctr, 0, sizeof(ac::DevCounters), st));
  AC_CUDA(cudaMemsetAsync(&d_ctr->stop_epoch, 0xFF, sizeof(unsigned), st));
  AC_CUDA(cudaMemsetAsync(d_ep, 0, ep_words * 4, st));
  return AC_OK;
}

// One run call on the epoch kernel.  The count check runs on the device: the count-range
// kernel writes the lattice's (min, max) and the epoch kernel refuses to start when they
// could leave the 16-bit window, in which case *fallback is set and the state is untouched.
// Only the counters are read back, once per launch.
ac_status run_ep(ac_sim* s, long long t_end, bool* fallback) {
  *fallback = false;
  const int D = s->cfg.rounds;
  const size_t N = s->ncells();
  if (!s->key2) {
    if (cudaMalloc(&s->key2, N * 8) != cudaSuccess || cudaMalloc(&s->cnt2, N * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(AC_ERR_OOM, "second state buffer (%zu cells) allocation failed", N);
    }
  }
  const int region = ac::tb_region_for(D, s->cfg.lb == 128);
  int tr = 0, tc = 0;
  ep_tiling(s->rows, s->cols, region, D, &tr, &tc);
  const int total = tr * tc;
  const double span = (double)(t_end - s->t_done) / kTicksPerUnit;
  const int E = ep_epochs(span, D, total);
  const size_t words = ep_words(total, E);
  ac_status st = ensure_ep_words(&s->d_ep, &s->ep_cap, words);
  if (st != AC_OK) return st;
  unsigned* d_range = reinterpret_cast<unsigned*>(s->d_red);
  ac::EpArgs ep{};
  ep.done = s->d_ep;
  ep.ep_count = ep_counts(s->d_ep, total);
  ep.max_epochs = E;
  ep.watchdog_ns = s->cfg.watchdog_ns;
  ep.range = d_range;
  ep.nrange = 1;
  ep.limit = count_window_limit(span);
  const int grid = (int)std::min<long long>((long long)total * E, ac::tb_grid(region));
  ac::DevCounters sum{};
  AC_CUDA(cudaEventRecord(s->ev0, s->stream));
  long long epochs_total = 0;
  for (int launch = 0;; ++launch) {
    ac::LatDesc d = s->host_desc(t_end, 0);
    d.tr = tr;
    d.tc = tc;
    d.cpair = 1;
    d.tmap = ensure_tmaps(s, s->stream);
    AC_CUDA(ac::launch_store_desc(d, s->d_desc, s->stream));
    st = reset_ep_counters(s->d_ctr, s->d_ep, words, s->stream);
    if (st != AC_OK) return st;
    if (launch == 0) {
      AC_CUDA(cudaMemsetAsync(d_range, 0xFF, 4, s->stream));
      AC_CUDA(cudaMemsetAsync(d_range + 1, 0, 4, s->stream));
      AC_CUDA(ac::launch_count_range(&d, d_range, s->stream));
    } else {
      ep.nrange = 0;    // the first launch checked the window for the whole call
    }
    AC_CUDA(ac::launch_ep(s->d_desc, 1, total, region, D, D, s->d_ctr, ep, s->stream, 0, s->d_rates != nullptr));
    ac::DevCounters c{};
    AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
    AC_CUDA(cudaStreamSynchronize(s->stream));
    if (c.error == ac::kEpWindow) {
      if (launch != 0) return fail(AC_ERR_STATE, "epoch kernel: count check refused a later launch");
      *fallback = true;
      return AC_OK;
    }
    sum.events += c.events;
    sum.rounds += c.rounds;
    sum.scanned += c.scanned;
    sum.enabled += c.enabled;
    // every CTA's claims beyond its last item: exactly one that found nothing left
    sum.visits += c.next_item > (unsigned)grid ? c.next_item - (unsigned)grid : 0u;
    sum.polls += c.polls;
    sum.launched += 1;
    if (c.error) {
      sum.error = c.error;
      sum.err_block = c.err_block;
      break;
    }
    // the state after `done` epochs is in the second buffer when `done` is odd
    const unsigned done = (c.stop_epoch != ~0u) ? c.stop_epoch : (unsigned)E;
    if (done & 1u) {
      std::swap(s->key, s->key2);
      std::swap(s->cnt, s->cnt2);
    }
    epochs_total += done;
    if (c.stop_epoch != ~0u) break;
    if ((double)epochs_total * D > 64.0 * (9.0 * std::ceil(span) + 16.0) + 4096.0)
      return fail(AC_ERR_STALL, "epoch kernel: no completion after %lld epochs", epochs_total);
  }
  AC_CUDA(cudaEventRecord(s->ev1, s->stream));
  AC_CUDA(cudaEventSynchronize(s->ev1));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  s->last_grid = grid;
  st = accumulate(s, sum, ms, true);
  if (st != AC_OK) return st;
  s->events += sum.events;
  s->t_done = t_end;
  return AC_OK;
}

// One synchronous round per launch with early commits of certain rejections (the one-round
// kernel's exact path, AC_OPT_EARLY_REJECT): the flip masks of the cells' pending arrivals
// are filled at the start of the call and kept by the commits.
ac_status run_round_er(ac_sim* s, long long t_end) {
  const size_t N = s->ncells();
  if (!s->d_fmask && cudaMalloc(&s->d_fmask, N) != cudaSuccess) {
    cudaGetLastError();
    s->d_fmask = nullptr;
    return fail(AC_ERR_OOM, "flip masks (%zu bytes) allocation failed", N);
  }
  const int total = s->tiles();
  ac::LatDesc d = s->host_desc(t_end, 0);
  d.fmask = s->d_fmask;
  AC_CUDA(cudaMemcpyAsync(s->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s->stream));
  AC_CUDA(cudaMemsetAsync(s->d_ctr, 0, sizeof(ac::DevCounters), s->stream));
  AC_CUDA(ac::launch_publish(s->d_desc, 1, total, s->cfg.lb, 0, s->stream));
  AC_CUDA(cudaEventRecord(s->ev0, s->stream));
  AC_CUDA(ac::launch_fmask(&d, s->stream));
  const double span = (double)(t_end - s->t_done) / kTicksPerUnit;
  int chunk = (int)std::min(4096.0, 9.0 * std::ceil(span) + 16.0);
  int launch_idx = 0, parity = 0;
  unsigned active = 1;
  for (;;) {
    for (int i = 0; i < chunk; ++i) {
      AC_CUDA(ac::launch_round_er(s->d_desc, 1, total, s->cfg.lb, parity, launch_idx, s->d_ctr, s->stream));
      parity ^= 1;
      ++launch_idx;
    }
    AC_CUDA(cudaMemcpyAsync(&active, &s->d_ctr->active[(launch_idx - 1) % 3], sizeof active,
                            cudaMemcpyDeviceToHost, s->stream));
    AC_CUDA(cudaStreamSynchronize(s->stream));
    if (active == 0) break;
    if ((double)launch_idx > 64.0 * (9.0 * std::ceil(span) + 16.0) + 4096.0)
      return fail(AC_ERR_STALL, "round kernel: no completion after %d launches", launch_idx);
    chunk = 16;
  }
  AC_CUDA(cudaEventRecord(s->ev1, s->stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  s->last_grid = total;
  const int saved = s->cfg.rounds;
  s->cfg.rounds = 0;   // not the plain synchronous rounds: no round history or Sec. 4 efficiency
  const ac_status st = accumulate(s, c, ms, true);
  s->cfg.rounds = saved;
  return st;
}

ac_status run_round(ac_sim* s, long long t_end) {
  if (s->model == 0 && s->early_reject && s->cfg.rounds == 1) return run_round_er(s, t_end);
  if (s->model != 0) {
    // the Life automaton and the q-th degree neighbourhood run on the temporal-blocked
    // kernel only (their enable tests need the diagonal / farther cells the region holds)
    int D = 0, R = 0;
    tb_depth(s, &D, &R);
    bool fits = false;
    ac_status st = tb_counts_fit(s, t_end, &fits);
    if (st != AC_OK) return st;
    if (!fits) return fail(AC_ERR_STATE, "event counts too uneven for the temporal-blocked kernel");
    return run_tb(s, t_end, D, R);
  }
  if (tb_applicable(s)) {
    bool fits = false;
    ac_status st = tb_counts_fit(s, t_end, &fits);
    if (st != AC_OK) return st;
    if (fits) return run_tb(s, t_end, s->cfg.rounds, s->cfg.rounds);
    // counts too uneven for the 16-bit window: one exact synchronous round per launch
    const int saved = s->cfg.rounds;
    s->cfg.rounds = 1;
    st = run_round(s, t_end);
    s->cfg.rounds = saved;
    return st;
  }
  const int total = s->tiles();
  const ac::LatDesc d = s->host_desc(t_end, 0);
  AC_CUDA(cudaMemcpyAsync(s->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s->stream));
  AC_CUDA(cudaMemsetAsync(s->d_ctr, 0, sizeof(ac::DevCounters), s->stream));
  AC_CUDA(ac::launch_publish(s->d_desc, 1, total, s->cfg.lb, 0, s->stream));
  const bool exact = (s->cfg.rounds == 1);
  if (exact && s->d_hist == nullptr) {
    s->hist_cap = 1 << 16;
    if (cudaMalloc(&s->d_hist, (size_t)s->hist_cap * 8) != cudaSuccess)
      return fail(AC_ERR_OOM, "round history allocation failed");
    AC_CUDA(cudaMemsetAsync(s->d_hist, 0, (size_t)s->hist_cap * 8, s->stream));
  }
  AC_CUDA(cudaEventRecord(s->ev0, s->stream));
  const double span = (double)(t_end - s->t_done) / kTicksPerUnit;
  int chunk = (int)std::min(4096.0, 9.0 * std::ceil(span) / std::max(1, s->cfg.rounds) + 16.0);
  int launch_idx = 0, parity = 0;
  unsigned active = 1;
  for (;;) {
    for (int i = 0; i < chunk; ++i) {
      AC_CUDA(ac::launch_round(s->d_desc, 1, total, s->cfg, parity, launch_idx, s->d_ctr,
                               exact ? s->d_hist : nullptr, s->hist_cap,
                               (int)std::min<unsigned long long>(s->global_rounds + launch_idx, 1u << 30),
                               s->stream));
      parity ^= 1;
      ++launch_idx;
    }
    AC_CUDA(cudaMemcpyAsync(&active, &s->d_ctr->active[(launch_idx - 1) % 3], sizeof active,
                            cudaMemcpyDeviceToHost, s->stream));
    AC_CUDA(cudaStreamSynchronize(s->stream));
    if (active == 0) break;
    // every synchronous round commits the globally smallest pending arrival, so a
    // run needs at most (pending arrivals) rounds; far beyond the ~8.3 rounds per
    // unit time of Sec. 4 only a defect could keep tiles active
    if ((double)launch_idx > 64.0 * (9.0 * std::ceil(span) + 16.0) + 4096.0)
      return fail(AC_ERR_STALL, "round kernel: no completion after %d launches", launch_idx);
    chunk = 16;
  }
  AC_CUDA(cudaEventRecord(s->ev1, s->stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  s->last_grid = total;
  if (exact) {
    // rounds with at least one commit form a prefix of this call's launches
    const long long first = (long long)s->global_rounds;
    const long long m = std::max(0ll, std::min<long long>(c.launched, (long long)s->hist_cap - first));
    std::vector<unsigned long long> h((size_t)m);
    if (m > 0) {
      AC_CUDA(cudaMemcpyAsync(h.data(), s->d_hist + first, (size_t)m * 8, cudaMemcpyDeviceToHost, s->stream));
      AC_CUDA(cudaStreamSynchronize(s->stream));
    }
    unsigned productive = 0;
    while (productive < (unsigned)m && h[productive] != 0) ++productive;
    c.launched = productive;
  }
  return accumulate(s, c, ms, true);
}

ac_status run_blocked(ac_sim* s, long long t_end) {
  const int total = s->tiles();
  int per_sm = 0;
  const int maxc = ac::blocked_max_ctas(s->cfg.lb, &per_sm);
  if (maxc <= 0) return fail(AC_ERR_CUDA, "blocked kernel cannot be resident (tile side %d)", s->cfg.lb);
  const int grid = std::min(total, maxc);
  const ac::LatDesc d = s->host_desc(t_end, 0);
  AC_CUDA(cudaMemcpyAsync(s->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s->stream));
  AC_CUDA(cudaMemsetAsync(s->d_ctr, 0, sizeof(ac::DevCounters), s->stream));
  AC_CUDA(cudaMemsetAsync(s->d_tile_done, 0, (size_t)total * 4, s->stream));
  AC_CUDA(ac::launch_publish(s->d_desc, 1, total, s->cfg.lb, 0, s->stream));
  AC_CUDA(cudaEventRecord(s->ev0, s->stream));
  AC_CUDA(ac::launch_blocked(s->d_desc, 1, total, s->cfg, grid, s->d_tile_done, s->d_ctr, s->stream));
  AC_CUDA(cudaEventRecord(s->ev1, s->stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  s->last_grid = grid;
  s->ctas_per_sm = per_sm;
  return accumulate(s, c, ms, false);
}

ac_status read_event_counter(ac_sim* s, unsigned long long* v) {
  AC_CUDA(cudaMemcpyAsync(v, s->d_events, 8, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  return AC_OK;
}

constexpr int kTbChunk = 8;   // launches per captured chunk

// Batched temporal-blocked rounds: every launch covers the tiles of all handles (one
// work list), so all lattices advance by the same synchronous rounds per launch.
ac_status batch_run_tb(int32_t n, ac_sim* const* sims, const int64_t* t_end, BatchRunner* R) {
  const cudaStream_t stream = R->stream;
  for (int i = 0; i < n; ++i) {
    ac_sim* s = sims[i];
    if (!s->key2) {
      if (cudaMalloc(&s->key2, s->ncells() * 8) != cudaSuccess || cudaMalloc(&s->cnt2, s->ncells() * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(AC_ERR_OOM, "second state buffer allocation failed (handle %d)", i);
      }
    }
  }
  int base = 0;
  double span = 0.0;
  for (int i = 0; i < n; ++i) {
    int tr = 0, tc = 0;
    tb_tiling_batch(sims[i]->rows, sims[i]->cols, R->region, R->halo, &tr, &tc);
    R->h_desc[i] = sims[i]->host_desc(t_end[i], base);
    R->h_desc[i].tr = tr;
    R->h_desc[i].tc = tc;
    base += tr * tc;
    span = std::max(span, (double)(t_end[i] - sims[i]->t_done) / kTicksPerUnit);
  }
  const int total = base;
  AC_CUDA(cudaMemcpyAsync(R->d_desc, R->h_desc, sizeof(ac::LatDesc) * n, cudaMemcpyHostToDevice, stream));
  // the 16-bit count window must hold every region of every lattice for the whole call
  std::vector<unsigned> range(2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    range[2 * i] = 0xFFFFFFFFu;
    range[2 * i + 1] = 0u;
  }
  AC_CUDA(cudaMemcpyAsync(R->d_range, range.data(), range.size() * 4, cudaMemcpyHostToDevice, stream));
  size_t max_cells = 0;
  for (int i = 0; i < n; ++i) max_cells = std::max(max_cells, sims[i]->ncells());
  AC_CUDA(ac::launch_count_range_batch(R->d_desc, n, max_cells, R->d_range, stream));
  AC_CUDA(cudaMemcpyAsync(range.data(), R->d_range, range.size() * 4, cudaMemcpyDeviceToHost, stream));
  std::vector<unsigned long long> before(n), after(n);
  for (int i = 0; i < n; ++i)
    AC_CUDA(cudaMemcpyAsync(&before[i], sims[i]->d_events, 8, cudaMemcpyDeviceToHost, stream));
  AC_CUDA(cudaStreamSynchronize(stream));
  const double margin = 2.0 * span + 64.0 * std::sqrt(span + 1.0) + 64.0;
  for (int i = 0; i < n; ++i) {
    if ((double)(range[2 * i + 1] - range[2 * i]) + margin >= 30000.0) {
      // very uneven counts (loaded states only): run every handle on its own, exactly
      for (int k = 0; k < n; ++k) {
        ac_status st = ac_run_until_ticks(sims[k], t_end[k]);
        if (st != AC_OK) return st;
      }
      return AC_OK;
    }
  }
  AC_CUDA(cudaMemsetAsync(R->d_ctr, 0, sizeof(ac::DevCounters), stream));
  AC_CUDA(cudaEventRecord(R->ev0, stream));
  const bool use_graph = R->calls++ > 0;   // repeated calls on the same handles replay a captured chunk
  if (use_graph && !R->chunk_exec) {
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; i < kTbChunk && e == cudaSuccess; ++i)
      e = ac::launch_tb(R->d_desc, n, total, R->region, R->halo, R->halo, R->d_ctr, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(stream, &g);
    if (e == cudaSuccess) e = e2;
    R->chunk_graph = g;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&R->chunk_exec, g, 0);
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "round-kernel graph capture failed: %s", cudaGetErrorString(e));
  }
  int issued = 0;
  for (;;) {
    if (use_graph) {
      AC_CUDA(cudaGraphLaunch(R->chunk_exec, stream));
    } else {
      for (int i = 0; i < kTbChunk; ++i) AC_CUDA(ac::launch_tb(R->d_desc, n, total, R->region, R->halo, R->halo, R->d_ctr, stream));
    }
    issued += kTbChunk;
    ac::DevCounters cc{};
    AC_CUDA(cudaMemcpyAsync(&cc, R->d_ctr, sizeof cc, cudaMemcpyDeviceToHost, stream));
    AC_CUDA(cudaStreamSynchronize(stream));
    if (cc.seq < (unsigned)issued || cc.error || (cc.seq > 0 && cc.active[(cc.seq + 2) % 3] == 0)) break;
    if ((double)issued * R->halo > 64.0 * (9.0 * std::ceil(span) + 16.0) + 4096.0)
      return fail(AC_ERR_STALL, "batched round kernel: no completion after %d launches", issued);
  }
  AC_CUDA(cudaEventRecord(R->ev1, stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, R->d_ctr, sizeof c, cudaMemcpyDeviceToHost, stream));
  for (int i = 0; i < n; ++i)
    AC_CUDA(cudaMemcpyAsync(&after[i], sims[i]->d_events, 8, cudaMemcpyDeviceToHost, stream));
  AC_CUDA(cudaStreamSynchronize(stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, R->ev0, R->ev1));
  const unsigned good = (c.error == AC_ERR_STATE) ? c.seq - 1u : c.seq;
  for (int i = 0; i < n; ++i) {
    ac_sim* s = sims[i];
    if (good & 1u) {
      std::swap(s->key, s->key2);
      std::swap(s->cnt, s->cnt2);
    }
    if (c.error) continue;
    s->events += after[i] - before[i];
    s->t_done = t_end[i];
    s->launches += c.launched;
    s->device_ms += ms;
    s->last_grid = std::min(total, ac::tb_grid(R->region));
  }
  if (c.error) return fail((ac_status)c.error, "batched round kernel: device error %d", c.error);
  sims[0]->rounds += c.rounds;
  sims[0]->scanned += c.scanned;
  sims[0]->enabled += c.enabled;
  return check_bounds();
}

// Batched epoch kernel: one persistent launch over the tiles of every handle (one work
// list; each lattice's tiles wait only on that lattice's neighbour tiles), so all
// lattices advance by the same epochs of D rounds.
ac_status batch_run_ep(int32_t n, ac_sim* const* sims, const int64_t* t_end, BatchRunner* R) {
  const cudaStream_t stream = R->stream;
  bool any_rates = false;   // the rate-free kernel serves batches without per-cell rates
  for (int i = 0; i < n; ++i) any_rates |= sims[i]->d_rates != nullptr;
  for (int i = 0; i < n; ++i) {
    ac_sim* s = sims[i];
    if (!s->key2) {
      if (cudaMalloc(&s->key2, s->ncells() * 8) != cudaSuccess || cudaMalloc(&s->cnt2, s->ncells() * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(AC_ERR_OOM, "second state buffer allocation failed (handle %d)", i);
      }
    }
  }
  const int D = R->halo;
  int base = 0;
  double span = 0.0;
  std::vector<int> tiles_tr(n), tiles_tc(n);
  for (int i = 0; i < n; ++i) {
    ep_tiling(sims[i]->rows, sims[i]->cols, R->region, D, &tiles_tr[i], &tiles_tc[i]);
    base += tiles_tr[i] * tiles_tc[i];
    span = std::max(span, (double)(t_end[i] - sims[i]->t_done) / kTicksPerUnit);
  }
  const int total = base;
  // the 16-bit count window must hold every region of every lattice for the whole call
  auto fill_desc = [&]() {
    int b = 0;
    for (int i = 0; i < n; ++i) {
      R->h_desc[i] = sims[i]->host_desc(t_end[i], b);
      R->h_desc[i].tr = tiles_tr[i];
      R->h_desc[i].tc = tiles_tc[i];
      R->h_desc[i].cpair = 1;
      R->h_desc[i].tmap = ensure_tmaps(sims[i], stream);
      b += tiles_tr[i] * tiles_tc[i];
    }
  };
  fill_desc();
  AC_CUDA(cudaMemcpyAsync(R->d_desc, R->h_desc, sizeof(ac::LatDesc) * n, cudaMemcpyHostToDevice, stream));
  std::vector<unsigned> range(2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    range[2 * i] = 0xFFFFFFFFu;
    range[2 * i + 1] = 0u;
  }
  AC_CUDA(cudaMemcpyAsync(R->d_range, range.data(), range.size() * 4, cudaMemcpyHostToDevice, stream));
  size_t max_cells = 0;
  for (int i = 0; i < n; ++i) max_cells = std::max(max_cells, sims[i]->ncells());
  AC_CUDA(ac::launch_count_range_batch(R->d_desc, n, max_cells, R->d_range, stream));
  AC_CUDA(cudaMemcpyAsync(range.data(), R->d_range, range.size() * 4, cudaMemcpyDeviceToHost, stream));
  std::vector<unsigned long long> before(n), after(n);
  for (int i = 0; i < n; ++i)
    AC_CUDA(cudaMemcpyAsync(&before[i], sims[i]->d_events, 8, cudaMemcpyDeviceToHost, stream));
  AC_CUDA(cudaStreamSynchronize(stream));
  const double margin = 2.0 * span + 64.0 * std::sqrt(span + 1.0) + 64.0;
  for (int i = 0; i < n; ++i) {
    if ((double)(range[2 * i + 1] - range[2 * i]) + margin >= 30000.0) {
      // very uneven counts (loaded states only): run every handle on its own, exactly
      for (int k = 0; k < n; ++k) {
        ac_status st = ac_run_until_ticks(sims[k], t_end[k]);
        if (st != AC_OK) return st;
      }
      return AC_OK;
    }
  }
  const int E = ep_epochs(span, D, total);
  ac_status st = ensure_ep_words(&R->d_ep, &R->ep_cap, ep_words(total, E));
  if (st != AC_OK) return st;
  ac::EpArgs ep{};
  ep.done = R->d_ep;
  ep.ep_count = ep_counts(R->d_ep, total);
  ep.max_epochs = E;
  ep.watchdog_ns = sims[0]->cfg.watchdog_ns;
  ac::DevCounters c0{};
  c0.stop_epoch = ~0u;
  ac::DevCounters sum{};
  AC_CUDA(cudaEventRecord(R->ev0, stream));
  long long epochs_total = 0;
  const int grid = (int)std::min<long long>((long long)total * E, ac::tb_grid(R->region));
  for (;;) {
    AC_CUDA(cudaMemcpyAsync(R->d_ctr, &c0, sizeof c0, cudaMemcpyHostToDevice, stream));
    AC_CUDA(cudaMemsetAsync(R->d_ep, 0, ep_words(total, E) * 4, stream));
    AC_CUDA(ac::launch_ep(R->d_desc, n, total, R->region, D, D, R->d_ctr, ep, stream, 0, any_rates));
    ac::DevCounters c{};
    AC_CUDA(cudaMemcpyAsync(&c, R->d_ctr, sizeof c, cudaMemcpyDeviceToHost, stream));
    AC_CUDA(cudaStreamSynchronize(stream));
    sum.rounds += c.rounds;
    sum.scanned += c.scanned;
    sum.enabled += c.enabled;
    sum.visits += c.next_item > (unsigned)grid ? c.next_item - (unsigned)grid : 0u;
    sum.polls += c.polls;
    sum.launched += 1;
    if (c.error) {
      sum.error = c.error;
      sum.err_block = c.err_block;
      break;
    }
    const unsigned done = (c.stop_epoch != ~0u) ? c.stop_epoch : (unsigned)E;
    if (done & 1u) {
      for (int i = 0; i < n; ++i) {
        std::swap(sims[i]->key, sims[i]->key2);
        std::swap(sims[i]->cnt, sims[i]->cnt2);
      }
      fill_desc();
      AC_CUDA(cudaMemcpyAsync(R->d_desc, R->h_desc, sizeof(ac::LatDesc) * n, cudaMemcpyHostToDevice, stream));
    }
    epochs_total += done;
    if (c.stop_epoch != ~0u) break;
    if ((double)epochs_total * D > 64.0 * (9.0 * std::ceil(span) + 16.0) + 4096.0)
      return fail(AC_ERR_STALL, "batched epoch kernel: no completion after %lld epochs", epochs_total);
  }
  AC_CUDA(cudaEventRecord(R->ev1, stream));
  for (int i = 0; i < n; ++i)
    AC_CUDA(cudaMemcpyAsync(&after[i], sims[i]->d_events, 8, cudaMemcpyDeviceToHost, stream));
  AC_CUDA(cudaStreamSynchronize(stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, R->ev0, R->ev1));
  if (sum.error == AC_ERR_STALL) return fail(AC_ERR_STALL, "batched epoch kernel: device watchdog (block %d)", sum.err_block);
  if (sum.error) return fail((ac_status)sum.error, "batched epoch kernel: device error %d", sum.error);
  for (int i = 0; i < n; ++i) {
    ac_sim* s = sims[i];
    s->events += after[i] - before[i];
    s->t_done = t_end[i];
    s->launches += sum.launched;
    s->device_ms += ms;
    s->last_grid = grid;
  }
  sims[0]->rounds += sum.rounds;
  sims[0]->scanned += sum.scanned;
  sims[0]->enabled += sum.enabled;
  sims[0]->visits += sum.visits;
  sims[0]->polls += sum.polls;
  return check_bounds();
}

ac_status run_core(ac_sim* sim, long long t_end) {
  if (sim->cfg.kernel == ac::kKernelEpoch && ep_applicable(sim)) {
    bool fallback = false;
    ac_status st = run_ep(sim, t_end, &fallback);
    // counts too uneven for the 16-bit window (nothing was run): the round kernel's exact
    // one-round path below
    if (st != AC_OK || !fallback) return st;
  }
  unsigned long long before = 0, after = 0;
  ac_status st = read_event_counter(sim, &before);
  if (st != AC_OK) return st;
  // the epoch kernel's other cases (frames, odd sizes or halos) run on the round kernel
  st = (sim->cfg.kernel != ac::kKernelBlocked) ? run_round(sim, t_end) : run_blocked(sim, t_end);
  if (st != AC_OK) return st;
  st = read_event_counter(sim, &after);
  if (st != AC_OK) return st;
  sim->events += after - before;
  sim->t_done = t_end;
  return AC_OK;
}

void frames_off(ac_sim* s) {
  if (s->frames) cudaFree(s->frames);
  s->frames = nullptr;
  s->f_B = 0;
  s->f_dt = 0;
  s->f_K = 0;
}

// Hand frame f_K to fn (a device pointer, or a copy in the pinned host buffer) and
// retire it.  The frame is complete: every cell's tick is above K dt.
// Asynchronous transfers: a pending load is waited for (on the host: its validation result
// decides whether the handle's time changes) and a pending read is ordered before the
// handle's next device work (on the device) by every call that uses the handle's state.
ac_status settle_async(ac_sim* s) {
  if (s->load_pending) {
    s->load_pending = false;
    AC_CUDA(cudaEventSynchronize(s->ev_load));
    if (*s->h_bad != ~0ull)
      return fail(AC_ERR_ARG,
                  "asynchronous load: cell %llu has a spin other than +-1 or a tick outside [max(t_done, 1), 2^61); "
                  "the state was left unchanged", *s->h_bad);
    s->t_done = s->load_t_done;
    frames_off(s);
  }
  if (s->read_pending) {
    s->read_pending = false;
    AC_CUDA(cudaStreamWaitEvent(s->stream, s->ev_read, 0));
  }
  return AC_OK;
}

ac_status ensure_async(ac_sim* s) {
  if (!s->ev_work) {
    if (cudaEventCreateWithFlags(&s->ev_work, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_load, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_read, cudaEventDisableTiming) != cudaSuccess)
      return fail(AC_ERR_CUDA, "cudaEventCreate failed");
  }
  if (!s->h_bad && cudaHostAlloc(&s->h_bad, sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    s->h_bad = nullptr;
    return fail(AC_ERR_OOM, "pinned host word allocation failed");
  }
  return AC_OK;
}

#define AC_SETTLE(sim)                            \
  do {                                            \
    ac_status st_ = settle_async(sim);            \
    if (st_ != AC_OK) return st_;                 \
  } while (0)

ac_status deliver_frame(ac_sim* s, ac_frame_fn fn, void* user, int on_host) {
  const size_t N = s->ncells();
  const int8_t* slot = s->frames + (size_t)(s->f_K % s->f_B) * N;
  if (fn) {
    if (on_host) {
      AC_CUDA(cudaMemcpyAsync(s->frame_host, slot, N, cudaMemcpyDeviceToHost, s->stream));
      AC_CUDA(cudaStreamSynchronize(s->stream));
      fn(user, s->f_K, s->frame_host, N);
    } else {
      AC_CUDA(cudaStreamSynchronize(s->stream));
      fn(user, s->f_K, slot, N);
    }
  }
  ++s->f_K;
  return AC_OK;
}

// Frames on the temporal-blocked kernel, with the window slid one frame at a time:
// between launch chunks the host reads the smallest tick of the last launch's output
// state, hands out every open frame below it, reopens those slots (filled from the
// current state buffer) and raises the commit cap to (f_K + B) dt + 1 for the next
// launches.  The lag bound is the same as with whole windows; no launch waits for
// the whole lattice to reach a window's end.
ac_status run_tb_frames(ac_sim* s, long long t_end, ac_frame_fn fn, void* user, int on_host, int D, int R) {
  const size_t N = s->ncells();
  if (!s->key2) {
    if (cudaMalloc(&s->key2, N * 8) != cudaSuccess || cudaMalloc(&s->cnt2, N * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(AC_ERR_OOM, "second state buffer (%zu cells) allocation failed", N);
    }
  }
  unsigned long long ev_before = 0, ev_after = 0;
  ac_status st = read_event_counter(s, &ev_before);
  if (st != AC_OK) return st;
  const int region = ac::tb_region_for_model(D, s->model, s->q, s->cfg.lb == 128);
  int tr = 0, tc = 0;
  tb_tiling(s->rows, s->cols, region, D, ac::tb_grid(region), &tr, &tc);
  const int total = tr * tc;
  long long cap = std::min<long long>(t_end, (s->f_K + s->f_B) * s->f_dt + 1);
  auto upload = [&](long long c) -> ac_status {
    ac::LatDesc d = s->host_desc(c, 0);
    d.tr = tr;
    d.tc = tc;
    AC_CUDA(cudaMemcpyAsync(s->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s->stream));
    return AC_OK;
  };
  st = upload(cap);
  if (st != AC_OK) return st;
  ac::DevCounters c0{};
  c0.kmin[0] = c0.kmin[1] = c0.kmin[2] = ~0ull;
  AC_CUDA(cudaMemcpyAsync(s->d_ctr, &c0, sizeof c0, cudaMemcpyHostToDevice, s->stream));
  AC_CUDA(cudaEventRecord(s->ev0, s->stream));
  // about 8.3 synchronous rounds per unit time (Sec. 4), D per launch: check often
  // enough that the cap is raised before cells wait long on it
  const double lag = (double)s->f_B * (double)s->f_dt / kTicksPerUnit;
  const int chunk = std::max(1, std::min(4, (int)(lag * 8.3 / R / 2.0)));
  const double span = (double)(t_end - s->t_done) / kTicksPerUnit;
  const double max_launches = 64.0 * (9.0 * std::ceil(span) + 16.0) / D + 4096.0;
  int issued = 0;
  ac::DevCounters c{};
  for (;;) {
    for (int i = 0; i < chunk; ++i) {
      AC_CUDA(ac::launch_tb(s->d_desc, 1, total, region, D, R, s->d_ctr, s->stream, true, s->model));
      ++issued;
    }
    AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
    AC_CUDA(cudaStreamSynchronize(s->stream));
    if (c.error) break;
    const bool idle = c.seq > 0 && c.active[(c.seq + 2) % 3] == 0;
    const long long W = s->f_K + s->f_B;
    const long long first = s->f_K;
    if (c.seq > 0) {
      const long long tmin = (long long)(c.kmin[(c.seq - 1) % 3] >> 1);
      while (s->f_K < W && s->f_K * s->f_dt < tmin && s->f_K * s->f_dt < t_end) {
        st = deliver_frame(s, fn, user, on_host);
        if (st != AC_OK) return st;
      }
    }
    if (s->f_K > first) {
      // reopened slots, filled from the state the last completed launch wrote
      ac::LatDesc dd = s->host_desc(cap, 0);
      if (c.seq & 1u) {
        dd.key = s->key2;
        dd.cnt = s->cnt2;
      }
      AC_CUDA(ac::launch_frames_fill(&dd, W, (int)(s->f_K - first), s->stream));
      const long long ncap = std::min<long long>(t_end, (s->f_K + s->f_B) * s->f_dt + 1);
      st = upload(ncap);
      if (st != AC_OK) return st;
      if (idle && ncap > cap) {   // the last launch found nothing below the old cap
        const unsigned one = 1u;
        AC_CUDA(cudaMemcpyAsync(&s->d_ctr->active[(c.seq + 2) % 3], &one, sizeof one, cudaMemcpyHostToDevice,
                                s->stream));
      }
      cap = ncap;
    } else if (idle || c.seq < (unsigned)issued) {
      if (cap >= t_end) break;       // everything below t_end is committed
    }
    if ((double)issued > max_launches)
      return fail(AC_ERR_STALL, "round kernel with frames: no completion after %d launches", issued);
  }
  AC_CUDA(cudaEventRecord(s->ev1, s->stream));
  AC_CUDA(cudaMemcpyAsync(&c, s->d_ctr, sizeof c, cudaMemcpyDeviceToHost, s->stream));
  AC_CUDA(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  const unsigned good = (c.error == AC_ERR_STATE) ? c.seq - 1u : c.seq;
  if (good & 1u) {
    std::swap(s->key, s->key2);
    std::swap(s->cnt, s->cnt2);
  }
  s->last_grid = std::min(total, ac::tb_grid(region));
  st = accumulate(s, c, ms, true);
  if (st != AC_OK) return st;
  st = read_event_counter(s, &ev_after);
  if (st != AC_OK) return st;
  s->events += ev_after - ev_before;
  s->t_done = t_end;
  return AC_OK;
}

// Snapshot frames (Fig. 3.7).  Frames [f_K, f_K + B) are open.  Commits are capped at
// tick <= (f_K + B) dt -- the figure's lag bound: no cell gets more than B frames ahead
// of the oldest frame not yet handed out -- so every frame a commit must write is
// open.  After the capped run the open frames are complete (all arrivals <= K dt
// committed); each is handed to fn in order, its slot is reopened for frame K + B and
// filled where no later commit will write it.
ac_status run_frames(ac_sim* s, long long t_end, ac_frame_fn fn, void* user, int on_host) {
  const size_t N = s->ncells();
  if (fn && on_host && !s->frame_host) {
    if (cudaMallocHost(&s->frame_host, N) != cudaSuccess) {
      cudaGetLastError();
      s->frame_host = nullptr;
      return fail(AC_ERR_OOM, "pinned frame buffer (%zu bytes) allocation failed", N);
    }
  }
  // the temporal-blocked kernel slides the window frame by frame (run_tb_frames); the
  // other kernels run whole windows: to the cap, then every open frame is complete
  if (t_end > s->t_done && s->cfg.kernel != ac::kKernelBlocked && (s->model != 0 || tb_applicable(s))) {
    int D = 0, R = 0;
    tb_depth(s, &D, &R);
    bool fits = false;
    ac_status st = tb_counts_fit(s, t_end, &fits);
    if (st != AC_OK) return st;
    if (fits) {
      st = run_tb_frames(s, t_end, fn, user, on_host, D, R);
      if (st != AC_OK) return st;
    } else if (s->model != 0) {
      return fail(AC_ERR_STATE, "event counts too uneven for the temporal-blocked kernel");
    }
  }
  for (;;) {
    const long long W = s->f_K + s->f_B;
    const long long cap = std::min<long long>(t_end, W * s->f_dt + 1);
    if (cap > s->t_done) {
      ac_status st = run_core(s, cap);
      if (st != AC_OK) return st;
    }
    const long long first = s->f_K;
    while (s->f_K < W && s->f_K * s->f_dt + 1 <= s->t_done) {
      ac_status st = deliver_frame(s, fn, user, on_host);
      if (st != AC_OK) return st;
    }
    if (s->f_K > first) {
      const ac::LatDesc d = s->host_desc(s->t_done, 0);
      AC_CUDA(ac::launch_frames_fill(&d, W, (int)(s->f_K - first), s->stream));
    }
    // done when the run reached t_end and the next frame is not complete (a frame just
    // reopened and already complete -- every cell past its tick -- is handed out first)
    if (s->t_done >= t_end && s->f_K * s->f_dt + 1 > s->t_done) break;
  }
  AC_CUDA(cudaStreamSynchronize(s->stream));
  return AC_OK;
}

}  // namespace

extern "C" {

const char* ac_last_error(void) { return g_err.c_str(); }

ac_status ac_thresholds(double beta, double J, double h, uint32_t thr[10]) {
  if (!thr) return fail(AC_ERR_ARG, "thr is NULL");
  if (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(J) || !std::isfinite(h))
    return fail(AC_ERR_ARG, "beta must be finite and >= 0; J, h finite");
  ac::make_thresholds(beta, J, h, thr);
  return AC_OK;
}

ac_status ac_create(ac_lattice lat, double beta, double J, double h, uint64_t seed, ac_sim** out) {
  if (!out) return fail(AC_ERR_ARG, "out is NULL");
  *out = nullptr;
  ac_status st = check_params(lat, beta, J, h);
  if (st != AC_OK) return st;
  return create_one(lat, beta, J, h, seed, out);
}

ac_status ac_create_life(ac_lattice lat, uint32_t density, uint32_t birth, uint32_t survive, uint64_t seed,
                         ac_sim** out) {
  if (!out) return fail(AC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (lat.rows < 4 || lat.cols < 4) return fail(AC_ERR_ARG, "Life needs rows, cols >= 4 (got %d x %d)", lat.rows, lat.cols);
  if (birth > 0x1FFu || survive > 0x1FFu) return fail(AC_ERR_ARG, "birth and survive are 9-bit masks (bits 0..8)");
  ac_status st = check_params(lat, 0.0, 0.0, 0.0);
  if (st != AC_OK) return st;
  st = create_one(lat, 0.0, 0.0, 0.0, seed, out);
  if (st != AC_OK) return st;
  ac_sim* s = *out;
  s->model = 1;
  s->life_birth = birth;
  s->life_survive = survive;
  s->life_density = density;
  s->cfg.kernel = ac::kKernelRound;
  s->cfg.rounds = 6;
  const ac::LatDesc d = s->host_desc(0, 0);
  cudaError_t e = ac::launch_init(&d, lat.init, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    free_sim(s);
    *out = nullptr;
    return fail(AC_ERR_CUDA, "Life initialisation failed: %s", cudaGetErrorString(e));
  }
  return AC_OK;
}

ac_status ac_create_q(ac_lattice lat, double beta, double J, double h, int32_t q, uint64_t seed, ac_sim** out) {
  if (!out) return fail(AC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (q < 2 || q > 3) return fail(AC_ERR_ARG, "q must be 2 or 3 (q = 1 is ac_create)");
  if (lat.rows < 4 * q || lat.cols < 4 * q) return fail(AC_ERR_ARG, "rows, cols must be >= 4q (got %d x %d)", lat.rows, lat.cols);
  ac_status st = check_params(lat, beta, J, h);
  if (st != AC_OK) return st;
  st = create_one(lat, beta, J, h, seed, out);
  if (st != AC_OK) return st;
  ac_sim* s = *out;
  s->model = 2;
  s->q = q;
  const int M = 2 * q * (q + 1);
  for (int sp = 0; sp < 2; ++sp) {
    const double sv = sp ? 1.0 : -1.0;
    for (int j = 0; j <= M; ++j) {
      const double S = (double)(2 * j - M);
      const double p = 1.0 / (1.0 + std::exp(beta * 2.0 * sv * (J * S + h)));
      const double v = std::ldexp(p, 32);
      s->thr[j + (M + 1) * sp] = (v < 4294967295.0) ? (uint32_t)std::floor(v) : 0xFFFFFFFFu;
    }
  }
  s->cfg.kernel = ac::kKernelRound;
  s->cfg.rounds = 6;
  return AC_OK;
}

ac_status ac_set_stream(ac_sim* sim, void* stream) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  sim->stream = (cudaStream_t)stream;
  drop_runners_of(sim);
  return AC_OK;
}

ac_status ac_configure(ac_sim* sim, int32_t kernel, int32_t Lb, int32_t rounds, int32_t polls) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  if (kernel != AC_KERNEL_ROUND && kernel != AC_KERNEL_BLOCKED && kernel != AC_KERNEL_EPOCH)
    return fail(AC_ERR_ARG, "kernel must be AC_KERNEL_ROUND, AC_KERNEL_BLOCKED or AC_KERNEL_EPOCH");
  if (Lb != 32 && Lb != 64 && Lb != 128) return fail(AC_ERR_ARG, "Lb must be 32, 64 or 128");
  if (rounds < 1 || rounds > 1 << 20) return fail(AC_ERR_ARG, "rounds must be in [1, 2^20]");
  if (polls < 0 || polls > 1 << 20) return fail(AC_ERR_ARG, "polls must be in [0, 2^20]");
  if (sim->model != 0 && kernel != AC_KERNEL_ROUND)
    return fail(AC_ERR_ARG, "the Life automaton and the q-th degree neighbourhood run on the round kernel only");
  sim->cfg.kernel = kernel;
  sim->cfg.lb = Lb;
  sim->cfg.threads = 4 * Lb;
  if (kernel != AC_KERNEL_BLOCKED) {
    sim->cfg.rounds = rounds;
  } else {
    sim->cfg.refresh = rounds;
    sim->cfg.polls = polls;
  }
  drop_runners_of(sim);
  return alloc_edges(sim);
}

ac_status ac_run_until_ticks(ac_sim* sim, int64_t t_end) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(sim);
  if (t_end < sim->t_done) return fail(AC_ERR_ARG, "t_end %lld is below the previous t_end %lld",
                                       (long long)t_end, sim->t_done);
  if (t_end >= kTickLimit) return fail(AC_ERR_ARG, "t_end must be < 2^61");
  if (sim->f_B > 0) return run_frames(sim, t_end, nullptr, nullptr, 0);
  return run_core(sim, t_end);
}

ac_status ac_set_rates(ac_sim* sim, const uint32_t* m) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(sim);
  if (sim->t_done != 0) return fail(AC_ERR_STATE, "rates are set at time 0 (before the first run or after ac_reset)");
  if (sim->model != 0) return fail(AC_ERR_ARG, "per-cell rates apply to the Ising array");
  const size_t N = sim->ncells();
  if (!m) {
    cudaFree(sim->d_rates);
    sim->d_rates = nullptr;
  } else {
    for (size_t c = 0; c < N; ++c)
      if (m[c] == 0u) return fail(AC_ERR_ARG, "rate multiplier of cell %zu is 0 (needs m >= 1)", c);
    if (!sim->d_rates && cudaMalloc(&sim->d_rates, N * 4) != cudaSuccess) {
      cudaGetLastError();
      sim->d_rates = nullptr;
      return fail(AC_ERR_OOM, "rate array (%zu cells) allocation failed", N);
    }
    AC_CUDA(cudaMemcpyAsync(sim->d_rates, m, N * 4, cudaMemcpyHostToDevice, sim->stream));
  }
  drop_runners_of(sim);
  return ac_reset(sim, sim->seed, sim->init);   // first arrivals drawn at the new rates
}

ac_status ac_frames_configure(ac_sim* sim, int64_t dt_ticks, int64_t K0, int32_t B) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(sim);
  if (B == 0) {
    frames_off(sim);
    return AC_OK;
  }
  if (B < 1 || B > AC_MAX_FRAMES) return fail(AC_ERR_ARG, "B must be in [1, %d] (or 0 to turn frames off)", AC_MAX_FRAMES);
  if (dt_ticks < 1 || dt_ticks > (kTickLimit / 2) / (B + 1)) return fail(AC_ERR_ARG, "dt_ticks must be in [1, 2^60 / (B + 1)]");
  if (K0 < 0 || K0 > (kTickLimit / 2) / dt_ticks) return fail(AC_ERR_ARG, "K0 must be >= 0 and K0 * dt_ticks < 2^60");
  if (K0 * dt_ticks + 1 < sim->t_done)
    return fail(AC_ERR_ARG, "frame K0 = %lld (tick %lld) is before the state's time %lld", (long long)K0,
                (long long)(K0 * dt_ticks), sim->t_done);
  frames_off(sim);
  const size_t N = sim->ncells();
  if (cudaMalloc(&sim->frames, (size_t)B * N) != cudaSuccess) {
    cudaGetLastError();
    sim->frames = nullptr;
    return fail(AC_ERR_OOM, "%d frames of %zu cells: allocation failed", B, N);
  }
  sim->f_B = B;
  sim->f_dt = dt_ticks;
  sim->f_K = K0;
  const ac::LatDesc d = sim->host_desc(sim->t_done, 0);
  AC_CUDA(ac::launch_frames_fill(&d, K0, B, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  return AC_OK;
}

ac_status ac_run_until_frames(ac_sim* sim, int64_t t_end, ac_frame_fn fn, void* user, int32_t on_host) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(sim);
  if (sim->f_B <= 0) return fail(AC_ERR_ARG, "no frames configured (ac_frames_configure)");
  if (t_end < sim->t_done) return fail(AC_ERR_ARG, "t_end %lld is below the previous t_end %lld",
                                       (long long)t_end, sim->t_done);
  if (t_end >= kTickLimit) return fail(AC_ERR_ARG, "t_end must be < 2^61");
  return run_frames(sim, t_end, fn, user, on_host);
}

ac_status ac_frames_status(const ac_sim* sim, int64_t* next_K, int32_t* B, int64_t* dt_ticks) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  if (next_K) *next_K = sim->f_K;
  if (B) *B = sim->f_B;
  if (dt_ticks) *dt_ticks = sim->f_dt;
  return AC_OK;
}

ac_status ac_run_until(ac_sim* sim, double T) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  if (!std::isfinite(T) || T < 0.0) return fail(AC_ERR_ARG, "T must be finite and >= 0");
  const double ticks = std::floor(T * kTicksPerUnit);
  if (ticks >= (double)kTickLimit) return fail(AC_ERR_ARG, "T too large (t_end must be < 2^61)");
  return ac_run_until_ticks(sim, (int64_t)ticks);
}

}  // extern "C"

namespace {
// Device staging for state transfers: the second state buffers (free between run calls)
// and a byte array for the spins.
ac_status ensure_staging(ac_sim* s) {
  const size_t N = s->ncells();
  if (!s->key2 && (cudaMalloc(&s->key2, N * 8) != cudaSuccess || cudaMalloc(&s->cnt2, N * 4) != cudaSuccess)) {
    cudaGetLastError();
    return fail(AC_ERR_OOM, "state staging allocation failed");
  }
  if (!s->stage8 && cudaMalloc(&s->stage8, N) != cudaSuccess) {
    cudaGetLastError();
    return fail(AC_ERR_OOM, "state staging allocation failed");
  }
  return AC_OK;
}
}  // namespace

extern "C" {

ac_status ac_read_state(const ac_sim* csim, int8_t* s, int64_t* t, uint32_t* n) {
  if (!csim) return fail(AC_ERR_ARG, "sim is NULL");
  ac_sim* sim = const_cast<ac_sim*>(csim);   // staging buffers only; the state is not modified
  const size_t N = sim->ncells();
  AC_SETTLE(sim);
  if (s || t) {
    ac_status st = ensure_staging(sim);
    if (st != AC_OK) return st;
    const ac::LatDesc d = sim->host_desc(sim->t_done, 0);
    AC_CUDA(ac::launch_unpack(&d, s ? sim->stage8 : nullptr, t ? (long long*)sim->key2 : nullptr, nullptr,
                              sim->stream));
    if (s) AC_CUDA(cudaMemcpyAsync(s, sim->stage8, N, cudaMemcpyDeviceToHost, sim->stream));
    if (t) AC_CUDA(cudaMemcpyAsync(t, sim->key2, N * 8, cudaMemcpyDeviceToHost, sim->stream));
  }
  if (n) AC_CUDA(cudaMemcpyAsync(n, sim->cnt, N * 4, cudaMemcpyDeviceToHost, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  return AC_OK;
}

ac_status ac_read_state_device(const ac_sim* sim, int8_t* s, int64_t* t, uint32_t* n) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(const_cast<ac_sim*>(sim));
  const ac::LatDesc d = sim->host_desc(sim->t_done, 0);
  AC_CUDA(ac::launch_unpack(&d, s, (long long*)t, n, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  return AC_OK;
}

ac_status ac_load_state(ac_sim* sim, const int8_t* s, const int64_t* t, const uint32_t* n,
                        int64_t t_done) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(sim);
  if (!s || !t || !n) return fail(AC_ERR_ARG, "s, t and n are required");
  if (t_done < 0 || t_done >= kTickLimit) return fail(AC_ERR_ARG, "t_done out of range");
  const size_t N = sim->ncells();
  ac_status st = ensure_staging(sim);
  if (st != AC_OK) return st;
  // copy into staging, validate on the device, and only then replace the state
  AC_CUDA(cudaMemcpyAsync(sim->stage8, s, N, cudaMemcpyHostToDevice, sim->stream));
  AC_CUDA(cudaMemcpyAsync(sim->key2, t, N * 8, cudaMemcpyHostToDevice, sim->stream));
  AC_CUDA(cudaMemcpyAsync(sim->cnt2, n, N * 4, cudaMemcpyHostToDevice, sim->stream));
  const long long tmin = std::max<long long>(t_done, 1);
  unsigned long long bad = ~0ull;
  AC_CUDA(cudaMemcpyAsync(sim->d_red, &bad, 8, cudaMemcpyHostToDevice, sim->stream));
  AC_CUDA(ac::launch_validate(sim->stage8, (const long long*)sim->key2, N, tmin, kTickLimit, sim->d_red,
                              sim->stream));
  AC_CUDA(cudaMemcpyAsync(&bad, sim->d_red, 8, cudaMemcpyDeviceToHost, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  if (bad != ~0ull)
    return fail(AC_ERR_ARG, "cell %llu: spin %d / tick %lld (spins must be +-1, ticks in [%lld, 2^61))",
                bad, (int)s[bad], (long long)t[bad], tmin);
  const ac::LatDesc d = sim->host_desc(t_done, 0);
  AC_CUDA(ac::launch_pack(&d, sim->stage8, (const long long*)sim->key2, sim->cnt2, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  sim->t_done = t_done;
  frames_off(sim);
  return AC_OK;
}

ac_status ac_load_state_async(ac_sim* sim, const int8_t* s, const int64_t* t, const uint32_t* n, int64_t t_done,
                              void* stream) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  if (!s || !t || !n) return fail(AC_ERR_ARG, "s, t and n are required");
  if (t_done < 0 || t_done >= kTickLimit) return fail(AC_ERR_ARG, "t_done out of range");
  AC_SETTLE(sim);
  ac_status st = ensure_staging(sim);
  if (st == AC_OK) st = ensure_async(sim);
  if (st != AC_OK) return st;
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const size_t N = sim->ncells();
  // the staging buffers are the handle's second state buffer: start after its earlier work
  AC_CUDA(cudaEventRecord(sim->ev_work, sim->stream));
  AC_CUDA(cudaStreamWaitEvent(cs, sim->ev_work, 0));
  AC_CUDA(cudaMemcpyAsync(sim->stage8, s, N, cudaMemcpyHostToDevice, cs));
  AC_CUDA(cudaMemcpyAsync(sim->key2, t, N * 8, cudaMemcpyHostToDevice, cs));
  AC_CUDA(cudaMemcpyAsync(sim->cnt2, n, N * 4, cudaMemcpyHostToDevice, cs));
  unsigned long long* d_bad = sim->d_red + 12;
  AC_CUDA(cudaMemsetAsync(d_bad, 0xFF, 8, cs));
  AC_CUDA(ac::launch_validate(sim->stage8, (const long long*)sim->key2, N, std::max<long long>(t_done, 1),
                              kTickLimit, d_bad, cs, kAsyncBlocks));
  AC_CUDA(cudaMemcpyAsync(sim->h_bad, d_bad, 8, cudaMemcpyDeviceToHost, cs));
  const ac::LatDesc d = sim->host_desc(t_done, 0);
  AC_CUDA(ac::launch_pack_checked(&d, sim->stage8, (const long long*)sim->key2, sim->cnt2, d_bad, cs, kAsyncBlocks));
  AC_CUDA(cudaEventRecord(sim->ev_load, cs));
  // no device-side wait on the handle's stream here: other handles may share that stream
  // and must not wait for this load; the handle's next call waits for it (settle_async)
  sim->load_pending = true;
  sim->load_t_done = t_done;
  return AC_OK;
}

ac_status ac_read_state_async(const ac_sim* csim, int8_t* s, int64_t* t, uint32_t* n, void* stream) {
  if (!csim) return fail(AC_ERR_ARG, "sim is NULL");
  ac_sim* sim = const_cast<ac_sim*>(csim);   // staging buffers and events only; the state is not modified
  AC_SETTLE(sim);
  ac_status st = ensure_staging(sim);
  if (st == AC_OK) st = ensure_async(sim);
  if (st != AC_OK) return st;
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const size_t N = sim->ncells();
  AC_CUDA(cudaEventRecord(sim->ev_work, sim->stream));
  AC_CUDA(cudaStreamWaitEvent(cs, sim->ev_work, 0));
  if (s || t) {
    const ac::LatDesc d = sim->host_desc(sim->t_done, 0);
    AC_CUDA(ac::launch_unpack(&d, s ? sim->stage8 : nullptr, t ? (long long*)sim->key2 : nullptr, nullptr, cs,
                              kAsyncBlocks));
    if (s) AC_CUDA(cudaMemcpyAsync(s, sim->stage8, N, cudaMemcpyDeviceToHost, cs));
    if (t) AC_CUDA(cudaMemcpyAsync(t, sim->key2, N * 8, cudaMemcpyDeviceToHost, cs));
  }
  if (n) AC_CUDA(cudaMemcpyAsync(n, sim->cnt, N * 4, cudaMemcpyDeviceToHost, cs));
  AC_CUDA(cudaEventRecord(sim->ev_read, cs));
  sim->read_pending = true;
  return AC_OK;
}

ac_status ac_stats(const ac_sim* sim, ac_stats_t* o) {
  if (!sim || !o) return fail(AC_ERR_ARG, "sim and out are required");
  AC_SETTLE(const_cast<ac_sim*>(sim));
  std::memset(o, 0, sizeof *o);
  unsigned long long r[4] = {0, 0, 0, 0};
  const ac::LatDesc d = sim->host_desc(sim->t_done, 0);
  AC_CUDA(cudaMemsetAsync(sim->d_red, 0, sizeof r, sim->stream));
  AC_CUDA(ac::launch_reduce(&d, sim->d_red, sim->stream));
  AC_CUDA(cudaMemcpyAsync(r, sim->d_red, sizeof r, cudaMemcpyDeviceToHost, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  o->events = sim->events;
  o->rounds = sim->rounds;
  o->launches = sim->launches;
  o->scanned = sim->scanned;
  o->enabled = sim->enabled;
  o->visits = sim->visits;
  o->polls = sim->polls;
  o->global_rounds = sim->global_rounds;
  o->device_ms = sim->device_ms;
  if (sim->global_rounds > 0)
    o->enabled_frac_mean = (double)sim->enabled_r1 / ((double)sim->global_rounds * (double)sim->ncells());
  else if (sim->scanned > 0)
    o->enabled_frac_mean = (double)sim->enabled / (double)sim->scanned;
  o->sum_s = (int64_t)r[0];
  o->sum_bonds = (int64_t)r[1];
  o->checksum = r[2];
  o->total_counts = r[3];
  o->t_done = sim->t_done;
  o->kernel = sim->cfg.kernel;
  o->Lb = sim->cfg.lb;
  o->threads = sim->cfg.threads;
  o->rounds_per_launch = sim->cfg.kernel != ac::kKernelBlocked ? sim->cfg.rounds : sim->cfg.refresh;
  o->grid = sim->last_grid;
  o->ctas_per_sm = sim->ctas_per_sm;
  o->early_commits = sim->early;
  return AC_OK;
}

ac_status ac_round_history(const ac_sim* sim, uint64_t* counts, int32_t cap, int32_t* n_rounds) {
  if (!sim || !n_rounds) return fail(AC_ERR_ARG, "sim and n_rounds are required");
  const int avail = (int)std::min<unsigned long long>(sim->global_rounds, (unsigned long long)sim->hist_cap);
  *n_rounds = avail;
  if (counts && cap > 0 && avail > 0 && sim->d_hist) {
    const int m = std::min(avail, cap);
    AC_CUDA(cudaMemcpyAsync(counts, sim->d_hist, (size_t)m * 8, cudaMemcpyDeviceToHost, sim->stream));
    AC_CUDA(cudaStreamSynchronize(sim->stream));
  }
  return AC_OK;
}

ac_status ac_class_counts(const ac_sim* sim, uint64_t counts[10]) {
  if (!sim || !counts) return fail(AC_ERR_ARG, "sim and counts are required");
  AC_SETTLE(const_cast<ac_sim*>(sim));
  if (sim->model != 0) return fail(AC_ERR_ARG, "classes are defined for the 4-neighbour Ising array");
  const ac::LatDesc d = sim->host_desc(sim->t_done, 0);
  AC_CUDA(cudaMemsetAsync(sim->d_red, 0, 10 * sizeof(unsigned long long), sim->stream));
  AC_CUDA(ac::launch_class_counts(&d, sim->d_red, sim->stream));
  AC_CUDA(cudaMemcpyAsync(counts, sim->d_red, 10 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  return AC_OK;
}

ac_status ac_reset(ac_sim* sim, uint64_t seed, int32_t init) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  AC_SETTLE(sim);
  if (init < AC_INIT_RANDOM || init > AC_INIT_DOWN) return fail(AC_ERR_ARG, "bad init mode");
  sim->seed = seed;
  sim->init = init;
  const ac::LatDesc d = sim->host_desc(0, 0);
  AC_CUDA(ac::launch_init(&d, init, sim->stream));
  AC_CUDA(cudaMemsetAsync(sim->d_events, 0, 8, sim->stream));
  if (sim->d_hist) AC_CUDA(cudaMemsetAsync(sim->d_hist, 0, (size_t)sim->hist_cap * 8, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  sim->t_done = 0;
  frames_off(sim);
  sim->events = sim->rounds = sim->launches = sim->scanned = sim->enabled = sim->visits = sim->polls = 0;
  sim->global_rounds = sim->enabled_r1 = sim->early = 0;
  sim->device_ms = 0.0;
  drop_runners_of(sim);
  return AC_OK;
}

ac_status ac_set_option(ac_sim* sim, int32_t option, int64_t value) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  switch (option) {
    case AC_OPT_WATCHDOG_NS:
      if (value < 1000000) return fail(AC_ERR_ARG, "watchdog must be >= 1e6 ns");
      sim->cfg.watchdog_ns = value;
      break;
    case AC_OPT_MAX_ROUNDS:
      if (value < 0 || value > (1 << 30)) return fail(AC_ERR_ARG, "max rounds out of range");
      sim->cfg.max_rounds = (int)value;
      break;
    case AC_OPT_DROP_PUBLISH:
      sim->drop_publish = value ? 1 : 0;
      break;
    case AC_OPT_EARLY_REJECT:
      if (value && sim->model != 0) return fail(AC_ERR_ARG, "early rejection applies to the Ising array");
      sim->early_reject = value != 0;
      break;
    default:
      return fail(AC_ERR_ARG, "unknown option %d", option);
  }
  drop_runners_of(sim);
  return AC_OK;
}

void ac_destroy(ac_sim* sim) {
  if (!sim) return;
  drop_runners_of(sim);
  cudaStreamSynchronize(sim->stream);
  free_sim(sim);
}

ac_status ac_batch_create(int32_t n, const ac_lattice* lats, const double* beta, const double* J,
                          const double* h, const uint64_t* seed, ac_sim** out) {
  if (n <= 0 || !lats || !beta || !J || !h || !seed || !out)
    return fail(AC_ERR_ARG, "n > 0 and all arrays are required");
  for (int i = 0; i < n; ++i) {
    ac_status st = check_params(lats[i], beta[i], J[i], h[i]);
    if (st != AC_OK) return fail(st, "lattice %d: %s", i, g_err.c_str());
  }
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  for (int i = 0; i < n; ++i) {
    ac_status st = create_one(lats[i], beta[i], J[i], h[i], seed[i], &out[i]);
    if (st != AC_OK) {
      for (int k = 0; k < i; ++k) {
        free_sim(out[k]);
        out[k] = nullptr;
      }
      return st;
    }
  }
  return AC_OK;
}

ac_status ac_batch_run_until(int32_t n, ac_sim* const* sims, const int64_t* t_end) {
  if (n <= 0 || !sims || !t_end) return fail(AC_ERR_ARG, "n > 0, sims and t_end are required");
  for (int i = 0; i < n; ++i) {
    if (!sims[i]) return fail(AC_ERR_ARG, "sims[%d] is NULL", i);
    AC_SETTLE(sims[i]);
    if (sims[i]->f_B > 0) return fail(AC_ERR_ARG, "sims[%d] has snapshot frames: run it with ac_run_until_frames", i);
    if (sims[i]->model != 0) return fail(AC_ERR_ARG, "sims[%d] is not the 4-neighbour Ising array: batches hold those only", i);
    if (sims[i]->cfg.lb != sims[0]->cfg.lb) return fail(AC_ERR_ARG, "all handles must share a tile side");
    if (sims[i]->stream != sims[0]->stream) return fail(AC_ERR_ARG, "all handles must share a stream");
    if (t_end[i] < sims[i]->t_done) return fail(AC_ERR_ARG, "t_end[%d] is below its previous t_end", i);
    if (t_end[i] >= kTickLimit) return fail(AC_ERR_ARG, "t_end[%d] must be < 2^61", i);
    for (int k = 0; k < i; ++k)
      if (sims[k] == sims[i]) return fail(AC_ERR_ARG, "handle %d appears twice", i);
  }
  std::vector<ac_sim*> keyv(sims, sims + n);
  bool want_ep = true;
  for (int i = 0; i < n; ++i)
    want_ep = want_ep && sims[i]->cfg.kernel == ac::kKernelEpoch && sims[i]->cfg.rounds == sims[0]->cfg.rounds &&
              ep_applicable(sims[i]);
  // epoch-kernel handles that cannot run on it run on the temporal-blocked round kernel
  bool want_tb = !want_ep;
  for (int i = 0; i < n; ++i)
    want_tb = want_tb && sims[i]->cfg.kernel != ac::kKernelBlocked && sims[i]->cfg.rounds == sims[0]->cfg.rounds &&
              tb_applicable(sims[i]);
  BatchRunner* R = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_runners.find(keyv);
    if (it != g_runners.end()) {
      if (it->second->tb != want_tb || it->second->ep != want_ep) {
        free_runner(it->second);
        g_runners.erase(it);
      } else {
        R = it->second;
      }
    }
  }
  if (want_tb || want_ep) {
    if (!R) {
      R = new BatchRunner();
      R->sims = keyv;
      R->tb = want_tb;
      R->ep = want_ep;
      R->halo = sims[0]->cfg.rounds;
      R->region = ac::tb_region_for(R->halo, sims[0]->cfg.lb == 128);
      R->lb = sims[0]->cfg.lb;
      if (sims[0]->stream == nullptr) {
        if (cudaStreamCreate(&R->own_stream) != cudaSuccess) {
          free_runner(R);
          return fail(AC_ERR_CUDA, "cudaStreamCreate failed");
        }
        R->stream = R->own_stream;
      } else {
        R->stream = sims[0]->stream;
      }
      if (cudaHostAlloc(&R->h_desc, sizeof(ac::LatDesc) * n, cudaHostAllocDefault) != cudaSuccess ||
          cudaMalloc(&R->d_desc, sizeof(ac::LatDesc) * n) != cudaSuccess ||
          cudaMalloc(&R->d_ctr, sizeof(ac::DevCounters)) != cudaSuccess ||
          cudaMalloc(&R->d_range, sizeof(unsigned) * 2 * n) != cudaSuccess ||
          cudaEventCreate(&R->ev0) != cudaSuccess || cudaEventCreate(&R->ev1) != cudaSuccess) {
        cudaGetLastError();
        free_runner(R);
        return fail(AC_ERR_OOM, "batch runner allocation failed");
      }
      std::lock_guard<std::mutex> lk(g_batch_mu);
      g_runners[keyv] = R;
    }
    return want_ep ? batch_run_ep(n, sims, t_end, R) : batch_run_tb(n, sims, t_end, R);
  }
  if (!R) {
    R = new BatchRunner();
    R->sims = keyv;
    R->lb = sims[0]->cfg.lb;
    // graph capture needs a capturable stream: the legacy default stream is not one,
    // so such handles get a blocking stream of the runner (ordered with the legacy stream)
    if (sims[0]->stream == nullptr) {
      if (cudaStreamCreate(&R->own_stream) != cudaSuccess) {
        free_runner(R);
        return fail(AC_ERR_CUDA, "cudaStreamCreate failed");
      }
      R->stream = R->own_stream;
    } else {
      R->stream = sims[0]->stream;
    }
    const cudaStream_t stream = R->stream;
    R->cfg = sims[0]->cfg;
    R->cfg.kernel = ac::kKernelBlocked;
    int per_sm = 0;
    const int maxc = ac::blocked_max_ctas(R->lb, &per_sm);
    int total = 0;
    for (int i = 0; i < n; ++i) total += sims[i]->tiles();
    R->total_tiles = total;
    R->grid = std::min(total, maxc);
    if (maxc <= 0 || cudaHostAlloc(&R->h_desc, sizeof(ac::LatDesc) * n, cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc(&R->d_desc, sizeof(ac::LatDesc) * n) != cudaSuccess ||
        cudaMalloc(&R->d_ctr, sizeof(ac::DevCounters)) != cudaSuccess ||
        cudaMalloc(&R->d_tile_done, (size_t)total * 4) != cudaSuccess ||
        cudaEventCreate(&R->ev0) != cudaSuccess || cudaEventCreate(&R->ev1) != cudaSuccess) {
      cudaGetLastError();
      free_runner(R);
      return fail(AC_ERR_OOM, "batch runner allocation failed");
    }
    int base = 0;
    for (int i = 0; i < n; ++i) {
      R->h_desc[i] = sims[i]->host_desc(t_end[i], base);
      base += sims[i]->tiles();
    }
    cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R->d_desc, R->h_desc, sizeof(ac::LatDesc) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(R->d_ctr, 0, sizeof(ac::DevCounters), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(R->d_tile_done, 0, (size_t)total * 4, stream);
    if (e == cudaSuccess) e = ac::launch_publish(R->d_desc, n, total, R->lb, 0, stream);
    if (e == cudaSuccess) e = ac::launch_blocked(R->d_desc, n, total, R->cfg, R->grid, R->d_tile_done, R->d_ctr, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(stream, &g);
    if (e == cudaSuccess) e = e2;
    R->graph = g;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&R->exec, g, 0);
    if (e != cudaSuccess) {
      free_runner(R);
      return fail(AC_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_runners[keyv] = R;
  }
  const cudaStream_t stream = R->stream;
  // per-lattice event counters before the launch
  std::vector<unsigned long long> before(n), after(n);
  for (int i = 0; i < n; ++i)
    AC_CUDA(cudaMemcpyAsync(&before[i], sims[i]->d_events, 8, cudaMemcpyDeviceToHost, stream));
  AC_CUDA(cudaStreamSynchronize(stream));
  int base = 0;
  for (int i = 0; i < n; ++i) {
    R->h_desc[i] = sims[i]->host_desc(t_end[i], base);
    base += sims[i]->tiles();
  }
  // the timed interval covers the whole graph: descriptor copy, flag resets, the edge-word
  // publish kernel (a few microseconds) and the blocked kernel
  AC_CUDA(cudaEventRecord(R->ev0, stream));
  AC_CUDA(cudaGraphLaunch(R->exec, stream));
  AC_CUDA(cudaEventRecord(R->ev1, stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, R->d_ctr, sizeof c, cudaMemcpyDeviceToHost, stream));
  for (int i = 0; i < n; ++i)
    AC_CUDA(cudaMemcpyAsync(&after[i], sims[i]->d_events, 8, cudaMemcpyDeviceToHost, stream));
  AC_CUDA(cudaStreamSynchronize(stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, R->ev0, R->ev1));
  if (c.error) return fail((ac_status)c.error, "device watchdog: no progress (block %d)", c.err_block);
  for (int i = 0; i < n; ++i) {
    ac_sim* s = sims[i];
    s->events += after[i] - before[i];
    s->t_done = t_end[i];
    s->launches += 1;
    s->device_ms += ms;
    s->last_grid = R->grid;
  }
  // aggregate counters are attributed to the first handle
  sims[0]->rounds += c.rounds;
  sims[0]->scanned += c.scanned;
  sims[0]->enabled += c.enabled;
  sims[0]->visits += c.visits;
  sims[0]->polls += c.polls;
  return check_bounds();
}

ac_status ac_slab_configure(ac_sim* sim, int32_t row0, int32_t nrows) {
  if (!sim) return fail(AC_ERR_ARG, "sim is NULL");
  if (nrows == 0) {
    sim->slab_row0 = sim->slab_rows = 0;
    return AC_OK;
  }
  const int R = sim->cfg.rounds;
  if (sim->model != 0 || sim->cfg.kernel == ac::kKernelBlocked || R < 2 || !tb_applicable(sim))
    return fail(AC_ERR_ARG, "row slabs run on the temporal-blocked round kernel (round or epoch kernel, rounds >= 2, "
                            "rows and cols >= 4 * rounds, the 4-neighbour Ising array)");
  if (row0 < 0 || row0 >= sim->rows || nrows < R || nrows > sim->rows - 2 * R)
    return fail(AC_ERR_ARG, "slab rows [%d, %d + %d) must lie in the torus with rounds <= nrows <= rows - 2 * rounds",
                row0, row0, nrows);
  if (sim->f_B > 0) return fail(AC_ERR_ARG, "snapshot frames are not taken on row slabs");
  sim->slab_row0 = row0;
  sim->slab_rows = nrows;
  return AC_OK;
}

ac_status ac_slab_step(ac_sim* sim, int64_t t_end, int32_t* live) {
  if (!sim || !live) return fail(AC_ERR_ARG, "sim and live are required");
  if (sim->slab_rows == 0) return fail(AC_ERR_STATE, "no slab configured (ac_slab_configure)");
  if (t_end < 0 || t_end >= kTickLimit) return fail(AC_ERR_ARG, "t_end must be in [0, 2^61)");
  AC_SETTLE(sim);
  const size_t N = sim->ncells();
  if (!sim->key2) {
    if (cudaMalloc(&sim->key2, N * 8) != cudaSuccess || cudaMalloc(&sim->cnt2, N * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(AC_ERR_OOM, "second state buffer (%zu cells) allocation failed", N);
    }
  }
  const int R = sim->cfg.rounds;
  const int region = ac::tb_region_for(R, sim->cfg.lb == 128);
  int tr = 0, tc = 0;
  tb_tiling(sim->slab_rows, sim->cols, region, R, ac::tb_grid(region), &tr, &tc);
  tr = std::min(tr, std::max(1, sim->slab_rows / R));   // tile heights >= R: the halo lies in the neighbour slabs
  ac::LatDesc d = sim->host_desc(t_end, 0);
  d.tr = tr;
  d.tc = tc;
  d.srow0 = sim->slab_row0;
  d.srows = sim->slab_rows;
  AC_CUDA(cudaMemcpyAsync(sim->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, sim->stream));
  AC_CUDA(cudaMemsetAsync(sim->d_ctr, 0, sizeof(ac::DevCounters), sim->stream));
  AC_CUDA(cudaEventRecord(sim->ev0, sim->stream));
  AC_CUDA(ac::launch_tb(sim->d_desc, 1, tr * tc, region, R, R, sim->d_ctr, sim->stream, false, 0, sim->d_rates != nullptr));
  AC_CUDA(cudaEventRecord(sim->ev1, sim->stream));
  ac::DevCounters c{};
  AC_CUDA(cudaMemcpyAsync(&c, sim->d_ctr, sizeof c, cudaMemcpyDeviceToHost, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  float ms = 0.f;
  AC_CUDA(cudaEventElapsedTime(&ms, sim->ev0, sim->ev1));
  if (c.error) return fail(c.error == AC_ERR_STATE ? AC_ERR_STATE : AC_ERR_CUDA,
                           "slab step: device error %d (counts left the 16-bit window: the state is unchanged)", c.error);
  // the launch wrote the slab's tiles into the second buffer: it becomes the current state, whose
  // rows outside the slab the caller refreshes (ac_slab_import) before the next step
  std::swap(sim->key, sim->key2);
  std::swap(sim->cnt, sim->cnt2);
  sim->events += c.events;
  *live = c.active[0] > 0 ? 1 : 0;
  sim->last_grid = std::min(tr * tc, ac::tb_grid(region));
  return accumulate(sim, c, ms, true);
}

ac_status ac_slab_export(const ac_sim* csim, int32_t row, int32_t count, void* dst_dev) {
  if (!csim || (!dst_dev && count > 0)) return fail(AC_ERR_ARG, "sim and dst are required");
  if (row < 0 || count < 0 || row + count > csim->rows) return fail(AC_ERR_ARG, "rows [%d, %d) out of range", row, row + count);
  ac_sim* sim = const_cast<ac_sim*>(csim);
  AC_SETTLE(sim);
  const size_t n = (size_t)count * sim->cols, off = (size_t)row * sim->cols;
  unsigned char* dst = static_cast<unsigned char*>(dst_dev);
  AC_CUDA(cudaMemcpyAsync(dst, sim->key + off, n * 8, cudaMemcpyDeviceToDevice, sim->stream));
  AC_CUDA(cudaMemcpyAsync(dst + n * 8, sim->cnt + off, n * 4, cudaMemcpyDeviceToDevice, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  return AC_OK;
}

ac_status ac_slab_import(ac_sim* sim, int32_t row, int32_t count, const void* src_dev) {
  if (!sim || (!src_dev && count > 0)) return fail(AC_ERR_ARG, "sim and src are required");
  if (row < 0 || count < 0 || row + count > sim->rows) return fail(AC_ERR_ARG, "rows [%d, %d) out of range", row, row + count);
  AC_SETTLE(sim);
  const size_t n = (size_t)count * sim->cols, off = (size_t)row * sim->cols;
  const unsigned char* src = static_cast<const unsigned char*>(src_dev);
  AC_CUDA(cudaMemcpyAsync(sim->key + off, src, n * 8, cudaMemcpyDeviceToDevice, sim->stream));
  AC_CUDA(cudaMemcpyAsync(sim->cnt + off, src + n * 8, n * 4, cudaMemcpyDeviceToDevice, sim->stream));
  AC_CUDA(cudaStreamSynchronize(sim->stream));
  return AC_OK;
}

ac_status ac_dev_exp_ticks(const uint32_t* x, uint64_t* out, int64_t n) {
  if (n < 0 || (n > 0 && (!x || !out))) return fail(AC_ERR_ARG, "bad arguments");
  AC_CUDA(ac::launch_exp_ticks(x, (unsigned long long*)out, n, nullptr));
  AC_CUDA(cudaStreamSynchronize(nullptr));
  return AC_OK;
}

ac_status ac_dev_philox(uint64_t seed, const uint32_t* c, const uint32_t* k, uint32_t w2, uint32_t* out4,
                        int64_t n) {
  if (n < 0 || (n > 0 && (!c || !k || !out4))) return fail(AC_ERR_ARG, "bad arguments");
  AC_CUDA(ac::launch_philox(seed, c, k, w2, out4, n, nullptr));
  AC_CUDA(cudaStreamSynchronize(nullptr));
  return AC_OK;
}

}  // extern "C"
