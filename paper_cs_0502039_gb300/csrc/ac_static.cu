// ac_static.cu -- a run entry point that allocates no memory.
//
// Some callers cannot let a library call cudaMalloc: applications whose own memory
// pool reserved the device's memory up front, hosts that give a plugin a fixed
// device budget and nothing else, and loops that must not call cudaMalloc or
// cudaFree because those calls can synchronise the device.  For them
// ac_run_blocked_static() advances a lattice held in the caller's own device
// buffers with the blocked persistent kernel, and keeps every other buffer the
// kernel needs (lattice descriptor, counters, tile flags, edge words) in one
// file-scope device array of fixed size, reserved when the library is loaded.
// The array's device address is looked up once per device and cached for the
// process; the cache does not survive cudaDeviceReset.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ac.h"
#include "ac_internal.h"

namespace {

constexpr int kStaticLb = 64;                                   // tile side of this entry point
constexpr size_t kStaticScratchBytes = AC_STATIC_SCRATCH_BYTES;  // 4 MiB, see include/ac.h

// Shared by every call on a device and kept by every GPU that loads the library
// until the process exits.  Host code may not use this name as an address (it is
// a host-side stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

ac_status fail_static(ac_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  ac::set_last_error(buf);
  return st;
}

#define AC_STATIC_CUDA(call)                                                                  \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail_static(AC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)

}  // namespace

extern "C" ac_status ac_run_blocked_static(int32_t rows, int32_t cols, double beta, double J, double h,
                                           uint64_t seed, uint64_t* key_dev, uint32_t* cnt_dev,
                                           int64_t t_end, void* stream) {
  if (rows < 2 || cols < 2 || (unsigned long long)rows * (unsigned long long)cols >= (1ull << 32))
    return fail_static(AC_ERR_ARG, "rows, cols must be >= 2 with rows * cols < 2^32");
  if (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(J) || !std::isfinite(h))
    return fail_static(AC_ERR_ARG, "beta must be finite and >= 0; J, h finite");
  if (!key_dev || !cnt_dev) return fail_static(AC_ERR_ARG, "key_dev and cnt_dev are required");
  if (t_end < 0 || t_end >= (1ll << 61)) return fail_static(AC_ERR_ARG, "t_end must be in [0, 2^61)");

  const int tr = (rows + kStaticLb - 1) / kStaticLb, tc = (cols + kStaticLb - 1) / kStaticLb;
  const size_t tiles = (size_t)tr * tc;
  const size_t off_ctr = align256(sizeof(ac::LatDesc));
  const size_t off_ev = off_ctr + align256(sizeof(ac::DevCounters));
  const size_t off_done = off_ev + 256;
  const size_t off_pub = off_done + align256(tiles * 4);
  const size_t need = off_pub + tiles * 4 * kStaticLb * 8;
  if (need > kStaticScratchBytes)
    return fail_static(AC_ERR_ARG,
                       "lattice %d x %d needs %zu bytes of static scratch (%zu tiles of %d x %d); "
                       "the maximum is %zu bytes (about %zu tiles)",
                       rows, cols, need, tiles, kStaticLb, kStaticLb, kStaticScratchBytes,
                       (kStaticScratchBytes - off_done) / (4 + 4 * kStaticLb * 8));

  int dev = 0;
  AC_STATIC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail_static(AC_ERR_ARG, "device index %d unsupported", dev);
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);   // with `dev` current
      if (e != cudaSuccess || p == nullptr)
        return fail_static(AC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                           cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ac::LatDesc* d_desc = reinterpret_cast<ac::LatDesc*>(base);
  ac::DevCounters* d_ctr = reinterpret_cast<ac::DevCounters*>(base + off_ctr);
  unsigned long long* d_ev = reinterpret_cast<unsigned long long*>(base + off_ev);
  unsigned int* d_done = reinterpret_cast<unsigned int*>(base + off_done);
  unsigned long long* d_pub = reinterpret_cast<unsigned long long*>(base + off_pub);

  ac::LatDesc d{};
  d.key = reinterpret_cast<unsigned long long*>(key_dev);
  d.cnt = cnt_dev;
  d.pub = d_pub;
  d.pub2 = d_pub;
  d.events = d_ev;
  d.rows = rows;
  d.cols = cols;
  d.tr = tr;
  d.tc = tc;
  d.lb = kStaticLb;
  d.tile_base = 0;
  ac::make_thresholds(beta, J, h, d.thr);
  d.seed_lo = (unsigned)(seed & 0xffffffffu);
  d.seed_hi = (unsigned)(seed >> 32);
  d.t_end = t_end;
  d.t2 = 2ull * (unsigned long long)t_end;
  d.two = 2u;

  ac::LaunchCfg cfg{};
  cfg.kernel = ac::kKernelBlocked;
  cfg.lb = kStaticLb;
  cfg.threads = 4 * kStaticLb;
  cfg.rounds = 1;
  cfg.polls = 8;
  cfg.refresh = 1;
  cfg.max_rounds = 0;
  cfg.watchdog_ns = 5ll * 1000 * 1000 * 1000;
  int per_sm = 0;
  const int maxc = ac::blocked_max_ctas(kStaticLb, &per_sm);
  if (maxc <= 0) return fail_static(AC_ERR_CUDA, "blocked kernel cannot be resident");
  const int grid = (int)std::min<size_t>(tiles, (size_t)maxc);

  // everything the previous call left in the scratch that must start at zero is cleared here
  AC_STATIC_CUDA(cudaMemcpyAsync(d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s));
  AC_STATIC_CUDA(cudaMemsetAsync(d_ctr, 0, sizeof(ac::DevCounters), s));
  AC_STATIC_CUDA(cudaMemsetAsync(d_ev, 0, 8, s));
  AC_STATIC_CUDA(cudaMemsetAsync(d_done, 0, tiles * 4, s));
  AC_STATIC_CUDA(ac::launch_publish(d_desc, 1, (int)tiles, kStaticLb, 0, s));
  AC_STATIC_CUDA(ac::launch_blocked(d_desc, 1, (int)tiles, cfg, grid, d_done, d_ctr, s));
  ac::DevCounters c{};
  AC_STATIC_CUDA(cudaMemcpyAsync(&c, d_ctr, sizeof c, cudaMemcpyDeviceToHost, s));
  AC_STATIC_CUDA(cudaStreamSynchronize(s));
  if (c.error) return fail_static(AC_ERR_STALL, "device watchdog: no progress (block %d)", c.err_block);
  return AC_OK;
}
