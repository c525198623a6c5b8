// Test-only reference: cuRAND's Philox4x32-10 device function, called (not
// reimplemented) so that the library's and the oracle's Philox can be checked
// against NVIDIA's.  Built by the GPU tests into a temporary directory.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void ref_kernel(unsigned long long seed, const uint32_t* c, const uint32_t* k, uint32_t w2,
                           uint32_t* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 ctr = make_uint4(c[i], k[i], w2, 0u);
  uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  uint4 r = curand_Philox4x32_10(ctr, key);
  out[4 * i + 0] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

extern "C" int curand_ref_philox(unsigned long long seed, const uint32_t* c, const uint32_t* k, uint32_t w2,
                                 uint32_t* out, long long n) {
  if (n <= 0) return 0;
  ref_kernel<<<(unsigned)((n + 255) / 256), 256>>>(seed, c, k, w2, out, n);
  cudaError_t e = cudaDeviceSynchronize();
  return (int)e;
}
