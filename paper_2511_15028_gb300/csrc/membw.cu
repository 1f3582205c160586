// Read-bandwidth probe for the roofline of traversals whose BVH fits in L2.
//
// A traversal of a BVH smaller than L2 fetches its nodes from L2 (and L1),
// not from HBM, so its bandwidth roof is the rate at which the SMs can read
// from L2. This kernel measures that rate: every thread streams 16-byte loads
// that bypass L1 (ld.global.cg) over a buffer which stays resident in L2, a
// configurable number of times in one launch; the caller times the launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/scion.h"
#include "../../include/scion_debug.h"

namespace {

constexpr int kThreads = 512;
constexpr int kUnroll = 4;  // independent loads in flight per thread

__device__ __forceinline__ uint4 ld_cg(const uint4 *p) {
  uint4 v;
  asm("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}

// reps passes over n16 16-byte words; pass r starts at a different CTA offset
// so that an SM does not read the same lines in consecutive passes.
__global__ void __launch_bounds__(kThreads) read_kernel(const uint4 *__restrict__ buf, unsigned long long n16,
                                                        uint32_t reps, uint32_t *sink) {
  uint32_t acc = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (uint32_t r = 0; r < reps; ++r) {
    const unsigned long long cta = (blockIdx.x + (unsigned long long)r * 37u) % gridDim.x;
    unsigned long long i = cta * blockDim.x + threadIdx.x;
    for (; i + (kUnroll - 1) * stride < n16; i += kUnroll * stride) {
      uint4 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) v[u] = ld_cg(buf + i + u * stride);
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    for (; i < n16; i += stride) {
      const uint4 v = ld_cg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  // the loads must not be optimised away: their xor goes to memory when it
  // has one (arbitrary) value, which the caller never relies on
  if (acc == 0x9E3779B9u) *sink = acc;
}

}  // namespace

extern "C" scion_status scion_debug_read_bandwidth(const void *d_buf, uint64_t bytes, uint32_t reps,
                                                   uint32_t *d_sink, scion_stream stream) {
  if (!d_buf || !d_sink || bytes < 16 || (bytes & 15u) || reps == 0 ||
      (reinterpret_cast<uintptr_t>(d_buf) & 15u) || (reinterpret_cast<uintptr_t>(d_sink) & 3u))
    return SCION_ERR_INVALID_ARG;
  cudaPointerAttributes at;
  cudaPointerAttributes as;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, d_buf) != cudaSuccess ||
      cudaPointerGetAttributes(&as, d_sink) != cudaSuccess) {
    cudaGetLastError();
    return SCION_ERR_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeDevice || as.type != cudaMemoryTypeDevice || at.device != dev || as.device != dev)
    return SCION_ERR_INVALID_ARG;
  int sms = 0, nb = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, read_kernel, kThreads, 0) != cudaSuccess)
    return SCION_ERR_CUDA;
  const unsigned long long n16 = bytes / 16;
  const unsigned grid = (unsigned)std::max(1, sms * std::max(nb, 1));
  read_kernel<<<grid, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(static_cast<const uint4 *>(d_buf),
                                                                           n16, reps, d_sink);
  return cudaGetLastError() == cudaSuccess ? SCION_OK : SCION_ERR_CUDA;
}
