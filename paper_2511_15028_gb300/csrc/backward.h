// Backward-pass kernel interface (see backward.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace scion {

struct BackwardArgs {
  const float *rays;       // scion_ray[n]
  const uint32_t *hits;    // scion_hit[n]
  const float *grad_tuv;   // float[n][3]
  const float4 *verts;     // BVH vertex table (float4)
  const uint32_t *tri_idx; // u32[3] per triangle or null (soup)
  float *grad_verts;       // float[n_verts][3], accumulated
  float *grad_rays;        // float[n][8] (scion_ray layout) or null
  unsigned long long n;
  uint32_t n_tris;
};

cudaError_t launch_backward(const BackwardArgs &a, int sms, cudaStream_t s);

}  // namespace scion
