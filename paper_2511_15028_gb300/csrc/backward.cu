// Backward pass of the closest-hit query: with the traversal's discrete choice
// (which triangle each ray hit) held fixed, carry dL/d(t, u, v) of every hit
// ray to the hit triangle's three vertices and to the ray's origin and
// direction. The paper has no gradient; this follows from differentiating the
// hit-point identity o + t d = (1-u-v) p0 + u p1 + v p2 (the barycentric
// convention b1 = u, b2 = v of the closest-hit listing in App. G).
//
// With J = [d | -(p1-p0) | -(p2-p0)] and g = (dL/dt, dL/du, dL/dv), lambda
// solves J^T lambda = g; then dL/do = -lambda, dL/dd = -t lambda,
// dL/dp0 = (1-u-v) lambda, dL/dp1 = u lambda, dL/dp2 = v lambda.
//
// One thread per ray (grid-stride). The 3x3 solve runs in double precision
// (a few dozen FP64 operations per ray, well conditioned even for grazing
// hits); the nine vertex contributions are scattered with FP32 atomicAdd.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/scion.h"
#include "backward.h"

namespace scion {

namespace {

__device__ __forceinline__ void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__global__ void __launch_bounds__(256) backward_kernel(BackwardArgs a) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const uint4 h = __ldg(reinterpret_cast<const uint4 *>(a.hits) + i);
    const uint32_t prim = h.w;
    float4 *gr = a.grad_rays ? reinterpret_cast<float4 *>(a.grad_rays) + 2 * i : nullptr;
    if (prim >= a.n_tris) {
      if (gr) {
        gr[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        gr[1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    uint32_t vid[3];
    if (a.tri_idx) {
      vid[0] = __ldg(a.tri_idx + 3 * (size_t)prim);
      vid[1] = __ldg(a.tri_idx + 3 * (size_t)prim + 1);
      vid[2] = __ldg(a.tri_idx + 3 * (size_t)prim + 2);
    } else {
      vid[0] = 3 * prim;
      vid[1] = 3 * prim + 1;
      vid[2] = 3 * prim + 2;
    }
    const float4 p0 = __ldg(a.verts + vid[0]), p1 = __ldg(a.verts + vid[1]), p2 = __ldg(a.verts + vid[2]);
    const float4 rd = __ldg(reinterpret_cast<const float4 *>(a.rays) + 2 * i + 1);
    const double c0[3] = {rd.x, rd.y, rd.z};
    const double c1[3] = {-((double)p1.x - p0.x), -((double)p1.y - p0.y), -((double)p1.z - p0.z)};
    const double c2[3] = {-((double)p2.x - p0.x), -((double)p2.y - p0.y), -((double)p2.z - p0.z)};
    double x12[3], x20[3], x01[3];
    cross3(c1, c2, x12);
    cross3(c2, c0, x20);
    cross3(c0, c1, x01);
    const double det = dot3(c0, x12);
    if (det == 0.0) {
      if (gr) {
        gr[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        gr[1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    const double gt = a.grad_tuv[3 * i], gu = a.grad_tuv[3 * i + 1], gv = a.grad_tuv[3 * i + 2];
    double lam[3];
    for (int k = 0; k < 3; ++k) lam[k] = (gt * x12[k] + gu * x20[k] + gv * x01[k]) / det;
    const double t = __uint_as_float(h.x), u = __uint_as_float(h.y), v = __uint_as_float(h.z);
    const double w[3] = {1.0 - u - v, u, v};
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) atomicAdd(a.grad_verts + 3 * (size_t)vid[j] + k, (float)(w[j] * lam[k]));
    if (gr) {
      gr[0] = make_float4((float)-lam[0], (float)-lam[1], (float)-lam[2], 0.f);
      gr[1] = make_float4((float)(-t * lam[0]), (float)(-t * lam[1]), (float)(-t * lam[2]), 0.f);
    }
  }
}

}  // namespace

cudaError_t launch_backward(const BackwardArgs &a, int sms, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const unsigned long long blocks = (a.n + 255) / 256;
  const unsigned grid = (unsigned)(blocks < (unsigned long long)sms * 8 ? blocks : (unsigned long long)sms * 8);
  backward_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace scion
