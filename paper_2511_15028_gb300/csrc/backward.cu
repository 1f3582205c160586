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
// One thread per ray (grid-stride). The 3x3 solve runs in single precision
// (Cramer's rule) followed by one step of iterative refinement whose residual
// g - J^T lambda is formed in double precision from the exact columns of J;
// the error after the step is of the order of the square of the first
// solve's, so lambda comes out accurate to double-precision-solve level for
// any system that is not extremely ill conditioned, with about 20 FP64
// operations per ray instead of a hundred (FP64 is slow on this part). A
// singular or non-finite single-precision solve falls back to the
// double-precision solve. The nine vertex contributions are scattered with
// FP32 atomicAdd.
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

__device__ __forceinline__ void cross3f(const float *a, const float *b, float *c) {
  c[0] = fmaf(a[1], b[2], -a[2] * b[1]);
  c[1] = fmaf(a[2], b[0], -a[0] * b[2]);
  c[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

// lambda with J^T lambda = (gt, gu, gv), J = [c0 | c1 | c2]: single-precision
// Cramer's rule, then one refinement step lambda += J^-T (g - J^T lambda)
// with the residual in double precision. False when the single-precision
// system is singular or the result is not finite.
__device__ __forceinline__ bool solve_refined(const double *c0, const double *c1, const double *c2, float gt,
                                              float gu, float gv, double *lam) {
  const float f0[3] = {(float)c0[0], (float)c0[1], (float)c0[2]};
  const float f1[3] = {(float)c1[0], (float)c1[1], (float)c1[2]};
  const float f2[3] = {(float)c2[0], (float)c2[1], (float)c2[2]};
  float x12[3], x20[3], x01[3];
  cross3f(f1, f2, x12);
  cross3f(f2, f0, x20);
  cross3f(f0, f1, x01);
  const float det = fmaf(f0[0], x12[0], fmaf(f0[1], x12[1], f0[2] * x12[2]));
  if (!(det != 0.0f) || !isfinite(det)) return false;
  const float inv = 1.0f / det;
  float l0[3];
  for (int k = 0; k < 3; ++k) l0[k] = fmaf(gt, x12[k], fmaf(gu, x20[k], gv * x01[k])) * inv;
  // residual of the equations c_i . lambda = g_i, in double
  const double r0 = (double)gt - (c0[0] * l0[0] + c0[1] * l0[1] + c0[2] * l0[2]);
  const double r1 = (double)gu - (c1[0] * l0[0] + c1[1] * l0[1] + c1[2] * l0[2]);
  const double r2 = (double)gv - (c2[0] * l0[0] + c2[1] * l0[1] + c2[2] * l0[2]);
  const float s0 = (float)r0, s1 = (float)r1, s2 = (float)r2;
  for (int k = 0; k < 3; ++k) {
    lam[k] = (double)l0[k] + (double)(fmaf(s0, x12[k], fmaf(s1, x20[k], s2 * x01[k])) * inv);
    if (!isfinite(lam[k])) return false;
  }
  return true;
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
    // columns of J, exact in double (differences of two floats)
    const double c0[3] = {rd.x, rd.y, rd.z};
    const double c1[3] = {-((double)p1.x - p0.x), -((double)p1.y - p0.y), -((double)p1.z - p0.z)};
    const double c2[3] = {-((double)p2.x - p0.x), -((double)p2.y - p0.y), -((double)p2.z - p0.z)};
    const float gt = a.grad_tuv[3 * i], gu = a.grad_tuv[3 * i + 1], gv = a.grad_tuv[3 * i + 2];
    double lam[3];
    if (!solve_refined(c0, c1, c2, gt, gu, gv, lam)) {
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
      for (int k = 0; k < 3; ++k) lam[k] = ((double)gt * x12[k] + (double)gu * x20[k] + (double)gv * x01[k]) / det;
    }
    // the scatter in single precision from lambda rounded once
    const float lf[3] = {(float)lam[0], (float)lam[1], (float)lam[2]};
    const float t = __uint_as_float(h.x), u = __uint_as_float(h.y), v = __uint_as_float(h.z);
    const float w[3] = {(1.0f - u) - v, u, v};
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) atomicAdd(a.grad_verts + 3 * (size_t)vid[j] + k, w[j] * lf[k]);
    if (gr) {
      gr[0] = make_float4(-lf[0], -lf[1], -lf[2], 0.f);
      gr[1] = make_float4(-t * lf[0], -t * lf[1], -t * lf[2], 0.f);
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
