// Layout-polymorphic closest-hit / any-hit traversal for sm_103a.
//
// One traversal loop (the closest_hit of Fig. 4 / App. G: test bounds, cull on
// distmin against the best hit, descend, loop the leaf's triangles) is
// instantiated per physical layout: the node codec (own-box binary node or
// children-in-parent wide node of width W with f32/f16/u8 boxes, AoS or SoA,
// direct or indirect child references) is a set of template parameters, so
// every field access compiles to fixed offsets into registers loaded with
// 256-bit non-coherent loads (node strides are multiples of 32 bytes).
//
// Execution model: a persistent grid (a few CTAs per SM); each warp takes 32
// rays at a time from a global counter with one atomicAdd (or an 8x4 pixel
// tile of a row-major image of camera rays), or refills its idle lanes from
// its CTA's share once enough of them are idle (body_refill); each lane
// traces one ray with a per-thread stack whose first entries live in shared
// memory (strided by blockDim, conflict-free) and whose tail spills to local
// memory, or, where a kernel has the register for it, whose shared part is a
// ring of the most recent entries (StackT). The current entry is always in
// registers.
//
// Arithmetic: the box test only has to be conservative; the triangle test is
// pinned bit for bit (see tri_test). Translation units are compiled with
// --fmad=false so that only the explicit fmaf calls fuse.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/scion.h"
#include "layout.h"

namespace scion {

struct TraceArgs {
  const uint4 *nodes;       // node buffer (AoS nodes, or own-box SoA boxes)
  const uint2 *nodes2;      // own-box SoA reference array
  const float4 *prims;      // direct primitives, 3 float4 per entry
  const uint32_t *prim_ids; // indirect primitives
  const float4 *verts;      // float4 vertex table
  const uint32_t *tri_idx;  // u32[3] per triangle, or null for a soup
  const float4 *rays;       // 2 float4 per ray
  void *out;                // scion_hit[n] (uint4) or uint32[n]
  unsigned long long n;
  uint32_t root_ref;
  uint32_t n_nodes;
  uint32_t prim_indirect;
  uint32_t max_steps;
  uint32_t ordered;         // 0 slot order, 1 sorted by entry distance, 2 nearest first
  uint32_t smem_stack;      // shared-memory stack entries per thread
  uint32_t refill_min;      // 0: 32-ray warp batches; k: refill once k lanes idle
  uint32_t raster_w;        // 0, or rays form a row-major image this wide: warp batches are 8x4 tiles
  unsigned long long n_work;  // warp-batch slots: n, or 32 per tile of the image
  unsigned long long *work; // persistent work counter (self-resetting)
  uint32_t *exit_count;     // CTAs finished (self-resetting)
  uint32_t *status;         // first device error code
  unsigned long long *stats;  // counting kernels: nodes, leaves, prim tests, rays
  uint32_t node_stride;     // own-box node (or SoA box record) bytes
  float frame[9];           // world grid of q16 {wlo, step} / eq10 {wlo, whi, bin}
};

// Per-thread visit counters of the counting (STATS) kernels.
struct Counts {
  uint32_t nodes = 0, leaves = 0, prims = 0;
};

constexpr int kLocalStack = 48;           // local-memory tail of the stack
constexpr float kNearScale = 1.0f - 9.5367431640625e-07f;  // 1 - 2^-20: relative slab widening
constexpr float kFarScale = 1.0f + 9.5367431640625e-07f;   // 1 + 2^-20
constexpr uint32_t kErrStack = 5, kErrIter = 6;   // scion_status codes

// ------------------------------------------------------------------ ray state
struct Ray {
  float ox, oy, oz, tmin, dx, dy, dz, tmax;
  // box test: reciprocal direction (zero components replaced by a tiny
  // signed value), o * rdir, and which plane is near per axis
  float rx, ry, rz, orx, ory, orz;
  bool nx, ny, nz;
  // watertight test: permuted axes and shear constants
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ float sel3(float x, float y, float z, int k) {
  return k == 0 ? x : (k == 1 ? y : z);
}

__device__ __forceinline__ float safe_rcp(float d) {
  const float dd = d == 0.0f ? copysignf(1e-30f, d) : d;
  return __fdiv_rn(1.0f, dd);
}

__device__ __forceinline__ void setup_ray(const float4 a, const float4 b, Ray &r) {
  // hits behind the origin are never reported: tmin below 0 (or NaN) is 0
  r.ox = a.x; r.oy = a.y; r.oz = a.z; r.tmin = a.w > 0.0f ? a.w : 0.0f;
  r.dx = b.x; r.dy = b.y; r.dz = b.z; r.tmax = b.w;
  r.rx = safe_rcp(r.dx); r.ry = safe_rcp(r.dy); r.rz = safe_rcp(r.dz);
  r.orx = __fmul_rn(r.ox, r.rx); r.ory = __fmul_rn(r.oy, r.ry); r.orz = __fmul_rn(r.oz, r.rz);
  r.nx = r.rx < 0.0f; r.ny = r.ry < 0.0f; r.nz = r.rz < 0.0f;
  // axis of largest |d| (ties to the lowest axis); the next two cyclically,
  // swapped when d[kz] < 0 to keep the winding
  const float ax = fabsf(r.dx), ay = fabsf(r.dy), az = fabsf(r.dz);
  int kz = 0;
  float m = ax;
  if (ay > m) { kz = 1; m = ay; }
  if (az > m) { kz = 2; }
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  const float dkz = sel3(r.dx, r.dy, r.dz, kz);
  if (dkz < 0.0f) { const int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  r.Sx = __fdiv_rn(sel3(r.dx, r.dy, r.dz, kx), dkz);
  r.Sy = __fdiv_rn(sel3(r.dx, r.dy, r.dz, ky), dkz);
  // 1 / d[kz] is the slab reciprocal of that axis already (the same IEEE
  // division: safe_rcp replaces only a zero component, and d[kz] = 0 only when
  // every component is 0, where 1 / +-0 = +-inf)
  r.Sz = dkz != 0.0f ? sel3(r.rx, r.ry, r.rz, kz) : copysignf(__int_as_float(0x7f800000), dkz);
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Conservative slab test from the six plane distances (near planes t0*, far
// planes t1*) against [tmin, tlim]; returns the widened entry distance in tn.
// Because tmin >= 0, scaling the entry distance by (1 - 2^-20) and the exit
// distance by (1 + 2^-20) widens the interval by that relative amount wherever
// the decision can change. NaNs from 0*inf are ignored by min/max (the axis
// then does not cull).
__device__ __forceinline__ bool slab_t(const Ray &r, float t0x, float t0y, float t0z, float t1x,
                                       float t1y, float t1z, float tlim, float &tn) {
  float a = fmax3(t0x, t0y, t0z) * kNearScale;
  float b = fmin3(t1x, t1y, t1z) * kFarScale;
  a = fmaxf(a, r.tmin);
  b = fminf(b, tlim);
  tn = a;
  return a <= b;
}

// Two fused multiply-adds with one instruction (fma.rn.f32x2, sm_100 and
// later): the same IEEE fma rounding per element as two fmaf calls.
__device__ __forceinline__ void fma_pair(float a0, float a1, float m, float b, float &r0, float &r1) {
  const float2 r = __ffma2_rn(make_float2(a0, a1), make_float2(m, m), make_float2(b, b));
  r0 = r.x;
  r1 = r.y;
}
// Two exact small-integer decodes x - 2^23 (the code sits in the low
// mantissa bits of 2^23) with one add.f32x2.
__device__ __forceinline__ void unbias_pair(float x0, float x1, float &r0, float &r1) {
  const float2 r = __fadd2_rn(make_float2(x0, x1), make_float2(-8388608.0f, -8388608.0f));
  r0 = r.x;
  r1 = r.y;
}

// The six plane distances of a box given by its corners: near/far planes by
// direction sign, distance = fma(plane, 1/d, -o/d), each axis's near and far
// plane in one paired fma.
__device__ __forceinline__ void box_planes(const Ray &r, float lox, float loy, float loz, float hix, float hiy,
                                           float hiz, float (&t0)[3], float (&t1)[3]) {
  fma_pair(r.nx ? hix : lox, r.nx ? lox : hix, r.rx, -r.orx, t0[0], t1[0]);
  fma_pair(r.ny ? hiy : loy, r.ny ? loy : hiy, r.ry, -r.ory, t0[1], t1[1]);
  fma_pair(r.nz ? hiz : loz, r.nz ? loz : hiz, r.rz, -r.orz, t0[2], t1[2]);
}

// The slab test of a box given by its corners. PAIRED = false takes one fmaf
// per plane: a paired fma wants each ray constant twice in a register pair,
// which makes the 64-register wide-node kernels spill.
template <bool PAIRED = true>
__device__ __forceinline__ bool slab(const Ray &r, float lox, float loy, float loz, float hix,
                                     float hiy, float hiz, float tlim, float &tn) {
  float t0[3], t1[3];
  if (PAIRED) {
    box_planes(r, lox, loy, loz, hix, hiy, hiz, t0, t1);
  } else {
    const float nx = r.nx ? hix : lox, fx = r.nx ? lox : hix;
    const float ny = r.ny ? hiy : loy, fy = r.ny ? loy : hiy;
    const float nz = r.nz ? hiz : loz, fz = r.nz ? loz : hiz;
    t0[0] = fmaf(nx, r.rx, -r.orx); t0[1] = fmaf(ny, r.ry, -r.ory); t0[2] = fmaf(nz, r.rz, -r.orz);
    t1[0] = fmaf(fx, r.rx, -r.orx); t1[1] = fmaf(fy, r.ry, -r.ory); t1[2] = fmaf(fz, r.rz, -r.orz);
  }
  return slab_t(r, t0[0], t0[1], t0[2], t1[0], t1[1], t1[2], tlim, tn);
}

// The conservative ray interval [tn, tf] of a box, clamped to [tmin, tlim].
__device__ __forceinline__ bool slab_interval(const Ray &r, float lox, float loy, float loz, float hix,
                                              float hiy, float hiz, float tlim, float &tn, float &tf) {
  float t0[3], t1[3];
  box_planes(r, lox, loy, loz, hix, hiy, hiz, t0, t1);
  tn = fmaxf(fmax3(t0[0], t0[1], t0[2]) * kNearScale, r.tmin);
  tf = fminf(fmin3(t1[0], t1[1], t1[2]) * kFarScale, tlim);
  return tn <= tf;
}

// Pinned watertight ray/triangle test (Woop, Benthin & Wald, JCGT 2(1) 2013;
// the paper's App. G uses Moller-Trumbore instead). Steps and rounding:
//   A = p0 - o, B = p1 - o, C = p2 - o; sheared Ax = fma(-Sx, A[kz], A[kx]),
//   Ay = fma(-Sy, A[kz], A[ky]) (same for B, C); edge functions
//   U = Cx*By - Cy*Bx, V = Ax*Cy - Ay*Cx, W = Bx*Ay - By*Ax with both
//   products rounded (so a shared edge evaluates to exactly opposite values);
//   if one is zero, all three are redone from exact double products; miss on
//   mixed signs; det = (U+V)+W, miss if 0; T = fma(W, Cz, fma(V, Bz, U*Az))
//   with Az = Sz*A[kz] etc.; t = T/det; accept iff tmin <= t <= tmax.
// Returns t (and det, U for the barycentrics) on acceptance.
__device__ __forceinline__ bool tri_test(const Ray &r, float4 p0, float4 p1, float4 p2,
                                         float &t_out, float &V_out, float &W_out,
                                         float &det_out) {
  const float Akx = __fsub_rn(sel3(p0.x, p0.y, p0.z, r.kx), sel3(r.ox, r.oy, r.oz, r.kx));
  const float Aky = __fsub_rn(sel3(p0.x, p0.y, p0.z, r.ky), sel3(r.ox, r.oy, r.oz, r.ky));
  const float Akz = __fsub_rn(sel3(p0.x, p0.y, p0.z, r.kz), sel3(r.ox, r.oy, r.oz, r.kz));
  const float Bkx = __fsub_rn(sel3(p1.x, p1.y, p1.z, r.kx), sel3(r.ox, r.oy, r.oz, r.kx));
  const float Bky = __fsub_rn(sel3(p1.x, p1.y, p1.z, r.ky), sel3(r.ox, r.oy, r.oz, r.ky));
  const float Bkz = __fsub_rn(sel3(p1.x, p1.y, p1.z, r.kz), sel3(r.ox, r.oy, r.oz, r.kz));
  const float Ckx = __fsub_rn(sel3(p2.x, p2.y, p2.z, r.kx), sel3(r.ox, r.oy, r.oz, r.kx));
  const float Cky = __fsub_rn(sel3(p2.x, p2.y, p2.z, r.ky), sel3(r.ox, r.oy, r.oz, r.ky));
  const float Ckz = __fsub_rn(sel3(p2.x, p2.y, p2.z, r.kz), sel3(r.ox, r.oy, r.oz, r.kz));
  const float Ax = fmaf(-r.Sx, Akz, Akx), Ay = fmaf(-r.Sy, Akz, Aky);
  const float Bx = fmaf(-r.Sx, Bkz, Bkx), By = fmaf(-r.Sy, Bkz, Bky);
  const float Cx = fmaf(-r.Sx, Ckz, Ckx), Cy = fmaf(-r.Sy, Ckz, Cky);
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = __double2float_rn(__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx)));
    V = __double2float_rn(__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx)));
    W = __double2float_rn(__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax)));
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
  const float det = __fadd_rn(__fadd_rn(U, V), W);
  if (det == 0.0f) return false;
  const float Az = __fmul_rn(r.Sz, Akz), Bz = __fmul_rn(r.Sz, Bkz), Cz = __fmul_rn(r.Sz, Ckz);
  const float T = fmaf(W, Cz, fmaf(V, Bz, __fmul_rn(U, Az)));
  const float t = __fdiv_rn(T, det);
  if (!(t >= r.tmin && t <= r.tmax)) return false;
  t_out = t;
  V_out = V;
  W_out = W;
  det_out = det;
  return true;
}

// ------------------------------------------------------------------ loads
__device__ __forceinline__ uint4 ldg4(const uint4 *p) { return __ldg(p); }
// 256-bit non-coherent load of two consecutive uint4 (p 32-byte aligned):
// one L1 request per 32-byte sector instead of one per 16 bytes
__device__ __forceinline__ void ldg8(const uint4 *p, uint4 &lo, uint4 &hi) {
  asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
      : "l"(p));
}
// A node of NQ 16-byte words at a 32-byte aligned address (node strides are
// multiples of 32 bytes and node buffers are separately allocated): 256-bit
// loads, and a 128-bit load for an odd last word.
template <int NQ>
__device__ __forceinline__ void load_node(const uint4 *np, uint4 (&q)[NQ]) {
#pragma unroll
  for (int i = 0; i + 1 < NQ; i += 2) ldg8(np + i, q[i], q[i + 1]);
  if constexpr ((NQ & 1) != 0) q[NQ - 1] = ldg4(np + NQ - 1);
}
__device__ __forceinline__ float4 ldg4f(const float4 *p) { return __ldg(p); }

template <int NQ>
__device__ __forceinline__ uint32_t qword(const uint4 (&q)[NQ], int i) {
  const uint4 v = q[i >> 2];
  switch (i & 3) {
    case 0: return v.x;
    case 1: return v.y;
    case 2: return v.z;
    default: return v.w;
  }
}

// ------------------------------------------------------------------ stack
// Entries (ref, entry distance); with TF also the exit distance of the
// entry's interval (the shared-slab traversal carries intervals, not boxes),
// in a second shared-memory column.
//
// Three tiers, newest entries first: R entries in registers (R = 0, 2 or 4,
// the traversal parameter reg_stack), then cap_sh entries in this thread's
// shared-memory column, then a local-memory tail. The register tier is a
// shift register (rr[0] newest; pushes and pops move every register entry,
// so each index is a compile-time constant and the entries stay in
// registers); when it is full, a push moves its oldest entry into shared
// memory. Pops take the register entries first and only then read memory.
// The local-memory tail of a stack, declared apart from the stack's scalar
// state: an array indexed at run time lives in local memory, and a struct
// that held one would take its other members (the stack pointer, the
// capacity) there with it, costing local loads and stores on every step.
template <bool TF>
struct StackTail {
  uint2 loc[kLocalStack];
  float locf[TF ? kLocalStack : 1];
};

template <bool TF, bool RING = false, int R = 0>
struct StackT {
  uint2 *sh;      // this thread's column in shared memory
  float *shf;     // exit distances (TF)
  int stride;     // blockDim.x
  int cap_sh;     // entries in shared memory (RING: a power of two)
  int sp;         // entries in memory (shared + local)
  int base;       // RING: entries [0, base) are in local memory, [base, sp) in shared memory
  int rn;         // entries in registers
  float ptf;      // exit distance of the last popped entry (TF)
  uint32_t rr[R > 0 ? R : 1];
  float rt[R > 0 ? R : 1];
  float rf[(R > 0 && TF) ? R : 1];
  uint2 *loc;     // the local-memory tail (StackTail)
  float *locf;
  static constexpr int kRegs = R;
  static constexpr bool kTF = TF;

  __device__ __forceinline__ void attach(StackTail<TF> &t) {
    loc = t.loc;
    locf = t.locf;
  }

  // Without RING the first cap_sh memory entries live in shared memory and
  // deeper ones in local memory. With RING the shared part holds the cap_sh
  // most recent memory entries: when it is full the oldest one moves to
  // local memory, which is read again only once the shared part is empty, so
  // pushes and pops near the top stay in shared memory however deep the
  // stack grows.
  __device__ __forceinline__ int slot(int i) const { return (RING ? (i & (cap_sh - 1)) : i) * stride; }
  __device__ __forceinline__ void reset() {
    sp = 0;
    base = 0;
    rn = 0;
  }
  __device__ __forceinline__ bool empty() const { return sp + rn == 0; }
  __device__ __forceinline__ bool mem_push(uint2 e, float tf) {
    if constexpr (RING) {
      if (sp - base == cap_sh) {
        if (base == kLocalStack) return false;
        loc[base] = sh[slot(base)];
        if (TF) locf[base] = shf[slot(base)];
        ++base;
      }
      sh[slot(sp)] = e;
      if (TF) shf[slot(sp)] = tf;
    } else {
      if (sp < cap_sh) {
        sh[sp * stride] = e;
        if (TF) shf[sp * stride] = tf;
      } else if (sp < cap_sh + kLocalStack) {
        loc[sp - cap_sh] = e;
        if (TF) locf[sp - cap_sh] = tf;
      } else {
        return false;
      }
    }
    ++sp;
    return true;
  }
  __device__ __forceinline__ uint2 mem_pop() {
    --sp;
    if constexpr (RING) {
      if (sp >= base) {
        if (TF) ptf = shf[slot(sp)];
        return sh[slot(sp)];
      }
      base = sp;
      if (TF) ptf = locf[sp];
      return loc[sp];
    } else {
      if (sp < cap_sh) {
        if (TF) ptf = shf[sp * stride];
        return sh[sp * stride];
      }
      if (TF) ptf = locf[sp - cap_sh];
      return loc[sp - cap_sh];
    }
  }
  __device__ __forceinline__ bool push(uint32_t ref, float tn, float tf = 0.f) {
    if constexpr (R > 0) {
      if (rn == R) {
        if (!mem_push(make_uint2(rr[R - 1], __float_as_uint(rt[R - 1])), TF ? rf[R - 1] : 0.f)) return false;
      } else {
        ++rn;
      }
#pragma unroll
      for (int i = R - 1; i > 0; --i) {
        rr[i] = rr[i - 1];
        rt[i] = rt[i - 1];
        if (TF) rf[i] = rf[i - 1];
      }
      rr[0] = ref;
      rt[0] = tn;
      if (TF) rf[0] = tf;
      return true;
    } else {
      return mem_push(make_uint2(ref, __float_as_uint(tn)), tf);
    }
  }
  // Only when !empty().
  __device__ __forceinline__ uint2 pop() {
    if constexpr (R > 0) {
      if (rn > 0) {
        const uint2 e = make_uint2(rr[0], __float_as_uint(rt[0]));
        if (TF) ptf = rf[0];
#pragma unroll
        for (int i = 0; i + 1 < R; ++i) {
          rr[i] = rr[i + 1];
          rt[i] = rt[i + 1];
          if (TF) rf[i] = rf[i + 1];
        }
        --rn;
        return e;
      }
    }
    return mem_pop();
  }
};
using Stack = StackT<false>;

// ------------------------------------------------------------------ leaf
struct Best {
  float t, u, v;
  uint32_t id;
};

// Test the triangles [first, first + count). Closest: keep the lexicographic
// minimum of (t, id). Any: return true at the first accepted hit.
template <bool ANY, bool STATS>
__device__ __forceinline__ bool visit_leaf(const TraceArgs &a, const Ray &r, uint32_t first,
                                           uint32_t count, Best &b, Counts &cnt) {
  if (STATS) cnt.leaves++;
  for (uint32_t i = first; i < first + count; ++i) {
    if (STATS) cnt.prims++;
    float4 p0, p1, p2;
    uint32_t id;
    if (a.prim_indirect) {
      id = __ldg(a.prim_ids + i);
      uint32_t i0, i1, i2;
      if (a.tri_idx) {
        i0 = __ldg(a.tri_idx + 3 * (size_t)id);
        i1 = __ldg(a.tri_idx + 3 * (size_t)id + 1);
        i2 = __ldg(a.tri_idx + 3 * (size_t)id + 2);
      } else {
        i0 = 3 * id; i1 = i0 + 1; i2 = i0 + 2;
      }
      p0 = ldg4f(a.verts + i0);
      p1 = ldg4f(a.verts + i1);
      p2 = ldg4f(a.verts + i2);
    } else {
      const float4 *q = a.prims + 3 * (size_t)i;
      p0 = ldg4f(q);
      p1 = ldg4f(q + 1);
      p2 = ldg4f(q + 2);
      id = __float_as_uint(p0.w);
    }
    float t, V, W, det;
    if (!tri_test(r, p0, p1, p2, t, V, W, det)) continue;
    if (ANY) return true;
    if (t < b.t || (t == b.t && id < b.id)) {
      b.t = t;
      b.u = __fdiv_rn(V, det);
      b.v = __fdiv_rn(W, det);
      b.id = id;
    }
  }
  return false;
}

// ------------------------------------------------------------------ wide node
template <int W, int PREC, int SOA, int CREF>
struct WideNode {
  static constexpr bool kGrid = PREC == PREC_U8 || PREC == PREC_U16;  // codes on a node frame
  static constexpr int kHdr = kGrid ? 16 : 0;
  static constexpr int kElem = PREC == PREC_F32 ? 4 : (PREC == PREC_U8 ? 1 : 2);
  static constexpr int kRefOff = kHdr + W * 6 * kElem;
  static constexpr int kBytes = kRefOff + (CREF == REF_DIRECT ? 4 * W : 8 + W);
  static constexpr int kStride = (kBytes + 31) & ~31;
  static constexpr int NQ = (kBytes + 15) / 16;
  // SoA sub-word boxes whose coordinate rows are whole words: the near/far
  // choice of an axis is made once per word for all children in it
  static constexpr bool kRowSel = SOA && kElem < 4 && (W * kElem) % 4 == 0;
  static constexpr int kRowWords = (W * kElem) / 4;
  static constexpr int kPerWord = 4 / kElem;

  static __device__ __forceinline__ int box_off(int k, int c) {
    return kHdr + (SOA ? (c * W + k) : (k * 6 + c)) * kElem;
  }
  // raw quantity of coordinate c of child k (f32 value, f16 bits or u8 code)
  static __device__ __forceinline__ uint32_t raw(const uint4 (&q)[NQ], int k, int c) {
    const int off = box_off(k, c);
    const uint32_t w = qword(q, off >> 2);
    if (kElem == 4) return w;
    if (kElem == 2) return (w >> ((off & 3) * 8)) & 0xFFFFu;
    return (w >> ((off & 3) * 8)) & 0xFFu;
  }
  // u8 / u16 code of coordinate c of child k as a float, exactly: a byte
  // permute puts the code into the low mantissa bits of 2^23, then 2^23 is
  // taken off (full-rate integer/float ops instead of an integer-to-float
  // conversion)
  static __device__ __forceinline__ float code_biased(const uint4 (&q)[NQ], int k, int c) {
    const int off = box_off(k, c);
    const uint32_t w = qword(q, off >> 2);
    const uint32_t b = (uint32_t)(off & 3);
    const uint32_t sel = kElem == 1 ? (0x7540u | b) : (0x7400u | ((b + 1u) << 4) | b);
    return __uint_as_float(__byte_perm(w, 0x4B000000u, sel));  // 2^23 + code
  }
  static __device__ __forceinline__ float code(const uint4 (&q)[NQ], int k, int c) {
    return code_biased(q, k, c) - 8388608.0f;
  }
};

// Per-lane traversal state that survives between steps, so that a lane can
// finish its ray and take a new one while the rest of its warp is mid-ray.
struct Lane {
  Ray r;
  Best b;
  uint32_t cur;      // entry being processed (kEmptyRef: ray finished)
  float ctn, ctf;    // shared-slab layout: the current node's ray interval
  uint32_t steps;
  uint32_t err;
  bool found;        // any-hit result
  unsigned long long rid;
};

// Next stacked entry that can still hold a closer hit (closest) or any
// stacked entry (any-hit); kEmptyRef when the stack is exhausted.
template <bool ANY, class S>
__device__ __forceinline__ uint32_t pop_next(S &st, float best_t, float &tn) {
  while (!st.empty()) {
    const uint2 e = st.pop();
    tn = __uint_as_float(e.y);
    if (ANY || tn <= best_t) return e.x;
  }
  return kEmptyRef;
}
template <bool ANY, class S>
__device__ __forceinline__ uint32_t pop_next(S &st, float best_t) {
  float tn;
  return pop_next<ANY>(st, best_t, tn);
}

// Ascending sort of (entry distance, reference) pairs with a fixed
// compare-exchange network: 1 comparator for 2 children, 5 for 4, 19 for 8
// (Batcher's odd-even merge sort).
__device__ __forceinline__ void cmpx(float *t, uint32_t *r, int i, int j) {
  const bool sw = t[j] < t[i];
  const float ti = sw ? t[j] : t[i], tj = sw ? t[i] : t[j];
  const uint32_t ri = sw ? r[j] : r[i], rj = sw ? r[i] : r[j];
  t[i] = ti; t[j] = tj; r[i] = ri; r[j] = rj;
}

template <int W>
__device__ __forceinline__ void sort_children(float (&t)[W], uint32_t (&r)[W]) {
  if constexpr (W == 2) {
    cmpx(t, r, 0, 1);
  } else if constexpr (W == 4) {
    cmpx(t, r, 0, 1); cmpx(t, r, 2, 3); cmpx(t, r, 0, 2); cmpx(t, r, 1, 3); cmpx(t, r, 1, 2);
  } else {
    cmpx(t, r, 0, 1); cmpx(t, r, 2, 3); cmpx(t, r, 4, 5); cmpx(t, r, 6, 7);
    cmpx(t, r, 0, 2); cmpx(t, r, 1, 3); cmpx(t, r, 4, 6); cmpx(t, r, 5, 7);
    cmpx(t, r, 1, 2); cmpx(t, r, 5, 6);
    cmpx(t, r, 0, 4); cmpx(t, r, 1, 5); cmpx(t, r, 2, 6); cmpx(t, r, 3, 7);
    cmpx(t, r, 2, 4); cmpx(t, r, 3, 5);
    cmpx(t, r, 1, 2); cmpx(t, r, 3, 4); cmpx(t, r, 5, 6);
  }
}

// One step of the wide-node traversal: process the entry L.cur (an interior
// node: test its W child boxes, push the hit ones far to near, continue with
// the nearest; or a leaf: test its triangles), then pick the next entry.
template <int W, int PREC, int SOA, int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void step_wide(const TraceArgs &a, Lane &L, S &st, Counts &cnt) {
  using N = WideNode<W, PREC, SOA, CREF>;
  const Ray &r = L.r;
  const uint32_t cur = L.cur;
  if (ref_is_interior(cur)) {
    if (STATS) cnt.nodes++;
    const uint4 *np = a.nodes + (size_t)ref_node(cur) * (N::kStride / 16);
    uint4 q[N::NQ];
    load_node<N::NQ>(np, q);
    // u8 / u16 frame: coordinate = origin + code * 2^e, folded into the plane
    // distance t = fma(code, 2^e / d, (origin - o) / d) per axis
    float ax = 0.f, bx = 0.f, ay = 0.f, by = 0.f, az = 0.f, bz = 0.f;
    if (N::kGrid) {
      ax = __uint_as_float((q[0].w & 0xFFu) << 23) * r.rx;
      ay = __uint_as_float(((q[0].w >> 8) & 0xFFu) << 23) * r.ry;
      az = __uint_as_float(((q[0].w >> 16) & 0xFFu) << 23) * r.rz;
      bx = fmaf(__uint_as_float(q[0].x), r.rx, -r.orx);
      by = fmaf(__uint_as_float(q[0].y), r.ry, -r.ory);
      bz = fmaf(__uint_as_float(q[0].z), r.rz, -r.orz);
    }
    const float tlim = ANY ? r.tmax : fminf(r.tmax, L.b.t);
    // paired decode and fma (f32x2) for the grid codes; the 8-wide kernels
    // would spill with the extra register pairs
    constexpr bool kPaired = W <= 4;
    uint32_t cref[W];
    float ctn[W];
    uint32_t base_node = 0, base_prim = 0, leaf_acc = 0;
    if (CREF == REF_INDIRECT) {
      base_node = qword(q, N::kRefOff / 4);
      base_prim = qword(q, N::kRefOff / 4 + 1);
    }
    // reference of child k (in increasing k: indirect leaves accumulate)
    auto child_ref = [&](int k) -> uint32_t {
      if (CREF == REF_DIRECT) return qword(q, N::kRefOff / 4 + k);
      const uint32_t m = (qword(q, N::kRefOff / 4 + 2 + (k >> 2)) >> ((k & 3) * 8)) & 0xFFu;
      if (m == 0) return kEmptyRef;
      if (m & kMetaInterior) return ref_interior(base_node + (m & 0x7Fu));
      const uint32_t rf = ref_leaf(base_prim + leaf_acc, m);
      leaf_acc += m;
      return rf;
    };
    if constexpr (N::kRowSel) {
      constexpr int kRow = N::kRowWords;
#pragma unroll
      for (int j = 0; j < kRow; ++j) {
        // word j of each coordinate row: near and far planes of its children
        uint32_t nw[3], fw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const uint32_t lw = qword(q, N::kHdr / 4 + c * kRow + j), hw = qword(q, N::kHdr / 4 + (c + 3) * kRow + j);
          const bool neg = c == 0 ? r.nx : (c == 1 ? r.ny : r.nz);
          nw[c] = neg ? hw : lw;
          fw[c] = neg ? lw : hw;
        }
#pragma unroll
        for (int i = 0; i < N::kPerWord; ++i) {
          const int k = j * N::kPerWord + i;
          const uint32_t ref = child_ref(k);
          const uint32_t b = (uint32_t)(i * N::kElem);  // byte of the child in the word
          float t0[3], t1[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float rc = c == 0 ? r.rx : (c == 1 ? r.ry : r.rz), oc = c == 0 ? r.orx : (c == 1 ? r.ory : r.orz);
            if (N::kGrid) {
              const uint32_t sel = N::kElem == 1 ? (0x7540u | b) : (0x7400u | ((b + 1u) << 4) | b);
              const float nb = __uint_as_float(__byte_perm(nw[c], 0x4B000000u, sel));
              const float fb = __uint_as_float(__byte_perm(fw[c], 0x4B000000u, sel));
              const float ac = c == 0 ? ax : (c == 1 ? ay : az), bc = c == 0 ? bx : (c == 1 ? by : bz);
              if (kPaired) {
                float nq, fq;
                unbias_pair(nb, fb, nq, fq);
                fma_pair(nq, fq, ac, bc, t0[c], t1[c]);
              } else {
                t0[c] = fmaf(nb - 8388608.0f, ac, bc);
                t1[c] = fmaf(fb - 8388608.0f, ac, bc);
              }
            } else {
              const float nv = __half2float(__ushort_as_half((unsigned short)((nw[c] >> (b * 8)) & 0xFFFFu)));
              const float fv = __half2float(__ushort_as_half((unsigned short)((fw[c] >> (b * 8)) & 0xFFFFu)));
              t0[c] = fmaf(nv, rc, -oc);
              t1[c] = fmaf(fv, rc, -oc);
            }
          }
          float tn;
          bool hit = slab_t(r, t0[0], t0[1], t0[2], t1[0], t1[1], t1[2], tlim, tn);
          hit = hit && ref != kEmptyRef;
          cref[k] = hit ? ref : kEmptyRef;
          ctn[k] = hit ? tn : __int_as_float(0x7f800000);
        }
      }
    } else {
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const uint32_t ref = child_ref(k);
      float tn;
      bool hit;
      if (N::kGrid) {
        // per axis: near and far code of the child (decoded in one paired
        // add), then both plane distances in one paired fma
        float t0[3], t1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const bool neg = c == 0 ? r.nx : (c == 1 ? r.ny : r.nz);
          const float lb = N::code_biased(q, k, c), hb = N::code_biased(q, k, c + 3);
          const float ac = c == 0 ? ax : (c == 1 ? ay : az), bc = c == 0 ? bx : (c == 1 ? by : bz);
          if (kPaired) {
            float nq, fq;
            unbias_pair(neg ? hb : lb, neg ? lb : hb, nq, fq);
            fma_pair(nq, fq, ac, bc, t0[c], t1[c]);
          } else {
            t0[c] = fmaf((neg ? hb : lb) - 8388608.0f, ac, bc);
            t1[c] = fmaf((neg ? lb : hb) - 8388608.0f, ac, bc);
          }
        }
        hit = slab_t(r, t0[0], t0[1], t0[2], t1[0], t1[1], t1[2], tlim, tn);
      } else {
        float lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const uint32_t ql = N::raw(q, k, c), qh = N::raw(q, k, c + 3);
          if (PREC == PREC_F32) {
            lo[c] = __uint_as_float(ql);
            hi[c] = __uint_as_float(qh);
          } else {
            lo[c] = __half2float(__ushort_as_half((unsigned short)ql));
            hi[c] = __half2float(__ushort_as_half((unsigned short)qh));
          }
        }
        hit = slab<false>(r, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], tlim, tn);
      }
      hit = hit && ref != kEmptyRef;
      cref[k] = hit ? ref : kEmptyRef;
      ctn[k] = hit ? tn : __int_as_float(0x7f800000);
    }
    }
    if (!ANY && a.ordered == 1) {
      sort_children<W>(ctn, cref);
    } else if (!ANY && a.ordered == 2) {
      // nearest first, the rest in slot order: move the nearest hit child
      // into slot 0 (one pass of compare-exchanges toward the front)
#pragma unroll
      for (int k = W - 1; k > 0; --k) cmpx(ctn, cref, k - 1, k);
    }
    // push every hit child but the first, last one first; go on with the first
    uint32_t next = kEmptyRef;
    float next_tn = 0.f;
    if (S::kRegs == 0 && st.sp - st.base + W <= st.cap_sh) {
      // room in shared memory for any node: predicated stores, one check
      int sp = st.sp;
#pragma unroll
      for (int k = W - 1; k >= 0; --k) {
        const bool h = cref[k] != kEmptyRef;
        if (h && next != kEmptyRef) st.sh[st.slot(sp++)] = make_uint2(next, __float_as_uint(next_tn));
        next = h ? cref[k] : next;
        next_tn = h ? ctn[k] : next_tn;
      }
      st.sp = sp;
    } else {
#pragma unroll
      for (int k = W - 1; k >= 0; --k) {
        if (cref[k] == kEmptyRef) continue;
        if (next != kEmptyRef && !st.push(next, next_tn)) { L.err = kErrStack; L.cur = kEmptyRef; return; }
        next = cref[k];
        next_tn = ctn[k];
      }
    }
    L.cur = next != kEmptyRef ? next : pop_next<ANY>(st, L.b.t);
  } else {
    // One triangle per step: the entry then names the leaf's remaining
    // triangles (first + 1, count - 1), so a lane in a leaf holds its warp for
    // one triangle test per step rather than for the whole leaf while the
    // other lanes wait. The counting kernels test the whole leaf at once (the
    // same triangles, so the same counts).
    const uint32_t count = ref_leaf_count(cur);
    constexpr bool kWhole = STATS;
    if (visit_leaf<ANY, STATS>(a, r, ref_leaf_first(cur), kWhole ? count : 1u, L.b, cnt)) {
      L.found = true;
      L.cur = kEmptyRef;
      return;
    }
    if (!kWhole && count > 1u) {
      L.cur = cur + (1u << 5) - (1u << 1);  // ref_leaf(first + 1, count - 1)
      return;
    }
    L.cur = pop_next<ANY>(st, L.b.t);
  }
}

// Exact small-integer to float conversions with full-rate integer ops: the
// code goes into the low mantissa bits of 2^23, then 2^23 is subtracted.
__device__ __forceinline__ float u16lo_b(uint32_t w) {  // 2^23 + low half
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7410u));
}
__device__ __forceinline__ float u16hi_b(uint32_t w) {  // 2^23 + high half
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7432u));
}
__device__ __forceinline__ float u16lo_f(uint32_t w) { return u16lo_b(w) - 8388608.0f; }
__device__ __forceinline__ float u16hi_f(uint32_t w) { return u16hi_b(w) - 8388608.0f; }
__device__ __forceinline__ float eq10_f(uint32_t w, int axis) {
  return __uint_as_float(0x4B000000u | eq10_code(w, axis)) - 8388608.0f;
}

// One step of the own-box binary traversal (pbrt LinearBVH, Fig. 4b): test
// the node's own box; a leaf tests its triangles, an interior node pushes its
// far child (by the split axis and the ray direction) and continues near.
// PREC selects the box codec: f32 corners, or world-grid codes decoded
// exactly as the packer verified them (q16: fma(code, step, wlo); eq10: one
// fused multiply-add rounded outward per coordinate) before the f32 slab test.
template <int PREC, int SOA, int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void step_bin(const TraceArgs &a, Lane &L, S &st, Counts &cnt) {
  const Ray &r = L.r;
  const uint32_t cur = L.cur;
  if (STATS) cnt.nodes++;
  float lo0, lo1, lo2, hi0, hi1, hi2;
  uint32_t field, n, axis;  // child reference / first prim, prim count, split axis
  if (PREC == PREC_F32) {
    uint32_t ref, meta;
    if (SOA) {
      const uint2 *bp = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(a.nodes) +
                                                        (size_t)cur * a.node_stride);
      const uint2 b0 = __ldg(bp), b1 = __ldg(bp + 1), b2 = __ldg(bp + 2);
      const uint2 rm = __ldg(a.nodes2 + cur);
      lo0 = __uint_as_float(b0.x); lo1 = __uint_as_float(b0.y); lo2 = __uint_as_float(b1.x);
      hi0 = __uint_as_float(b1.y); hi1 = __uint_as_float(b2.x); hi2 = __uint_as_float(b2.y);
      ref = rm.x; meta = rm.y;
    } else {
      uint4 q0, q1;
      ldg8(a.nodes + 2 * (size_t)cur, q0, q1);
      lo0 = __uint_as_float(q0.x); lo1 = __uint_as_float(q0.y); lo2 = __uint_as_float(q0.z);
      hi0 = __uint_as_float(q0.w); hi1 = __uint_as_float(q1.x); hi2 = __uint_as_float(q1.y);
      ref = q1.z; meta = q1.w;
    }
    field = ref;
    n = bin_meta_count(meta);
    axis = bin_meta_axis(meta);
  } else {
    const char *np = reinterpret_cast<const char *>(a.nodes) + (size_t)cur * a.node_stride;
    uint32_t w0, w1, w2, w3 = 0;
    if (a.node_stride == 16) {
      const uint4 v = ldg4(reinterpret_cast<const uint4 *>(np));
      w0 = v.x; w1 = v.y; w2 = v.z; w3 = v.w;
    } else {
      const uint32_t *wp = reinterpret_cast<const uint32_t *>(np);
      w0 = __ldg(wp); w1 = __ldg(wp + 1); w2 = __ldg(wp + 2);
    }
    uint32_t word;
    if (PREC == PREC_Q16) {
      // codes: w0 = lo.x | lo.y << 16, w1 = lo.z | hi.x << 16, w2 = hi.y | hi.z << 16
      word = SOA ? __ldg(reinterpret_cast<const uint32_t *>(a.nodes2) + cur) : w3;
      // per axis the lo and hi code decoded, then placed on the grid, in pairs
      float c0l, c0h, c1l, c1h, c2l, c2h;
      unbias_pair(u16lo_b(w0), u16hi_b(w1), c0l, c0h);
      unbias_pair(u16hi_b(w0), u16lo_b(w2), c1l, c1h);
      unbias_pair(u16lo_b(w1), u16hi_b(w2), c2l, c2h);
      fma_pair(c0l, c0h, a.frame[3], a.frame[0], lo0, hi0);
      fma_pair(c1l, c1h, a.frame[4], a.frame[1], lo1, hi1);
      fma_pair(c2l, c2h, a.frame[5], a.frame[2], lo2, hi2);
    } else {
      // w0 = lo codes counted up from wlo, w1 = hi codes counted down from whi
      word = w2;
      lo0 = __fmaf_rd(eq10_f(w0, 0), a.frame[6], a.frame[0]);
      lo1 = __fmaf_rd(eq10_f(w0, 1), a.frame[7], a.frame[1]);
      lo2 = __fmaf_rd(eq10_f(w0, 2), a.frame[8], a.frame[2]);
      hi0 = __fmaf_ru(-eq10_f(w1, 0), a.frame[6], a.frame[3]);
      hi1 = __fmaf_ru(-eq10_f(w1, 1), a.frame[7], a.frame[4]);
      hi2 = __fmaf_ru(-eq10_f(w1, 2), a.frame[8], a.frame[5]);
    }
    n = qbin_count(word);
    axis = qbin_axis(word);
    field = n > 0 ? qbin_first(word) : qbin_field(word);
  }
  const float tlim = ANY ? r.tmax : fminf(r.tmax, L.b.t);
  float tn;
  if (slab(r, lo0, lo1, lo2, hi0, hi1, hi2, tlim, tn)) {
    const uint32_t ref = field;
    if (n > 0) {
      if (visit_leaf<ANY, STATS>(a, r, ref, n, L.b, cnt)) {
        L.found = true;
        L.cur = kEmptyRef;
        return;
      }
    } else {
      const uint32_t l = CREF == REF_DIRECT ? cur + 1 : ref;
      const uint32_t rr = CREF == REF_DIRECT ? cur + ref : ref + 1;
      const bool neg = axis == 0 ? r.nx : (axis == 1 ? r.ny : r.nz);
      const bool swap = !ANY && a.ordered && neg;
      if (!st.push(swap ? l : rr, 0.0f)) { L.err = kErrStack; L.cur = kEmptyRef; return; }
      L.cur = swap ? rr : l;
      return;
    }
  }
  L.cur = !st.empty() ? st.pop().x : kEmptyRef;
}

// Shared-slab binary node (Section 8.3): the node's box is not stored; the
// lane carries the ray interval of the current node's box, and a child's
// interval is that interval clipped by the one plane the child moves (slo:
// the left child's upper bound on the split axis, shi: the right child's
// lower bound), widened like every slab distance. Stacked entries keep their
// interval.
template <bool ANY, class S>
__device__ __forceinline__ void slab_pop(Lane &L, S &st) {
  while (!st.empty()) {
    const uint2 e = st.pop();
    const float tn = __uint_as_float(e.y);
    if (ANY || tn <= L.b.t) {
      L.cur = e.x;
      L.ctn = tn;
      L.ctf = st.ptf;
      return;
    }
  }
  L.cur = kEmptyRef;
}

template <int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void step_slab(const TraceArgs &a, Lane &L, S &st, Counts &cnt) {
  const Ray &r = L.r;
  const uint32_t cur = L.cur;
  if (STATS) cnt.nodes++;
  const uint4 v = ldg4(a.nodes + cur);
  const uint32_t n = bin_meta_count(v.w);
  if (n > 0) {
    if (visit_leaf<ANY, STATS>(a, r, v.z, n, L.b, cnt)) {
      L.found = true;
      L.cur = kEmptyRef;
      return;
    }
    slab_pop<ANY>(L, st);
    return;
  }
  const uint32_t ax = bin_meta_axis(v.w);
  const float rd = ax == 0 ? r.rx : (ax == 1 ? r.ry : r.rz);
  const float od = ax == 0 ? r.orx : (ax == 1 ? r.ory : r.orz);
  const bool neg = ax == 0 ? r.nx : (ax == 1 ? r.ny : r.nz);
  const float tlo = fmaf(__uint_as_float(v.x), rd, -od), thi = fmaf(__uint_as_float(v.y), rd, -od);
  const float tf = fminf(L.ctf, ANY ? r.tmax : fminf(r.tmax, L.b.t));
  float ln = L.ctn, lf = tf, rn = L.ctn, rf = tf;
  if (!neg) {
    lf = fminf(lf, tlo * kFarScale);   // left: coordinate <= slo, reached before tlo
    rn = fmaxf(rn, thi * kNearScale);  // right: coordinate >= shi, reached after thi
  } else {
    ln = fmaxf(ln, tlo * kNearScale);
    rf = fminf(rf, thi * kFarScale);
  }
  const bool hl = ln <= lf, hr = rn <= rf;
  const uint32_t l = CREF == REF_DIRECT ? cur + 1 : v.z, rc = CREF == REF_DIRECT ? cur + v.z : v.z + 1;
  if (hl && hr) {
    const bool right_first = !ANY && a.ordered && rn < ln;
    const bool ok = right_first ? st.push(l, ln, lf) : st.push(rc, rn, rf);
    if (!ok) { L.err = kErrStack; L.cur = kEmptyRef; return; }
    L.cur = right_first ? rc : l;
    L.ctn = right_first ? rn : ln;
    L.ctf = right_first ? rf : lf;
  } else if (hl) {
    L.cur = l; L.ctn = ln; L.ctf = lf;
  } else if (hr) {
    L.cur = rc; L.ctn = rn; L.ctf = rf;
  } else {
    slab_pop<ANY>(L, st);
  }
}

// First entry of a ray: the root (own-box and wide nodes), or for the
// shared-slab layout the root with the ray interval of the frame box.
template <bool OWN, int PREC>
__device__ __forceinline__ void start_ray(const TraceArgs &a, Lane &L) {
  if constexpr (OWN && PREC == PREC_SLAB) {
    float tn, tf;
    const bool in = a.n_nodes > 0 && slab_interval(L.r, a.frame[0], a.frame[1], a.frame[2], a.frame[3], a.frame[4],
                                                   a.frame[5], L.r.tmax, tn, tf);
    L.cur = in ? 0u : kEmptyRef;
    L.ctn = tn;
    L.ctf = tf;
  } else if constexpr (OWN) {
    L.cur = a.n_nodes > 0 ? 0u : kEmptyRef;
  } else {
    L.cur = a.root_ref;
  }
}

// The ring pays for its extra register where the kernel has room: the own-box
// bvh2 kernels (all but the shared slab) and the kernels of 2/4-wide nodes; the
// 8-wide kernels measured slower with it.
template <bool OWN, int PREC, int W, bool ANY, int REG>
using StackFor = StackT<OWN && PREC == PREC_SLAB, (OWN && PREC != PREC_SLAB) || (!OWN && W <= 4), REG>;

// ------------------------------------------------------------------ kernel body
// Trace one ray to completion with the layout's step function.
template <bool OWN, int W, int PREC, int SOA, int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void step_any_layout(const TraceArgs &a, Lane &L, S &st, Counts &cnt) {
  if constexpr (OWN && PREC == PREC_SLAB) step_slab<CREF, ANY, STATS>(a, L, st, cnt);
  else if constexpr (OWN) step_bin<PREC, SOA, CREF, ANY, STATS>(a, L, st, cnt);
  else step_wide<W, PREC, SOA, CREF, ANY, STATS>(a, L, st, cnt);
}

template <bool OWN, int W, int PREC, int SOA, int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void trace_lane(const TraceArgs &a, Lane &L, S &st, Counts &cnt) {
  while (L.cur != kEmptyRef) {
    if (++L.steps > a.max_steps) {
      L.err = kErrIter;
      L.cur = kEmptyRef;
      break;
    }
    step_any_layout<OWN, W, PREC, SOA, CREF, ANY, STATS>(a, L, st, cnt);
  }
}

// Persistent warps: each warp takes 32 consecutive rays with one atomicAdd on
// the global counter, every lane traces one of them to completion, repeat.
template <bool OWN, int W, int PREC, int SOA, int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void body_warp_batch(const TraceArgs &a, S &st) {
  Counts cnt;
  uint32_t n_rays = 0;
  const uint32_t lane = threadIdx.x & 31u;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.work, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= a.n_work) break;
    unsigned long long rid = base + lane;
    if (a.raster_w) {
      // slot batch t is the 8x4 pixel tile (t mod tiles_x, t / tiles_x)
      const unsigned long long t = base >> 5, tiles_x = (a.raster_w + 7ull) >> 3;  // 64-bit: no wrap near 2^32
      const unsigned long long px = (t % tiles_x) * 8u + (lane & 7u), py = (t / tiles_x) * 4u + (lane >> 3);
      rid = px < a.raster_w ? py * a.raster_w + px : a.n;
    }
    if (rid >= a.n) continue;
    Lane L;
    L.rid = rid;
    setup_ray(ldg4f(a.rays + 2 * rid), ldg4f(a.rays + 2 * rid + 1), L.r);
    L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_MISS};
    L.steps = 0;
    L.err = 0;
    L.found = false;
    st.reset();
    start_ray<OWN, PREC>(a, L);
    if (STATS) n_rays++;
    trace_lane<OWN, W, PREC, SOA, CREF, ANY, STATS>(a, L, st, cnt);
    if (L.err) atomicCAS(a.status, 0u, L.err);
    if (ANY) {
      static_cast<uint32_t *>(a.out)[rid] = L.err ? SCION_PRIM_ERROR : (L.found ? 1u : 0u);
    } else {
      if (L.err) L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_ERROR};
      static_cast<uint4 *>(a.out)[rid] =
          make_uint4(__float_as_uint(L.b.t), __float_as_uint(L.b.u), __float_as_uint(L.b.v), L.b.id);
    }
  }
  if (STATS) {
    atomicAdd(a.stats + 0, (unsigned long long)cnt.nodes);
    atomicAdd(a.stats + 1, (unsigned long long)cnt.leaves);
    atomicAdd(a.stats + 2, (unsigned long long)cnt.prims);
    atomicAdd(a.stats + 3, (unsigned long long)n_rays);
  }
  // the last CTA to finish resets the counters for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(a.exit_count, 1u);
    if (prev == gridDim.x - 1) {
      *a.work = 0ull;
      *a.exit_count = 0u;
      __threadfence();
    }
  }
}

// Refilled warps. The rays are cut into 32-ray blocks dealt to the CTAs
// round-robin (CTA c owns blocks c, c + G, c + 2G, ... for a grid of G CTAs),
// so every CTA sees a spatially uniform share and no global atomic is needed.
// A lane whose ray is finished idles until at least `refill_min` lanes of its
// warp are idle; then the warp takes that many consecutive rays of its CTA's
// share with one shared-memory atomicAdd and the idle lanes set them up
// together (refill_min = 1: a lane is refilled at the next step).
template <bool OWN, int W, int PREC, int SOA, int CREF, bool ANY, bool STATS, class S>
__device__ __forceinline__ void body_refill(const TraceArgs &a, S &st) {
  __shared__ uint32_t cta_next;
  if (threadIdx.x == 0) cta_next = 0;
  __syncthreads();
  Counts cnt;
  uint32_t n_rays = 0;
  const unsigned long long G = gridDim.x, c = blockIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t below = (1u << lane) - 1u;  // lanes ranked before this one
  Lane L;
  L.cur = kEmptyRef;
  bool has_ray = false, exhausted = false;  // exhausted: warp-uniform
  while (true) {
    const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !has_ray);
    const uint32_t k = __popc(idle);
    if (!exhausted && k >= a.refill_min) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&cta_next, k);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      // ray ids grow with the index, so the last index decides exhaustion
      const uint32_t jl = base + k - 1u;
      exhausted = (c + (unsigned long long)(jl >> 5) * G) * 32ull + (jl & 31u) >= a.n;
      if (!has_ray) {
        const uint32_t j = base + __popc(idle & below);
        const unsigned long long rid = (c + (unsigned long long)(j >> 5) * G) * 32ull + (j & 31u);
        if (rid < a.n) {
          L.rid = rid;
          setup_ray(ldg4f(a.rays + 2 * rid), ldg4f(a.rays + 2 * rid + 1), L.r);
          L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_MISS};
          L.steps = 0;
          L.err = 0;
          L.found = false;
          st.reset();
          start_ray<OWN, PREC>(a, L);
          has_ray = true;
          if (STATS) n_rays++;
        }
      }
    }
    if (__ballot_sync(0xFFFFFFFFu, has_ray) == 0u) {
      if (exhausted) break;
      continue;
    }
    if (has_ray && L.cur != kEmptyRef) {
      if (++L.steps > a.max_steps) {
        L.err = kErrIter;
        L.cur = kEmptyRef;
      } else {
        step_any_layout<OWN, W, PREC, SOA, CREF, ANY, STATS>(a, L, st, cnt);
      }
    }
    if (has_ray && L.cur == kEmptyRef) {
      if (L.err) atomicCAS(a.status, 0u, L.err);
      if (ANY) {
        static_cast<uint32_t *>(a.out)[L.rid] = L.err ? SCION_PRIM_ERROR : (L.found ? 1u : 0u);
      } else {
        if (L.err) L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_ERROR};
        static_cast<uint4 *>(a.out)[L.rid] =
            make_uint4(__float_as_uint(L.b.t), __float_as_uint(L.b.u), __float_as_uint(L.b.v), L.b.id);
      }
      has_ray = false;
    }
  }
  if (STATS) {
    atomicAdd(a.stats + 0, (unsigned long long)cnt.nodes);
    atomicAdd(a.stats + 1, (unsigned long long)cnt.leaves);
    atomicAdd(a.stats + 2, (unsigned long long)cnt.prims);
    atomicAdd(a.stats + 3, (unsigned long long)n_rays);
  }
}


// REG: register entries at the top of the stack (0, 2 or 4).
template <bool OWN, int W, int PREC, int SOA, int CREF, bool ANY, bool STATS, int REG = 0>
__device__ __forceinline__ void trace_kernel_body(const TraceArgs &a) {
  extern __shared__ uint2 smem_stack[];
  StackFor<OWN, PREC, W, ANY, REG> st;
  StackTail<decltype(st)::kTF> tail;
  st.attach(tail);
  st.sh = smem_stack + threadIdx.x;
  // exit distances (shared-slab layout) follow the entry columns
  st.shf = reinterpret_cast<float *>(smem_stack + blockDim.x * a.smem_stack) + threadIdx.x;
  st.stride = blockDim.x;
  st.cap_sh = (int)a.smem_stack;
  st.reset();
  if (a.refill_min) body_refill<OWN, W, PREC, SOA, CREF, ANY, STATS>(a, st);
  else body_warp_batch<OWN, W, PREC, SOA, CREF, ANY, STATS>(a, st);
}

}  // namespace scion
