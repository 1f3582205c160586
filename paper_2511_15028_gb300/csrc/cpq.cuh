// Closest point query on the same layouts (App. G "Closest Point Query").
//
// For a point p and a squared search radius r2, the result is the
// lexicographic minimum of (d2, id) over triangles with d2 <= r2, where d2 is
// the squared distance from p to the closest point on the triangle computed
// by the Voronoi-region method of Ericson, Real-Time Collision Detection
// (2005), Section 5.1.5, in float with a fixed order of roundings:
//   dot(x, y) = (x0*y0 + x1*y1) + x2*y2; ab = b - a, ac = c - a, ap = p - a;
//   d1 = dot(ab, ap), d2 = dot(ac, ap) -> vertex a if d1 <= 0 && d2 <= 0;
//   bp = p - b, d3 = dot(ab, bp), d4 = dot(ac, bp) -> vertex b if d3 >= 0 && d4 <= d3;
//   vc = d1*d4 - d3*d2 -> edge ab if vc <= 0 && d1 >= 0 && d3 <= 0, s = d1/(d1-d3);
//   cp = p - c, d5 = dot(ab, cp), d6 = dot(ac, cp) -> vertex c if d6 >= 0 && d5 <= d6;
//   vb = d5*d2 - d1*d6 -> edge ac if vb <= 0 && d2 >= 0 && d6 <= 0, s = d2/(d2-d6);
//   va = d3*d6 - d5*d4 -> edge bc if va <= 0 && d4-d3 >= 0 && d5-d6 >= 0,
//     s = (d4-d3)/((d4-d3)+(d5-d6)), q = b + s*(c-b);
//   else face: r = 1/((va+vb)+vc), v = vb*r, w = vc*r, clamped to >= 0 and
//     divided by v+w when that exceeds 1, q = (a + ab*v) + ac*w;
//   d2 = dot(p-q, p-q).
// The clamp keeps q inside the triangle when rounding makes the region tests
// disagree, so q lies inside every (padded, outward-rounded) box on the path
// to the triangle. The box bound is therefore safe: per axis the gap to the
// box and its square are rounded toward -inf, summed toward -inf, and scaled
// by (1 - 2^-20), which covers the rounding of the subtraction p - q and of
// the dot product (at most 5 units of 2^-24 relative); a box is entered iff
// that bound <= min(best d2, r2). The paper's "distmax" bound update is not
// used: it does not bound the distance to the nearest triangle for boxes
// that are not tight.
#pragma once

#include "trace.cuh"

namespace scion {

constexpr float kLbScale = 1.0f - 9.5367431640625e-07f;  // 1 - 2^-20

struct CpBest {
  float d2, u, v;
  uint32_t id;
};

struct CpLane {
  float px, py, pz, r2;
  CpBest b;
  uint32_t cur;
  uint32_t steps;
  uint32_t err;
  unsigned long long rid;
};

__device__ __forceinline__ float cp_dot(float x0, float x1, float x2, float y0, float y1, float y2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(x0, y0), __fmul_rn(x1, y1)), __fmul_rn(x2, y2));
}

// squared distance to the pinned closest point on triangle (a, b, c); (u, v)
// are the weights of b and c
__device__ __forceinline__ float cp_triangle(float px, float py, float pz, float4 A, float4 B, float4 C,
                                             float &u, float &v) {
  const float abx = __fsub_rn(B.x, A.x), aby = __fsub_rn(B.y, A.y), abz = __fsub_rn(B.z, A.z);
  const float acx = __fsub_rn(C.x, A.x), acy = __fsub_rn(C.y, A.y), acz = __fsub_rn(C.z, A.z);
  const float apx = __fsub_rn(px, A.x), apy = __fsub_rn(py, A.y), apz = __fsub_rn(pz, A.z);
  float qx, qy, qz;
  const float d1 = cp_dot(abx, aby, abz, apx, apy, apz), d2 = cp_dot(acx, acy, acz, apx, apy, apz);
  if (d1 <= 0.0f && d2 <= 0.0f) {
    u = 0.0f; v = 0.0f;
    qx = A.x; qy = A.y; qz = A.z;
  } else {
    const float bpx = __fsub_rn(px, B.x), bpy = __fsub_rn(py, B.y), bpz = __fsub_rn(pz, B.z);
    const float d3 = cp_dot(abx, aby, abz, bpx, bpy, bpz), d4 = cp_dot(acx, acy, acz, bpx, bpy, bpz);
    const float vc = __fsub_rn(__fmul_rn(d1, d4), __fmul_rn(d3, d2));
    if (d3 >= 0.0f && d4 <= d3) {
      u = 1.0f; v = 0.0f;
      qx = B.x; qy = B.y; qz = B.z;
    } else if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
      const float s = __fdiv_rn(d1, __fsub_rn(d1, d3));
      u = s; v = 0.0f;
      qx = __fadd_rn(A.x, __fmul_rn(s, abx));
      qy = __fadd_rn(A.y, __fmul_rn(s, aby));
      qz = __fadd_rn(A.z, __fmul_rn(s, abz));
    } else {
      const float cpx = __fsub_rn(px, C.x), cpy = __fsub_rn(py, C.y), cpz = __fsub_rn(pz, C.z);
      const float d5 = cp_dot(abx, aby, abz, cpx, cpy, cpz), d6 = cp_dot(acx, acy, acz, cpx, cpy, cpz);
      const float vb = __fsub_rn(__fmul_rn(d5, d2), __fmul_rn(d1, d6));
      const float va = __fsub_rn(__fmul_rn(d3, d6), __fmul_rn(d5, d4));
      const float e43 = __fsub_rn(d4, d3), e56 = __fsub_rn(d5, d6);
      if (d6 >= 0.0f && d5 <= d6) {
        u = 0.0f; v = 1.0f;
        qx = C.x; qy = C.y; qz = C.z;
      } else if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
        const float s = __fdiv_rn(d2, __fsub_rn(d2, d6));
        u = 0.0f; v = s;
        qx = __fadd_rn(A.x, __fmul_rn(s, acx));
        qy = __fadd_rn(A.y, __fmul_rn(s, acy));
        qz = __fadd_rn(A.z, __fmul_rn(s, acz));
      } else if (va <= 0.0f && e43 >= 0.0f && e56 >= 0.0f) {
        const float s = __fdiv_rn(e43, __fadd_rn(e43, e56));
        u = __fsub_rn(1.0f, s); v = s;
        qx = __fadd_rn(B.x, __fmul_rn(s, __fsub_rn(C.x, B.x)));
        qy = __fadd_rn(B.y, __fmul_rn(s, __fsub_rn(C.y, B.y)));
        qz = __fadd_rn(B.z, __fmul_rn(s, __fsub_rn(C.z, B.z)));
      } else {
        const float r = __fdiv_rn(1.0f, __fadd_rn(__fadd_rn(va, vb), vc));
        float fv = __fmul_rn(vb, r), fw = __fmul_rn(vc, r);
        if (!(fv >= 0.0f)) fv = 0.0f;
        if (!(fw >= 0.0f)) fw = 0.0f;
        const float sum = __fadd_rn(fv, fw);
        if (sum > 1.0f) {
          fv = __fdiv_rn(fv, sum);
          fw = __fdiv_rn(fw, sum);
        }
        u = fv; v = fw;
        qx = __fadd_rn(__fadd_rn(A.x, __fmul_rn(abx, fv)), __fmul_rn(acx, fw));
        qy = __fadd_rn(__fadd_rn(A.y, __fmul_rn(aby, fv)), __fmul_rn(acy, fw));
        qz = __fadd_rn(__fadd_rn(A.z, __fmul_rn(abz, fv)), __fmul_rn(acz, fw));
      }
    }
  }
  const float xx = __fsub_rn(px, qx), xy = __fsub_rn(py, qy), xz = __fsub_rn(pz, qz);
  return cp_dot(xx, xy, xz, xx, xy, xz);
}

// Lower bound on the squared distance from p to any point of the box (see the
// file comment); +inf for an empty box (lo > hi on an axis with infinities)
__device__ __forceinline__ float box_lower(const CpLane &L, float lox, float loy, float loz, float hix, float hiy,
                                           float hiz) {
  const float gx = fmaxf(fmaxf(__fsub_rd(lox, L.px), __fsub_rd(L.px, hix)), 0.0f);
  const float gy = fmaxf(fmaxf(__fsub_rd(loy, L.py), __fsub_rd(L.py, hiy)), 0.0f);
  const float gz = fmaxf(fmaxf(__fsub_rd(loz, L.pz), __fsub_rd(L.pz, hiz)), 0.0f);
  const float s = __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
  return __fmul_rd(s, kLbScale);
}

__device__ __forceinline__ float cp_limit(const CpLane &L) { return fminf(L.b.d2, L.r2); }

// triangles [first, first + count): keep the lexicographic minimum of (d2, id)
template <bool STATS>
__device__ __forceinline__ void cp_leaf(const TraceArgs &a, CpLane &L, uint32_t first, uint32_t count,
                                        Counts &cnt) {
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
    if (!(isfinite(p0.x) && isfinite(p0.y) && isfinite(p0.z) && isfinite(p1.x) && isfinite(p1.y) &&
          isfinite(p1.z) && isfinite(p2.x) && isfinite(p2.y) && isfinite(p2.z)))
      continue;
    float u, v;
    const float d2 = cp_triangle(L.px, L.py, L.pz, p0, p1, p2, u, v);
    if (d2 <= L.r2 && (d2 < L.b.d2 || (d2 == L.b.d2 && id < L.b.id))) L.b = CpBest{d2, u, v, id};
  }
}

// next stacked entry whose bound can still hold a closer point
__device__ __forceinline__ uint32_t cp_pop(const CpLane &L, Stack &st) {
  while (st.sp > 0) {
    const uint2 e = st.pop();
    if (__uint_as_float(e.y) <= cp_limit(L)) return e.x;
  }
  return kEmptyRef;
}

// Wide node: bound every child box, enter the nearest, stack the others
// (nearest last pushed, so popped first); a leaf entry tests its triangles.
template <int W, int PREC, int SOA, int CREF, bool STATS>
__device__ __forceinline__ void cp_step_wide(const TraceArgs &a, CpLane &L, Stack &st, Counts &cnt) {
  using N = WideNode<W, PREC, SOA, CREF>;
  const uint32_t cur = L.cur;
  if (!ref_is_interior(cur)) {
    cp_leaf<STATS>(a, L, ref_leaf_first(cur), ref_leaf_count(cur), cnt);
    L.cur = cp_pop(L, st);
    return;
  }
  if (STATS) cnt.nodes++;
  const uint4 *np = a.nodes + (size_t)ref_node(cur) * (N::kStride / 16);
  uint4 q[N::NQ];
  load_node<N::NQ>(np, q);
  float ox = 0.f, oy = 0.f, oz = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
  if (N::kGrid) {
    ox = __uint_as_float(q[0].x); oy = __uint_as_float(q[0].y); oz = __uint_as_float(q[0].z);
    sx = __uint_as_float((q[0].w & 0xFFu) << 23);
    sy = __uint_as_float(((q[0].w >> 8) & 0xFFu) << 23);
    sz = __uint_as_float(((q[0].w >> 16) & 0xFFu) << 23);
  }
  const float lim = cp_limit(L);
  uint32_t cref[W];
  float clb[W];
  uint32_t base_node = 0, base_prim = 0, leaf_acc = 0;
  if (CREF == REF_INDIRECT) {
    base_node = qword(q, N::kRefOff / 4);
    base_prim = qword(q, N::kRefOff / 4 + 1);
  }
#pragma unroll
  for (int k = 0; k < W; ++k) {
    uint32_t ref;
    if (CREF == REF_DIRECT) {
      ref = qword(q, N::kRefOff / 4 + k);
    } else {
      const uint32_t m = (qword(q, N::kRefOff / 4 + 2 + (k >> 2)) >> ((k & 3) * 8)) & 0xFFu;
      if (m == 0) ref = kEmptyRef;
      else if (m & kMetaInterior) ref = ref_interior(base_node + (m & 0x7Fu));
      else { ref = ref_leaf(base_prim + leaf_acc, m); leaf_acc += m; }
    }
    float lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (PREC == PREC_F32) {
        lo[c] = __uint_as_float(N::raw(q, k, c));
        hi[c] = __uint_as_float(N::raw(q, k, c + 3));
      } else if (PREC == PREC_F16) {
        lo[c] = __half2float(__ushort_as_half((unsigned short)N::raw(q, k, c)));
        hi[c] = __half2float(__ushort_as_half((unsigned short)N::raw(q, k, c + 3)));
      } else {
        const float o = c == 0 ? ox : (c == 1 ? oy : oz), sc = c == 0 ? sx : (c == 1 ? sy : sz);
        lo[c] = fmaf(N::code(q, k, c), sc, o);
        hi[c] = fmaf(N::code(q, k, c + 3), sc, o);
      }
    }
    const float lb = box_lower(L, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
    const bool in = ref != kEmptyRef && lb <= lim;
    cref[k] = in ? ref : kEmptyRef;
    clb[k] = in ? lb : __int_as_float(0x7f800000);
  }
  if (a.ordered == 1) sort_children<W>(clb, cref);
  else if (a.ordered == 2) {
#pragma unroll
    for (int k = W - 1; k > 0; --k) cmpx(clb, cref, k - 1, k);
  }
  uint32_t next = kEmptyRef;
  float next_lb = 0.f;
#pragma unroll
  for (int k = W - 1; k >= 0; --k) {
    if (cref[k] == kEmptyRef) continue;
    if (next != kEmptyRef && !st.push(next, next_lb)) { L.err = kErrStack; L.cur = kEmptyRef; return; }
    next = cref[k];
    next_lb = clb[k];
  }
  L.cur = next != kEmptyRef ? next : cp_pop(L, st);
}

// own box of node x of an own-box layout (every codec), and its word
template <int PREC, int SOA>
__device__ __forceinline__ void own_node(const TraceArgs &a, uint32_t x, float (&lo)[3], float (&hi)[3],
                                         uint32_t &count, uint32_t &field) {
  if (PREC == PREC_F32) {
    uint32_t ref, meta;
    if (SOA) {
      const uint2 *bp = reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(a.nodes) +
                                                        (size_t)x * a.node_stride);
      const uint2 b0 = __ldg(bp), b1 = __ldg(bp + 1), b2 = __ldg(bp + 2);
      const uint2 rm = __ldg(a.nodes2 + x);
      lo[0] = __uint_as_float(b0.x); lo[1] = __uint_as_float(b0.y); lo[2] = __uint_as_float(b1.x);
      hi[0] = __uint_as_float(b1.y); hi[1] = __uint_as_float(b2.x); hi[2] = __uint_as_float(b2.y);
      ref = rm.x; meta = rm.y;
    } else {
      uint4 q0, q1;
      ldg8(a.nodes + 2 * (size_t)x, q0, q1);
      lo[0] = __uint_as_float(q0.x); lo[1] = __uint_as_float(q0.y); lo[2] = __uint_as_float(q0.z);
      hi[0] = __uint_as_float(q0.w); hi[1] = __uint_as_float(q1.x); hi[2] = __uint_as_float(q1.y);
      ref = q1.z; meta = q1.w;
    }
    count = bin_meta_count(meta);
    field = ref;
    return;
  }
  const char *np = reinterpret_cast<const char *>(a.nodes) + (size_t)x * a.node_stride;
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
    word = SOA ? __ldg(reinterpret_cast<const uint32_t *>(a.nodes2) + x) : w3;
    lo[0] = fmaf(u16lo_f(w0), a.frame[3], a.frame[0]);
    lo[1] = fmaf(u16hi_f(w0), a.frame[4], a.frame[1]);
    lo[2] = fmaf(u16lo_f(w1), a.frame[5], a.frame[2]);
    hi[0] = fmaf(u16hi_f(w1), a.frame[3], a.frame[0]);
    hi[1] = fmaf(u16lo_f(w2), a.frame[4], a.frame[1]);
    hi[2] = fmaf(u16hi_f(w2), a.frame[5], a.frame[2]);
  } else {
    word = w2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = __fmaf_rd(eq10_f(w0, c), a.frame[6 + c], a.frame[c]);
      hi[c] = __fmaf_ru(-eq10_f(w1, c), a.frame[6 + c], a.frame[3 + c]);
    }
  }
  count = qbin_count(word);
  field = count > 0 ? qbin_first(word) : qbin_field(word);
}

// Own-box binary node: the entered node's box was bounded by its parent; a
// leaf tests its triangles, an interior node bounds both children's boxes
// (the paper's children sorting), enters the nearer and stacks the other.
template <int PREC, int SOA, int CREF, bool STATS>
__device__ __forceinline__ void cp_step_bin(const TraceArgs &a, CpLane &L, Stack &st, Counts &cnt) {
  const uint32_t cur = L.cur;
  if (STATS) cnt.nodes++;
  float lo[3], hi[3];
  uint32_t n, field;
  own_node<PREC, SOA>(a, cur, lo, hi, n, field);
  if (n > 0) {
    cp_leaf<STATS>(a, L, field, n, cnt);
    L.cur = cp_pop(L, st);
    return;
  }
  const uint32_t l = CREF == REF_DIRECT ? cur + 1 : field;
  const uint32_t r = CREF == REF_DIRECT ? cur + field : field + 1;
  float llo[3], lhi[3], rlo[3], rhi[3];
  uint32_t t0, t1;
  own_node<PREC, SOA>(a, l, llo, lhi, t0, t1);
  own_node<PREC, SOA>(a, r, rlo, rhi, t0, t1);
  const float lim = cp_limit(L);
  const float bl = box_lower(L, llo[0], llo[1], llo[2], lhi[0], lhi[1], lhi[2]);
  const float br = box_lower(L, rlo[0], rlo[1], rlo[2], rhi[0], rhi[1], rhi[2]);
  const bool inl = bl <= lim, inr = br <= lim;
  const bool right_first = a.ordered && inl && inr && br < bl;
  uint32_t first = kEmptyRef;
  if (inl && inr) {
    if (!st.push(right_first ? l : r, right_first ? bl : br)) { L.err = kErrStack; L.cur = kEmptyRef; return; }
    first = right_first ? r : l;
  } else if (inl) {
    first = l;
  } else if (inr) {
    first = r;
  }
  L.cur = first != kEmptyRef ? first : cp_pop(L, st);
}

// Persistent warps take 32 consecutive points per atomicAdd; a lane answers
// one point to completion.
template <bool OWN, int W, int PREC, int SOA, int CREF, bool STATS>
__device__ __forceinline__ void cpq_kernel_body(const TraceArgs &a) {
  extern __shared__ uint2 smem_stack[];
  Stack st;
  StackTail<false> tail;
  st.attach(tail);
  st.sh = smem_stack + threadIdx.x;
  st.stride = blockDim.x;
  st.cap_sh = (int)a.smem_stack;
  st.reset();
  Counts cnt;
  uint32_t n_pts = 0;
  const uint32_t lane = threadIdx.x & 31u;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.work, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= a.n) break;
    const unsigned long long rid = base + lane;
    if (rid >= a.n) continue;
    const float4 pt = ldg4f(a.rays + rid);
    CpLane L;
    L.rid = rid;
    L.px = pt.x; L.py = pt.y; L.pz = pt.z; L.r2 = pt.w;
    L.b = CpBest{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_MISS};
    L.steps = 0;
    L.err = 0;
    st.reset();
    // a point that is not finite, or a radius that is not >= 0, finds nothing
    const bool live = isfinite(pt.x) && isfinite(pt.y) && isfinite(pt.z) && pt.w >= 0.0f;
    if constexpr (OWN) L.cur = live && a.n_nodes > 0 ? 0u : kEmptyRef;
    else L.cur = live ? a.root_ref : kEmptyRef;
    if (STATS) n_pts++;
    while (L.cur != kEmptyRef) {
      if (++L.steps > a.max_steps) {
        L.err = kErrIter;
        L.cur = kEmptyRef;
        break;
      }
      if constexpr (OWN) cp_step_bin<PREC, SOA, CREF, STATS>(a, L, st, cnt);
      else cp_step_wide<W, PREC, SOA, CREF, STATS>(a, L, st, cnt);
    }
    if (L.err) {
      atomicCAS(a.status, 0u, L.err);
      L.b = CpBest{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_ERROR};
    }
    static_cast<uint4 *>(a.out)[rid] =
        make_uint4(__float_as_uint(L.b.d2), __float_as_uint(L.b.u), __float_as_uint(L.b.v), L.b.id);
  }
  if (STATS) {
    atomicAdd(a.stats + 0, (unsigned long long)cnt.nodes);
    atomicAdd(a.stats + 1, (unsigned long long)cnt.leaves);
    atomicAdd(a.stats + 2, (unsigned long long)cnt.prims);
    atomicAdd(a.stats + 3, (unsigned long long)n_pts);
  }
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

}  // namespace scion
