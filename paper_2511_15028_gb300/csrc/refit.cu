// Refit: new vertex positions, same tree. See refit.h.
//
// Works on the packed tree itself, so every layout refits without any host
// state: (1) the vertex table and the direct triangle copies are rewritten;
// (2) each node's parent and its number of interior children are read off
// the packed references; (3) exact boxes are computed bottom-up: a thread
// starts at every node without interior children and climbs while it is the
// last child to arrive at a node (an atomic counter; nothing waits); (4) the
// world grid of q16/eq10 is recomputed from the new root box; (5) every node
// re-encodes its box fields with the shared host/device codecs.
#include "refit.h"

#include "codec.h"

namespace scion {

namespace {

constexpr uint32_t kNoParent = 0xFFFFFFFFu;

struct Tree {
  uint8_t *nodes;
  const uint8_t *nodes2;
  float4 *prims;            // direct triangle copies (or null)
  const uint32_t *prim_ids; // indirect entries (or null)
  float4 *verts;            // float4 vertex table
  const uint32_t *tri_idx;  // u32[3] per triangle, or null for a soup
  uint32_t n_nodes, stride, own, W, prec, soa, cref, prim_indirect;
};

__device__ __forceinline__ float3 vtx(const Tree &t, uint32_t i) {
  const float4 v = t.verts[i];
  return make_float3(v.x, v.y, v.z);
}

// exact box of the leaf entries [first, first + count); triangles with a
// non-finite vertex are left out (they are never hit)
__device__ Box3 leaf_box(const Tree &t, uint32_t first, uint32_t count) {
  Box3 b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = INFINITY;
    b.hi[a] = -INFINITY;
  }
  for (uint32_t e = first; e < first + count; ++e) {
    const uint32_t id = t.prim_indirect ? t.prim_ids[e] : __float_as_uint(t.prims[3 * (size_t)e].w);
    const uint32_t i0 = t.tri_idx ? t.tri_idx[3 * (size_t)id] : 3 * id;
    const uint32_t i1 = t.tri_idx ? t.tri_idx[3 * (size_t)id + 1] : 3 * id + 1;
    const uint32_t i2 = t.tri_idx ? t.tri_idx[3 * (size_t)id + 2] : 3 * id + 2;
    const float3 p[3] = {vtx(t, i0), vtx(t, i1), vtx(t, i2)};
    bool finite = true;
    for (int k = 0; k < 3; ++k) finite &= isfinite(p[k].x) && isfinite(p[k].y) && isfinite(p[k].z);
    if (!finite) continue;
    for (int k = 0; k < 3; ++k) {
      b.lo[0] = fminf(b.lo[0], p[k].x); b.hi[0] = fmaxf(b.hi[0], p[k].x);
      b.lo[1] = fminf(b.lo[1], p[k].y); b.hi[1] = fmaxf(b.hi[1], p[k].y);
      b.lo[2] = fminf(b.lo[2], p[k].z); b.hi[2] = fmaxf(b.hi[2], p[k].z);
    }
  }
  return b;
}

__device__ __forceinline__ void grow(Box3 &b, const Box3 &c) {
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = fminf(b.lo[a], c.lo[a]);
    b.hi[a] = fmaxf(b.hi[a], c.hi[a]);
  }
}

__device__ __forceinline__ Box3 load_box(const Box3 *boxes, uint32_t i) {
  const float *f = reinterpret_cast<const float *>(boxes + i);
  Box3 b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = __ldcg(f + a);
    b.hi[a] = __ldcg(f + 3 + a);
  }
  return b;
}

// One child slot of a node: kind 0 empty, 1 interior (node), 2 leaf (first, count).
struct Slot {
  int kind;
  uint32_t node, first, count;
};

// the node's children in slot order (own-box: 2 interior children or 1 leaf);
// returns the number of non-empty slots
__device__ int node_slots(const Tree &t, uint32_t x, Slot *s) {
  for (int k = 0; k < 8; ++k) s[k] = Slot{0, 0, 0, 0};
  const uint8_t *p = t.nodes + (size_t)x * t.stride;
  if (t.own) {
    uint32_t cnt, field;
    if (t.prec == PREC_SLAB) {
      field = get_u32(p + 8);
      cnt = bin_meta_count(get_u32(p + 12));
    } else if (t.prec == PREC_F32) {
      const uint8_t *q = t.soa ? t.nodes2 + (size_t)x * kBinRefBytes : p + 24;
      field = get_u32(q);
      cnt = bin_meta_count(get_u32(q + 4));
    } else {
      const uint32_t w = get_u32(t.prec == PREC_Q16 ? (t.soa ? t.nodes2 + (size_t)x * 4 : p + 12) : p + 8);
      cnt = qbin_count(w);
      field = cnt > 0 ? qbin_first(w) : qbin_field(w);
    }
    if (cnt > 0) {
      s[0] = Slot{2, 0, field, cnt};
      return 1;
    }
    const uint32_t l = t.cref == REF_DIRECT ? x + 1 : field, r = t.cref == REF_DIRECT ? x + field : field + 1;
    s[0] = Slot{1, l, 0, 0};
    s[1] = Slot{1, r, 0, 0};
    return 2;
  }
  const uint32_t ref_off = wide_ref_offset(t.W, t.prec);
  int n = 0;
  uint32_t leaf_acc = 0;
  for (uint32_t k = 0; k < t.W; ++k) {
    Slot c{0, 0, 0, 0};
    if (t.cref == REF_DIRECT) {
      const uint32_t r = get_u32(p + ref_off + 4 * k);
      if (r != kEmptyRef) c = ref_is_interior(r) ? Slot{1, ref_node(r), 0, 0}
                                                 : Slot{2, 0, ref_leaf_first(r), ref_leaf_count(r)};
    } else {
      const uint32_t m = p[ref_off + 8 + k];
      if (m & kMetaInterior) c = Slot{1, get_u32(p + ref_off) + (m & 0x7Fu), 0, 0};
      else if (m) {
        c = Slot{2, 0, get_u32(p + ref_off + 4) + leaf_acc, m};
        leaf_acc += m;
      }
    }
    s[k] = c;
    if (c.kind) ++n;
  }
  return n;
}

__global__ void update_vertices_kernel(Tree t, const float *__restrict__ v, uint64_t n_verts) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_verts; i += (uint64_t)gridDim.x * blockDim.x)
    t.verts[i] = make_float4(v[3 * i], v[3 * i + 1], v[3 * i + 2], 0.f);
}

__global__ void update_prims_kernel(Tree t, uint32_t n_entries) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_entries; e += gridDim.x * blockDim.x) {
    float4 *q = t.prims + 3 * (size_t)e;
    const uint32_t id = __float_as_uint(q[0].w);
    const uint32_t i0 = t.tri_idx ? t.tri_idx[3 * (size_t)id] : 3 * id;
    const uint32_t i1 = t.tri_idx ? t.tri_idx[3 * (size_t)id + 1] : 3 * id + 1;
    const uint32_t i2 = t.tri_idx ? t.tri_idx[3 * (size_t)id + 2] : 3 * id + 2;
    const float4 a = t.verts[i0], b = t.verts[i1], c = t.verts[i2];
    q[0] = make_float4(a.x, a.y, a.z, __uint_as_float(id));
    q[1] = make_float4(b.x, b.y, b.z, 0.f);
    q[2] = make_float4(c.x, c.y, c.z, 0.f);
  }
}

// parent of every interior child and the number of interior children
__global__ void links_kernel(Tree t, uint32_t *parent, uint32_t *pending) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < t.n_nodes; x += gridDim.x * blockDim.x) {
    Slot s[8];
    node_slots(t, x, s);
    uint32_t c = 0;
    for (int k = 0; k < 8; ++k)
      if (s[k].kind == 1) {
        parent[s[k].node] = x;
        ++c;
      }
    pending[x] = c;
  }
}

__device__ Box3 node_box(const Tree &t, uint32_t x, const Box3 *boxes) {
  Slot s[8];
  node_slots(t, x, s);
  Box3 b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = INFINITY;
    b.hi[a] = -INFINITY;
  }
  for (int k = 0; k < 8; ++k) {
    if (s[k].kind == 1) grow(b, load_box(boxes, s[k].node));
    else if (s[k].kind == 2) grow(b, leaf_box(t, s[k].first, s[k].count));
  }
  return b;
}

__global__ void boxes_kernel(Tree t, const uint32_t *parent, uint32_t *pending, Box3 *boxes) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < t.n_nodes; x += gridDim.x * blockDim.x) {
    Slot s[8];
    node_slots(t, x, s);
    bool starts = true;  // no interior child: decided from the node, not from the counters
    for (int k = 0; k < 8; ++k) starts &= s[k].kind != 1;
    if (!starts) continue;
    uint32_t y = x;
    while (true) {
      boxes[y] = node_box(t, y, boxes);
      const uint32_t p = parent[y];
      if (p == kNoParent) break;
      __threadfence();
      if (atomicSub(pending + p, 1u) != 1u) break;  // not the last child of p
      y = p;
    }
  }
}

__global__ void frame_kernel(Tree t, const Box3 *boxes, float *frame) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  Box3 r = load_box(boxes, 0);
  if (box_is_empty(r))
    for (int a = 0; a < 3; ++a) r.lo[a] = r.hi[a] = 0.0f;
  const Box3 pr = padded(r);
  if (t.prec == PREC_SLAB) {  // the root's carried box
    for (int a = 0; a < 3; ++a) {
      frame[a] = pr.lo[a];
      frame[3 + a] = pr.hi[a];
    }
    return;
  }
  float bins_inv[3];
  world_frame(t.prec, pr, frame, bins_inv);
  for (int a = 0; a < 3; ++a) frame[9 + a] = bins_inv[a];
}

__global__ void encode_kernel(Tree t, const Box3 *boxes, const float *frame, uint32_t *status) {
  float fr[12];
  for (int k = 0; k < 12; ++k) fr[k] = frame ? frame[k] : 0.f;
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < t.n_nodes; x += gridDim.x * blockDim.x) {
    uint8_t *p = t.nodes + (size_t)x * t.stride;
    bool ok = true;
    if (t.own && t.prec == PREC_SLAB) {
      Slot s[8];
      node_slots(t, x, s);
      if (s[0].kind == 1)
        encode_slab_planes(load_box(boxes, s[0].node), load_box(boxes, s[1].node), bin_meta_axis(get_u32(p + 12)), p);
    } else if (t.own) {
      ok = encode_own_box(t.prec, load_box(boxes, x), fr, fr + 9, p);
    } else {
      Slot s[8];
      Box3 cb[8];
      node_slots(t, x, s);
      uint32_t n = 0;  // the packer fills slots from 0; empty slots follow
      for (int k = 0; k < 8; ++k)
        if (s[k].kind) cb[n++] = s[k].kind == 1 ? load_box(boxes, s[k].node) : leaf_box(t, s[k].first, s[k].count);
      ok = encode_wide_boxes(t.W, t.prec, t.soa, cb, n, p) == 0;
    }
    if (!ok) atomicCAS(status, 0u, (uint32_t)SCION_ERR_BAD_INPUT);
  }
}

int grid_for(uint64_t n) {
  return (int)(n == 0 ? 1 : (n + 255) / 256 < 152ull * 16 ? (n + 255) / 256 : 152ull * 16);
}

}  // namespace

cudaError_t refit_launch(const RefitBuffers &b, const float *d_new_verts, cudaStream_t s) {
  Tree t;
  t.nodes = static_cast<uint8_t *>(b.nodes);
  t.nodes2 = static_cast<const uint8_t *>(b.nodes2);
  t.prims = static_cast<float4 *>(b.prims);
  t.prim_ids = b.prim_ids;
  t.verts = static_cast<float4 *>(b.verts4);
  t.tri_idx = b.tri_idx;
  t.n_nodes = b.n_nodes;
  t.stride = b.node_stride;
  t.own = b.own_box;
  t.W = b.desc.width;
  t.prec = b.desc.box_prec;
  t.soa = b.desc.box_layout;
  t.cref = b.desc.child_ref;
  t.prim_indirect = b.desc.prim_ref;
  update_vertices_kernel<<<grid_for(b.n_verts), 256, 0, s>>>(t, d_new_verts, b.n_verts);
  if (!t.prim_indirect && b.n_leaf_entries)
    update_prims_kernel<<<grid_for(b.n_leaf_entries), 256, 0, s>>>(t, b.n_leaf_entries);
  if (b.n_nodes == 0) return cudaGetLastError();
  cudaError_t e = cudaMemsetAsync(b.parent, 0xFF, (size_t)b.n_nodes * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  links_kernel<<<grid_for(b.n_nodes), 256, 0, s>>>(t, b.parent, b.pending);
  boxes_kernel<<<grid_for(b.n_nodes), 256, 0, s>>>(t, b.parent, b.pending, reinterpret_cast<Box3 *>(b.boxes));
  const bool grid = prec_has_frame(t.prec);
  if (grid) frame_kernel<<<1, 32, 0, s>>>(t, reinterpret_cast<const Box3 *>(b.boxes), b.frame);
  encode_kernel<<<grid_for(b.n_nodes), 256, 0, s>>>(t, reinterpret_cast<const Box3 *>(b.boxes),
                                                    grid ? b.frame : nullptr, b.status);
  return cudaGetLastError();
}

}  // namespace scion
