// Packing on the GPU. See gpack.h.
//
// The physical tree is built level by level from the root: a level's nodes
// (in breadth-first order) each find their children (the own-box node: the
// logical node's two children; the wide node: the greedy collapse that opens
// the interior child of largest surface area until W children, exactly as
// the host packer), an exclusive scan of their interior-child counts places
// the next level, so the numbering is the breadth-first order of the host
// packer. Subtree sizes bottom-up then give the depth-first positions (with
// sibling groups kept contiguous for indirect child references), an
// exclusive scan of the leaf-entry counts in physical order gives every
// node's first leaf entry, and one thread per node writes it with the shared
// host/device codecs. The host only sequences the levels (one 4-byte read
// per level).
#include "gpack.h"

#include <algorithm>
#include <vector>

namespace scion {

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;

int grid_for(uint64_t n) {
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + kThreads - 1) / kThreads, 152ull * 32));
}

// ------------------------------------------------------------ scan
// Exclusive prefix sum of the block's per-thread values (blockDim.x <= 1024);
// *total receives the block sum.
__device__ uint32_t block_scan(uint32_t x, uint32_t *warp_sums, uint32_t *total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  const uint32_t nw = blockDim.x >> 5;
  if (warp == 0) {
    const uint32_t s = lane < nw ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, si, o);
      if (lane >= (uint32_t)o) si += y;
    }
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == nw - 1) warp_sums[32] = si;
  }
  __syncthreads();
  const uint32_t r = warp_sums[warp] + inc - x;
  *total = warp_sums[32];
  __syncthreads();
  return r;
}

// sum of each kScanTile-element tile
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *__restrict__ in, uint64_t m,
                                                                    uint32_t *tile_sums) {
  __shared__ uint32_t ws[33];
  const uint64_t b = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (b + k < m) s += in[b + k];
  uint32_t total;
  block_scan(s, ws, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// exclusive scan of the tile sums in place (one block, any count); the grand
// total goes to *total
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(uint32_t *tile_sums, uint32_t n, uint32_t *total) {
  __shared__ uint32_t ws[33];
  uint32_t carry = 0;
  for (uint32_t base = 0; base < n; base += kScanThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t x = i < n ? tile_sums[i] : 0u;
    uint32_t sum;
    const uint32_t r = block_scan(x, ws, &sum);
    if (i < n) tile_sums[i] = carry + r;
    carry += sum;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *__restrict__ in, uint32_t *out,
                                                                   uint64_t m, const uint32_t *__restrict__ tile_sums) {
  __shared__ uint32_t ws[33];
  const uint64_t b = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = b + k < m ? in[b + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = tile_sums[blockIdx.x] + block_scan(s, ws, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (b + k < m) {
      out[b + k] = run;
      run += v[k];
    }
}

// out[0..m) = exclusive prefix sums of in[0..m) (in == out allowed); *total
// (device) = sum. tiles: scratch of at least ceil(m / kScanTile) words.
cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, uint64_t m, uint32_t *tiles, uint32_t *total,
                           cudaStream_t s) {
  if (m == 0) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
  const uint32_t nt = (uint32_t)((m + kScanTile - 1) / kScanTile);
  scan_reduce_kernel<<<nt, kScanThreads, 0, s>>>(in, m, tiles);
  scan_tiles_kernel<<<1, kScanThreads, 0, s>>>(tiles, nt, total);
  scan_apply_kernel<<<nt, kScanThreads, 0, s>>>(in, out, m, tiles);
  return cudaGetLastError();
}

// ------------------------------------------------------------ the device tree
struct DTree {
  uint32_t nv;
  const uint32_t *ids, *left, *right, *rlo, *rhi;
  const uint8_t *axis, *whole;
  const float *nlo, *nhi;
};

// a logical leaf: a radix leaf, or a subtree kept as one leaf
__device__ __forceinline__ bool lleaf(const DTree &t, uint32_t x) { return x + 1 >= t.nv || t.whole[x]; }

__device__ __forceinline__ void leaf_range(const DTree &t, uint32_t x, uint32_t &first, uint32_t &count) {
  if (x + 1 >= t.nv) {
    first = x - (t.nv - 1);
    count = 1;
  } else {
    first = t.rlo[x];
    count = t.rhi[x] - t.rlo[x] + 1;
  }
}

__device__ __forceinline__ Box3 node_box(const DTree &t, uint32_t x) {
  Box3 b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = t.nlo[3 * (size_t)x + a];
    b.hi[a] = t.nhi[3 * (size_t)x + a];
  }
  return b;
}

// surface area in double, as the host packer's collapse measures it
__device__ __forceinline__ double box_area_d(const Box3 &b) {
  const double e0 = fmax(0.0, (double)b.hi[0] - (double)b.lo[0]);
  const double e1 = fmax(0.0, (double)b.hi[1] - (double)b.lo[1]);
  const double e2 = fmax(0.0, (double)b.hi[2] - (double)b.lo[2]);
  return 2.0 * (e0 * e1 + e1 * e2 + e2 * e0);
}

// ------------------------------------------------------------ levels
// Per physical node (breadth-first index i): rad[i] = its logical node (the
// radix node the own-box node is, or the wide node's root); wide nodes also
// keep their W logical children; nk[i] = physical children; kfirst[i] =
// breadth-first index of the first of them (they are consecutive).
struct Levels {
  uint32_t *rad, *wchild, *wn, *nk, *kfirst, *cnt, *off, *tiles, *total;
};

__global__ void expand_kernel(DTree t, Levels L, uint32_t b, uint32_t m, uint32_t W, int own) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const uint32_t i = b + j, x = L.rad[i];
    uint32_t nk = 0;
    if (own) {
      nk = lleaf(t, x) ? 0u : 2u;
    } else {
      uint32_t ch[8];
      uint32_t n;
      if (lleaf(t, x)) {  // only a root can be a leaf: a one-child wide root
        n = 1;
        ch[0] = x;
      } else {
        n = 2;
        ch[0] = t.left[x];
        ch[1] = t.right[x];
        while (n < W) {
          int best = -1;
          double ba = -1.0;
          for (uint32_t k = 0; k < n; ++k)
            if (!lleaf(t, ch[k])) {
              const double a = box_area_d(node_box(t, ch[k]));
              if (a > ba) {
                ba = a;
                best = (int)k;
              }
            }
          if (best < 0) break;
          const uint32_t c = ch[best];
          for (uint32_t k = n; k > (uint32_t)best + 1; --k) ch[k] = ch[k - 1];
          ch[best] = t.left[c];
          ch[best + 1] = t.right[c];
          ++n;
        }
      }
      for (uint32_t k = 0; k < 8; ++k) L.wchild[8 * (size_t)i + k] = k < n ? ch[k] : kEmptyRef;
      L.wn[i] = n;
      for (uint32_t k = 0; k < n; ++k) nk += lleaf(t, ch[k]) ? 0u : 1u;
    }
    L.nk[i] = nk;
    L.cnt[j] = nk;
  }
}

__global__ void emit_kernel(DTree t, Levels L, uint32_t b, uint32_t m, int own) {
  const uint32_t e = b + m;  // first index of the next level
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const uint32_t i = b + j;
    const uint32_t kf = e + L.off[j];
    L.kfirst[i] = kf;
    if (L.nk[i] == 0) continue;
    if (own) {
      const uint32_t x = L.rad[i];
      L.rad[kf] = t.left[x];
      L.rad[kf + 1] = t.right[x];
    } else {
      uint32_t r = 0;
      for (uint32_t k = 0; k < L.wn[i]; ++k) {
        const uint32_t c = L.wchild[8 * (size_t)i + k];
        if (!lleaf(t, c)) L.rad[kf + r++] = c;
      }
    }
  }
}

// subtree sizes of one level (its children's are known)
__global__ void size_kernel(const Levels L, uint32_t *size, uint32_t b, uint32_t m) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const uint32_t i = b + j;
    uint32_t s = 1;
    for (uint32_t r = 0; r < L.nk[i]; ++r) s += size[L.kfirst[i] + r];
    size[i] = s;
  }
}

// depth-first positions of the children of one level's nodes: pre-order
// (group = 0), or with every node's children consecutive and each child's
// descendants after its siblings' (group = 1; base[i] = position of node i's
// first child)
__global__ void place_kernel(const Levels L, const uint32_t *size, uint32_t *pos, uint32_t *base, uint32_t b,
                             uint32_t m, int group) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const uint32_t i = b + j, kf = L.kfirst[i], nk = L.nk[i];
    if (!group) {
      uint32_t acc = pos[i] + 1;
      for (uint32_t r = 0; r < nk; ++r) {
        pos[kf + r] = acc;
        acc += size[kf + r];
      }
    } else {
      const uint32_t bi = base[i];
      uint32_t acc = bi + nk;
      for (uint32_t r = 0; r < nk; ++r) {
        pos[kf + r] = bi + r;
        base[kf + r] = acc;
        acc += size[kf + r] - 1;
      }
    }
  }
}

__global__ void iota_kernel(uint32_t *pos, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pos[i] = i;
}

// leaf entries of each physical node, indexed by physical position
__global__ void leaf_count_kernel(DTree t, const Levels L, const uint32_t *pos, uint32_t n, int own,
                                  uint32_t *lcnt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t c = 0, first, count;
    if (own) {
      if (lleaf(t, L.rad[i])) {
        leaf_range(t, L.rad[i], first, count);
        c = count;
      }
    } else {
      for (uint32_t k = 0; k < L.wn[i]; ++k) {
        const uint32_t ch = L.wchild[8 * (size_t)i + k];
        if (lleaf(t, ch)) {
          leaf_range(t, ch, first, count);
          c += count;
        }
      }
    }
    lcnt[pos[i]] = c;
  }
}

// ------------------------------------------------------------ encode
struct PrimOut {
  const float *verts;        // float[n_verts][3]
  const uint32_t *indices;   // u32[n_tris][3] or null
  float *direct;             // 12 floats per leaf entry, or null
  uint32_t *ids;             // 1 id per leaf entry, or null
};

// leaf entries [at, at + count) from the sorted triangles first.. of a leaf
__device__ void emit_prims(const DTree &t, const PrimOut &po, uint32_t first, uint32_t count, uint32_t at) {
  for (uint32_t k = 0; k < count; ++k) {
    const uint32_t id = t.ids[first + k];
    if (po.direct) {
      const uint32_t i0 = po.indices ? po.indices[3 * (size_t)id] : 3 * id;
      const uint32_t i1 = po.indices ? po.indices[3 * (size_t)id + 1] : 3 * id + 1;
      const uint32_t i2 = po.indices ? po.indices[3 * (size_t)id + 2] : 3 * id + 2;
      float4 *rec = reinterpret_cast<float4 *>(po.direct + 12 * (size_t)(at + k));
      rec[0] = make_float4(po.verts[3 * (size_t)i0], po.verts[3 * (size_t)i0 + 1], po.verts[3 * (size_t)i0 + 2],
                           __uint_as_float(id));
      rec[1] = make_float4(po.verts[3 * (size_t)i1], po.verts[3 * (size_t)i1 + 1], po.verts[3 * (size_t)i1 + 2], 0.f);
      rec[2] = make_float4(po.verts[3 * (size_t)i2], po.verts[3 * (size_t)i2 + 1], po.verts[3 * (size_t)i2 + 2], 0.f);
    } else {
      po.ids[at + k] = id;
    }
  }
}

struct OwnArgs {
  uint32_t prec, soa, cref, stride;
  float frame[9], bins_inv[3];
};

__global__ void encode_own_kernel(DTree t, const Levels L, const uint32_t *pos, const uint32_t *pbase, uint32_t n,
                                  OwnArgs oa, uint8_t *nodes, uint8_t *nodes2, PrimOut po, int *bad) {
  const bool quant = prec_is_world_grid(oa.prec);
  int badl = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t x = L.rad[i], p = pos[i];
    const bool leaf = lleaf(t, x);
    uint32_t ref, meta, count = 0, first = 0;
    if (leaf) {
      leaf_range(t, x, first, count);
      ref = pbase[p];
      meta = bin_pack_meta(count, 0);
      emit_prims(t, po, first, count, pbase[p]);
    } else {
      const uint32_t l = pos[L.kfirst[i]], r = pos[L.kfirst[i] + 1];
      if (oa.cref == REF_DIRECT) {
        badl |= l != p + 1 ? 1 : 0;
        ref = r - p;
      } else {
        badl |= r != l + 1 ? 1 : 0;
        ref = l;
      }
      meta = bin_pack_meta(0, t.axis[x]);
    }
    uint8_t *q = nodes + (size_t)p * oa.stride;
    badl |= encode_own_box(oa.prec, node_box(t, x), oa.frame, oa.bins_inv, q) ? 0 : 2;
    if (!quant) {
      uint8_t *rq = oa.soa ? nodes2 + (size_t)p * kBinRefBytes : q + 24;
      put_u32(rq, ref);
      put_u32(rq + 4, meta);
    } else {
      const uint32_t word = leaf ? qbin_leaf(ref, count) : qbin_interior(ref, t.axis[x]);
      put_u32(oa.prec == PREC_Q16 ? (oa.soa ? nodes2 + (size_t)p * 4 : q + 12) : q + 8, word);
    }
  }
  if (badl) atomicOr(bad, badl);
}

struct WideArgs {
  uint32_t W, prec, soa, cref, stride, ref_off;
};

__global__ void encode_wide_kernel(DTree t, const Levels L, const uint32_t *pos, const uint32_t *pbase, uint32_t n,
                                   WideArgs wa, uint8_t *nodes, PrimOut po, int *bad) {
  int badl = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t p = pos[i], wn = L.wn[i];
    uint8_t *q = nodes + (size_t)p * wa.stride;
    Box3 cb[8];
    uint32_t first_interior = kEmptyRef, rank = 0, at = pbase[p];
    for (uint32_t k = 0; k < wa.W; ++k) {
      uint32_t refv = kEmptyRef, meta = 0;
      if (k < wn) {
        const uint32_t c = L.wchild[8 * (size_t)i + k];
        cb[k] = node_box(t, c);
        if (!lleaf(t, c)) {
          const uint32_t cp = pos[L.kfirst[i] + rank];
          if (first_interior == kEmptyRef) first_interior = cp;
          if (wa.cref == REF_INDIRECT && cp != first_interior + rank) badl |= 1;
          refv = ref_interior(cp);
          meta = kMetaInterior | rank;
          ++rank;
        } else {
          uint32_t first, count;
          leaf_range(t, c, first, count);
          refv = ref_leaf(at, count);
          meta = count;
          emit_prims(t, po, first, count, at);
          at += count;
        }
      }
      if (wa.cref == REF_DIRECT) put_u32(q + wa.ref_off + 4 * k, refv);
      else q[wa.ref_off + 8 + k] = (uint8_t)meta;
    }
    if (wa.cref == REF_INDIRECT) {
      put_u32(q + wa.ref_off, first_interior == kEmptyRef ? 0u : first_interior);
      put_u32(q + wa.ref_off + 4, pbase[p]);
    }
    badl |= encode_wide_boxes(wa.W, wa.prec, wa.soa, cb, wn, q);
  }
  if (badl) atomicOr(bad, badl);
}

__global__ void verts4_kernel(const float *__restrict__ v, uint64_t n, float4 *out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = make_float4(v[3 * i], v[3 * i + 1], v[3 * i + 2], 0.f);
}

// device allocations of one packing; released unless kept
struct Pool {
  std::vector<void *> ptrs;
  ~Pool() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T **p, size_t count) {
    void *q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return e;
  }
  void release(void *p) { ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end()); }
};

__global__ void index_check_kernel(const uint32_t *__restrict__ ix, uint64_t n, uint64_t n_verts, int *bad) {
  int b = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    b |= ix[i] >= n_verts ? 1 : 0;
  if (__any_sync(0xFFFFFFFFu, b) && (threadIdx.x & 31u) == 0) atomicOr(bad, 1);
}

scion_status cuda_err(cudaError_t e, std::string *err) {
  *err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SCION_ERR_OOM : SCION_ERR_CUDA;
}

}  // namespace

scion_status gpu_indices_in_range(const uint32_t *d_indices, uint64_t n_tris, uint64_t n_verts, cudaStream_t s,
                                  bool *ok, std::string *err) {
  *ok = true;
  if (!d_indices || n_tris == 0) return SCION_OK;
  int *bad = nullptr;
  cudaError_t e = cudaMalloc(&bad, sizeof(int));
  if (e != cudaSuccess) return cuda_err(e, err);
  int hb = 0;
  e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    index_check_kernel<<<grid_for(3 * n_tris), kThreads, 0, s>>>(d_indices, 3 * n_tris, n_verts, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_err(e, err);
  *ok = hb == 0;
  return SCION_OK;
}

bool gpu_pack_supported(const scion_layout_desc &d, bool own_box) {
  if (d.order == ORDER_TREELET) return false;
  if (own_box && d.box_prec == PREC_SLAB) return false;
  return true;
}

scion_status gpu_pack(const LbvhTree &t, const float *d_verts, uint64_t n_verts, const uint32_t *d_indices,
                      uint64_t n_tris, const scion_layout_desc &d, bool own_box, cudaStream_t s,
                      DevicePacked *out, std::string *err) {
  *out = DevicePacked{};
  Pool pool;
  cudaError_t e;
#define SCION_GP(call)                                \
  do {                                                \
    e = (call);                                       \
    if (e != cudaSuccess) return cuda_err(e, err);    \
  } while (0)
  cudaEvent_t ev0, ev1;
  SCION_GP(cudaEventCreate(&ev0));
  SCION_GP(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  SCION_GP(cudaEventRecord(ev0, s));
  // vertex / index tables (indirect triangles and the backward pass use them)
  float4 *verts4 = nullptr;
  SCION_GP(pool.get(&verts4, n_verts));
  out->vert_bytes = n_verts * sizeof(float4);
  if (n_verts > 0) verts4_kernel<<<grid_for(n_verts), kThreads, 0, s>>>(d_verts, n_verts, verts4);
  SCION_GP(cudaGetLastError());
  uint32_t *idx = nullptr;
  if (d_indices) {
    SCION_GP(pool.get(&idx, 3 * n_tris));
    out->idx_bytes = 3 * n_tris * sizeof(uint32_t);
    SCION_GP(cudaMemcpyAsync(idx, d_indices, out->idx_bytes, cudaMemcpyDeviceToDevice, s));
  }
  const uint32_t nv = t.nv;
  const uint32_t W = d.width;
  void *nodes = nullptr, *nodes2 = nullptr, *prims = nullptr, *prim_ids = nullptr;
  if (nv > 0) {
    const DTree dt{nv, t.ids, t.left, t.right, t.rlo, t.rhi, t.axis, t.whole, t.nlo, t.nhi};
    const uint64_t cap = own_box ? 2ull * nv - 1 : std::max<uint64_t>(1, nv - 1);
    Levels L{};
    SCION_GP(pool.get(&L.rad, cap));
    SCION_GP(pool.get(&L.nk, cap));
    SCION_GP(pool.get(&L.kfirst, cap));
    SCION_GP(pool.get(&L.cnt, cap));
    SCION_GP(pool.get(&L.off, cap));
    SCION_GP(pool.get(&L.tiles, (cap + kScanTile - 1) / kScanTile));
    SCION_GP(pool.get(&L.total, 1));
    if (!own_box) {
      SCION_GP(pool.get(&L.wchild, 8 * cap));
      SCION_GP(pool.get(&L.wn, cap));
    }
    // levels, breadth first from the root (logical node 0)
    const uint32_t root = 0;
    SCION_GP(cudaMemcpyAsync(L.rad, &root, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    std::vector<uint32_t> lvl{0, 1};  // level k = [lvl[k], lvl[k+1])
    for (;;) {
      const uint32_t b = lvl[lvl.size() - 2], m = lvl.back() - b;
      expand_kernel<<<grid_for(m), kThreads, 0, s>>>(dt, L, b, m, W, own_box ? 1 : 0);
      SCION_GP(cudaGetLastError());
      SCION_GP(exclusive_scan(L.cnt, L.off, m, L.tiles, L.total, s));
      emit_kernel<<<grid_for(m), kThreads, 0, s>>>(dt, L, b, m, own_box ? 1 : 0);
      SCION_GP(cudaGetLastError());
      uint32_t next = 0;
      SCION_GP(cudaMemcpyAsync(&next, L.total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      SCION_GP(cudaStreamSynchronize(s));
      if (next == 0) break;
      if (lvl.back() + (uint64_t)next > cap) {
        *err = "GPU packer: level sizes exceed the node count";
        return SCION_ERR_CUDA;
      }
      lvl.push_back(lvl.back() + next);
    }
    const uint32_t nn = lvl.back();
    const uint32_t levels = (uint32_t)lvl.size() - 1;
    if (own_box && prec_is_world_grid(d.box_prec) && nn >= kQMaxNodes) {
      *err = "too many nodes for the quantised own-box node";
      return SCION_ERR_UNSUPPORTED_LAYOUT;
    }
    if (!own_box && nn >= kMaxNodes) {
      *err = "too many nodes";
      return SCION_ERR_INVALID_ARG;
    }
    // physical positions
    uint32_t *pos = nullptr;
    SCION_GP(pool.get(&pos, nn));
    if (d.order == ORDER_BFS) {
      iota_kernel<<<grid_for(nn), kThreads, 0, s>>>(pos, nn);
    } else {
      const int group = d.child_ref == REF_INDIRECT ? 1 : 0;
      uint32_t *size = nullptr, *base = nullptr;
      SCION_GP(pool.get(&size, nn));
      for (uint32_t k = levels; k-- > 0;)
        size_kernel<<<grid_for(lvl[k + 1] - lvl[k]), kThreads, 0, s>>>(L, size, lvl[k], lvl[k + 1] - lvl[k]);
      const uint32_t zero_one[2] = {0u, 1u};
      SCION_GP(cudaMemcpyAsync(pos, &zero_one[0], sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      if (group) {
        SCION_GP(pool.get(&base, nn));
        SCION_GP(cudaMemcpyAsync(base, &zero_one[1], sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      }
      for (uint32_t k = 0; k + 1 < levels; ++k)
        place_kernel<<<grid_for(lvl[k + 1] - lvl[k]), kThreads, 0, s>>>(L, size, pos, base, lvl[k],
                                                                        lvl[k + 1] - lvl[k], group);
      // the host values above are read by the copies before this returns
      SCION_GP(cudaStreamSynchronize(s));
    }
    SCION_GP(cudaGetLastError());
    // leaf entries: counts in physical order, prefix sums
    uint32_t *pbase = nullptr;
    SCION_GP(pool.get(&pbase, nn));
    leaf_count_kernel<<<grid_for(nn), kThreads, 0, s>>>(dt, L, pos, nn, own_box ? 1 : 0, pbase);
    SCION_GP(cudaGetLastError());
    SCION_GP(exclusive_scan(pbase, pbase, nn, L.tiles, L.total, s));
    uint32_t entries = 0;
    SCION_GP(cudaMemcpyAsync(&entries, L.total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SCION_GP(cudaStreamSynchronize(s));
    // buffers
    PrimOut po{d_verts, d_indices, nullptr, nullptr};
    if (d.prim_ref == REF_DIRECT) {
      float *pd = nullptr;
      SCION_GP(pool.get(&pd, 12 * (size_t)entries));
      po.direct = pd;
      prims = pd;
      out->prim_direct_bytes = 48ull * entries;
    } else {
      uint32_t *pi = nullptr;
      SCION_GP(pool.get(&pi, entries));
      po.ids = pi;
      prim_ids = pi;
      out->prim_id_bytes = 4ull * entries;
    }
    int *bad = nullptr;
    SCION_GP(pool.get(&bad, 1));
    SCION_GP(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (own_box) {
      OwnArgs oa{};
      oa.prec = d.box_prec;
      oa.soa = d.box_layout;
      oa.cref = d.child_ref;
      const bool soa = d.box_layout == LAYOUT_SOA, a16 = d.align == 16;
      uint32_t ref_bytes = 0;
      if (oa.prec == PREC_F32) {
        oa.stride = soa ? (a16 ? 32u : kBinBoxBytes) : kBinNodeBytes;
        ref_bytes = soa ? kBinRefBytes : 0u;
      } else if (oa.prec == PREC_Q16) {
        oa.stride = soa ? (a16 ? 16u : kQBoxBytes) : 16u;
        ref_bytes = soa ? 4u : 0u;
      } else {
        oa.stride = a16 ? 16u : kQBoxBytes;
      }
      if (prec_is_world_grid(oa.prec)) {
        // world grid over the padded root box, computed by the host codec
        float rb[6];
        SCION_GP(cudaMemcpyAsync(rb, t.nlo, 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
        SCION_GP(cudaMemcpyAsync(rb + 3, t.nhi, 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
        SCION_GP(cudaStreamSynchronize(s));
        Box3 root_box;
        for (int a = 0; a < 3; ++a) {
          root_box.lo[a] = rb[a];
          root_box.hi[a] = rb[3 + a];
        }
        world_frame(oa.prec, padded(root_box), oa.frame, oa.bins_inv);
        for (int k = 0; k < 9; ++k) out->frame[k] = oa.frame[k];
      }
      out->node_stride = oa.stride;
      out->node_bytes = (uint64_t)nn * oa.stride;
      SCION_GP(pool.get(reinterpret_cast<uint8_t **>(&nodes), out->node_bytes));
      SCION_GP(cudaMemsetAsync(nodes, 0, out->node_bytes, s));
      if (ref_bytes) {
        out->node2_bytes = (uint64_t)nn * ref_bytes;
        SCION_GP(pool.get(reinterpret_cast<uint8_t **>(&nodes2), out->node2_bytes));
        SCION_GP(cudaMemsetAsync(nodes2, 0, out->node2_bytes, s));
      }
      encode_own_kernel<<<grid_for(nn), kThreads, 0, s>>>(dt, L, pos, pbase, nn, oa, static_cast<uint8_t *>(nodes),
                                                           static_cast<uint8_t *>(nodes2), po, bad);
      out->root_ref = 0;
      out->depth = levels;
      out->stack_need = levels;
    } else {
      WideArgs wa{W, d.box_prec, d.box_layout, d.child_ref, wide_node_stride(W, d.box_prec, d.child_ref),
                  wide_ref_offset(W, d.box_prec)};
      out->node_stride = wa.stride;
      out->node_bytes = (uint64_t)nn * wa.stride;
      SCION_GP(pool.get(reinterpret_cast<uint8_t **>(&nodes), out->node_bytes));
      SCION_GP(cudaMemsetAsync(nodes, 0, out->node_bytes, s));
      encode_wide_kernel<<<grid_for(nn), kThreads, 0, s>>>(dt, L, pos, pbase, nn, wa, static_cast<uint8_t *>(nodes),
                                                            po, bad);
      out->root_ref = ref_interior(0);
      out->depth = levels;
      out->stack_need = (W - 1) * levels + 1;
    }
    SCION_GP(cudaGetLastError());
    int hbad = 0;
    SCION_GP(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCION_GP(cudaStreamSynchronize(s));
    if (hbad & 1) {
      *err = own_box ? "node order violates the child reference encoding" : "siblings not contiguous";
      return SCION_ERR_UNSUPPORTED_LAYOUT;
    }
    if (hbad & 2) {
      *err = own_box ? "world-grid enclosure" : "f16 enclosure";
      return SCION_ERR_BAD_INPUT;
    }
    if (hbad & 4) {
      *err = "u8/u16 enclosure";
      return SCION_ERR_BAD_INPUT;
    }
    out->n_nodes = nn;
    out->n_leaf_entries = entries;
  } else {
    out->root_ref = kEmptyRef;
  }
  SCION_GP(cudaEventRecord(ev1, s));
  SCION_GP(cudaStreamSynchronize(s));
  float ms = 0.f;
  SCION_GP(cudaEventElapsedTime(&ms, ev0, ev1));
  out->pack_ms = ms;
#undef SCION_GP
  // hand the result buffers to the caller
  out->nodes = nodes;
  out->nodes2 = nodes2;
  out->prims = prims;
  out->prim_ids = prim_ids;
  out->verts4 = verts4;
  out->idx = idx;
  for (void *p : {nodes, nodes2, prims, prim_ids, static_cast<void *>(verts4), static_cast<void *>(idx)})
    if (p) pool.release(p);
  return SCION_OK;
}

}  // namespace scion
