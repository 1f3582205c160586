// Linear BVH construction on the GPU. See lbvh.h.
//
// Steps, each its own kernel on the caller's stream:
//   1. triangle boxes, centroid bounds (ordered-integer atomics), valid count;
//   2. 30-bit Morton code of each centroid (10 bits per axis, x highest);
//      triangles with a non-finite vertex get the code 0xFFFFFFFF;
//   3. stable LSD radix sort of (code, triangle) pairs, 4-bit digits, 8
//      passes; each pass = per-tile digit histogram, one exclusive scan over
//      [digit][tile], and a scatter in which each tile ranks its keys with a
//      [digit][thread] counting table in shared memory (stable: a thread
//      owns 16 consecutive keys);
//   4. binary radix tree over the sorted codes, one thread per interior node
//      (Karras 2012, "Maximizing parallelism in the construction of BVHs,
//      octrees, and k-d trees"); equal codes are ordered by their position;
//   5. boxes bottom-up: a thread per leaf climbs while it is the second of
//      the two children to arrive at a node (an atomic counter per node;
//      nothing waits on another thread);
//   6. leaf choice bottom-up in the same way: a subtree of at most leaf_max
//      triangles becomes one leaf where the surface area heuristic prefers
//      it to the subtree's best split.
#include "lbvh.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

namespace scion {

namespace {

constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per sort tile
constexpr int kRadix = 16;                             // 4-bit digits
constexpr int kScanThreads = 1024;

// order-preserving float <-> u32 map (for atomicMin / atomicMax on floats)
__device__ __forceinline__ uint32_t f2o(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

// 1. boxes (lo/hi, 3 floats each per triangle; empty box when not finite),
//    centroid bounds cb[0..2] min, cb[3..5] max (ordered u32), valid count
__global__ void tri_bounds_kernel(const float *__restrict__ v, const uint32_t *__restrict__ ix, uint32_t n,
                                  float *__restrict__ tlo, float *__restrict__ thi, uint32_t *cb,
                                  uint32_t *n_valid) {
  uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0u, 0u, 0u};
  uint32_t cnt = 0;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const uint32_t i0 = ix ? ix[3 * (size_t)t] : 3 * t;
    const uint32_t i1 = ix ? ix[3 * (size_t)t + 1] : 3 * t + 1;
    const uint32_t i2 = ix ? ix[3 * (size_t)t + 2] : 3 * t + 2;
    const float *p0 = v + 3 * (size_t)i0, *p1 = v + 3 * (size_t)i1, *p2 = v + 3 * (size_t)i2;
    const bool ok = finite3(p0[0], p0[1], p0[2]) && finite3(p1[0], p1[1], p1[2]) && finite3(p2[0], p2[1], p2[2]);
    for (int a = 0; a < 3; ++a) {
      float lo = fminf(fminf(p0[a], p1[a]), p2[a]), hi = fmaxf(fmaxf(p0[a], p1[a]), p2[a]);
      if (!ok) {
        lo = __int_as_float(0x7f800000);
        hi = -__int_as_float(0x7f800000);
      } else {
        const uint32_t c = f2o((p0[a] + p1[a] + p2[a]) * (1.0f / 3.0f));
        mn[a] = min(mn[a], c);
        mx[a] = max(mx[a], c);
      }
      tlo[3 * (size_t)t + a] = lo;
      thi[3 * (size_t)t + a] = hi;
    }
    cnt += ok ? 1u : 0u;
  }
  for (int a = 0; a < 3; ++a) {
    mn[a] = __reduce_min_sync(0xFFFFFFFFu, mn[a]);
    mx[a] = __reduce_max_sync(0xFFFFFFFFu, mx[a]);
  }
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if ((threadIdx.x & 31u) == 0) {
    for (int a = 0; a < 3; ++a) {
      atomicMin(cb + a, mn[a]);
      atomicMax(cb + 3 + a, mx[a]);
    }
    atomicAdd(n_valid, cnt);
  }
}

// spread the low 10 bits of x to every third bit
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

// 2. Morton codes of the triangle centroids (same centroid as the bounds pass)
__global__ void morton_kernel(const float *__restrict__ v, const uint32_t *__restrict__ ix,
                              const float *__restrict__ tlo, const float *__restrict__ thi, uint32_t n,
                              const uint32_t *cb, uint32_t *keys, uint32_t *vals) {
  float lo[3], sc[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = o2f(cb[a]);
    const float ext = o2f(cb[3 + a]) - lo[a];
    sc[a] = ext > 0.0f ? 1024.0f / ext : 0.0f;
  }
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    uint32_t key = kInvalidKey;
    if (tlo[3 * (size_t)t] <= thi[3 * (size_t)t]) {
      const uint32_t i0 = ix ? ix[3 * (size_t)t] : 3 * t;
      const uint32_t i1 = ix ? ix[3 * (size_t)t + 1] : 3 * t + 1;
      const uint32_t i2 = ix ? ix[3 * (size_t)t + 2] : 3 * t + 2;
      uint32_t q[3];
      for (int a = 0; a < 3; ++a) {
        const float c = (v[3 * (size_t)i0 + a] + v[3 * (size_t)i1 + a] + v[3 * (size_t)i2 + a]) * (1.0f / 3.0f);
        const float f = (c - lo[a]) * sc[a];
        q[a] = f >= 1023.0f ? 1023u : (f > 0.0f ? (uint32_t)f : 0u);
      }
      key = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    }
    keys[t] = key;
    vals[t] = t;
  }
}

// 3a. digit histogram of one tile of kSortTile keys: hist[digit * tiles + tile]
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t *__restrict__ keys, int shift,
                                                                   uint32_t *hist, uint32_t tiles) {
  __shared__ uint32_t cnt[kRadix];
  if (threadIdx.x < kRadix) cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint4 *p = reinterpret_cast<const uint4 *>(keys + (size_t)blockIdx.x * kSortTile +
                                                   (size_t)threadIdx.x * kSortItems);
#pragma unroll
  for (int i = 0; i < kSortItems / 4; ++i) {
    const uint4 k = p[i];
    atomicAdd(&cnt[(k.x >> shift) & 15u], 1u);
    atomicAdd(&cnt[(k.y >> shift) & 15u], 1u);
    atomicAdd(&cnt[(k.z >> shift) & 15u], 1u);
    atomicAdd(&cnt[(k.w >> shift) & 15u], 1u);
  }
  __syncthreads();
  if (threadIdx.x < kRadix) hist[(size_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix sum of the 256 per-thread values of a block (returns the
// thread's prefix; *total receives the block sum).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sums, uint32_t *total) {
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
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
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

// 3b. exclusive scan of m values in place (one block)
__global__ void __launch_bounds__(kScanThreads) scan_kernel(uint32_t *a, uint32_t m) {
  __shared__ uint32_t warp_sums[33];
  const uint32_t per = (m + kScanThreads - 1) / kScanThreads;
  const uint32_t b = threadIdx.x * per, e = min(m, b + per);
  uint32_t s = 0;
  for (uint32_t i = b; i < e; ++i) s += a[i];
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, warp_sums, &total);
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t x = a[i];
    a[i] = run;
    run += x;
  }
}

// 3c. stable scatter of one tile
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint32_t *__restrict__ kin,
                                                                      const uint32_t *__restrict__ vin,
                                                                      uint32_t *__restrict__ kout,
                                                                      uint32_t *__restrict__ vout, int shift,
                                                                      const uint32_t *__restrict__ hist,
                                                                      uint32_t tiles) {
  __shared__ uint32_t cnt[kRadix * kSortThreads];  // [digit][thread]
  __shared__ uint32_t dstart[kRadix];
  __shared__ uint32_t warp_sums[33];
  const uint32_t t = threadIdx.x;
  const size_t base = (size_t)blockIdx.x * kSortTile + (size_t)t * kSortItems;
  uint32_t k[kSortItems], val[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems / 4; ++i) {
    const uint4 a = reinterpret_cast<const uint4 *>(kin + base)[i];
    const uint4 b = reinterpret_cast<const uint4 *>(vin + base)[i];
    k[4 * i] = a.x; k[4 * i + 1] = a.y; k[4 * i + 2] = a.z; k[4 * i + 3] = a.w;
    val[4 * i] = b.x; val[4 * i + 1] = b.y; val[4 * i + 2] = b.z; val[4 * i + 3] = b.w;
  }
#pragma unroll
  for (int d = 0; d < kRadix; ++d) cnt[d * kSortThreads + t] = 0;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) cnt[((k[i] >> shift) & 15u) * kSortThreads + t] += 1u;
  __syncthreads();
  // exclusive scan over the table in [digit][thread] order: thread t takes
  // the 16 consecutive entries t*16 .. t*16+15
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kRadix; ++i) s += cnt[t * kRadix + i];
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, warp_sums, &total);
#pragma unroll
  for (int i = 0; i < kRadix; ++i) {
    const uint32_t x = cnt[t * kRadix + i];
    cnt[t * kRadix + i] = run;
    run += x;
  }
  __syncthreads();
  if (t < kRadix) dstart[t] = cnt[t * kSortThreads];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t d = (k[i] >> shift) & 15u;
    const uint32_t p = cnt[d * kSortThreads + t]++;
    const uint32_t g = hist[(size_t)d * tiles + blockIdx.x] + (p - dstart[d]);
    kout[g] = k[i];
    vout[g] = val[i];
  }
}

// 4. radix tree (Karras 2012). Interior node i in [0, n-2]; leaf k is node
//    n-1+k. Common prefix length of keys i and j; equal keys compare their
//    positions; -1 outside [0, n).
__device__ __forceinline__ int delta(const uint32_t *keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const uint32_t a = keys[i], b = keys[j];
  if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
  return __clz(a ^ b);
}

__global__ void radix_tree_kernel(const uint32_t *__restrict__ keys, int n, uint32_t *left, uint32_t *right,
                                  uint32_t *parent, uint8_t *axis, uint32_t *range_lo, uint32_t *range_hi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n - 1; i += gridDim.x * blockDim.x) {
    const int d = delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1) >= 0 ? 1 : -1;
    const int dmin = delta(keys, n, i, i - d);
    // the other end of the range: exponential then binary search
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
      if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(keys, n, i, j);
    // split: the last position sharing more than dnode prefix bits with i
    int s = 0;
    for (int div = 2;; div <<= 1) {
      const int t = (l + div - 1) / div;
      if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
      if (t <= 1) break;
    }
    const int g = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const uint32_t lc = lo == g ? (uint32_t)(n - 1 + g) : (uint32_t)g;
    const uint32_t rc = hi == g + 1 ? (uint32_t)(n - 1 + g + 1) : (uint32_t)(g + 1);
    left[i] = lc;
    right[i] = rc;
    range_lo[i] = (uint32_t)lo;  // the node's leaves: sorted triangles lo..hi
    range_hi[i] = (uint32_t)hi;
    parent[lc] = (uint32_t)i;
    parent[rc] = (uint32_t)i;
    // split axis: the highest bit in which the range's end codes differ
    const uint32_t x = keys[lo] ^ keys[hi];
    uint8_t ax = 0;
    if (x) {
      const int bit = 31 - __clz(x);  // Morton bit 3m+2 = x, 3m+1 = y, 3m = z
      ax = (uint8_t)(bit % 3 == 2 ? 0 : (bit % 3 == 1 ? 1 : 2));
    }
    axis[i] = ax;
  }
}

// 5. boxes bottom-up
__global__ void boxes_kernel(int n, const uint32_t *__restrict__ ids, const float *__restrict__ tlo,
                             const float *__restrict__ thi, const uint32_t *__restrict__ left,
                             const uint32_t *__restrict__ right, const uint32_t *__restrict__ parent, float *nlo,
                             float *nhi, uint32_t *arrived) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t node = (uint32_t)(n - 1 + k), id = ids[k];
    for (int a = 0; a < 3; ++a) {
      nlo[3 * (size_t)node + a] = tlo[3 * (size_t)id + a];
      nhi[3 * (size_t)node + a] = thi[3 * (size_t)id + a];
    }
    uint32_t p = parent[node];
    // at most one thread continues past each interior node: the second to arrive
    while (p != kNone) {
      __threadfence();
      if (atomicAdd(arrived + p, 1u) == 0u) break;
      const uint32_t l = left[p], r = right[p];
      for (int a = 0; a < 3; ++a) {
        nlo[3 * (size_t)p + a] = fminf(__ldcg(nlo + 3 * (size_t)l + a), __ldcg(nlo + 3 * (size_t)r + a));
        nhi[3 * (size_t)p + a] = fmaxf(__ldcg(nhi + 3 * (size_t)l + a), __ldcg(nhi + 3 * (size_t)r + a));
      }
      p = parent[p];
    }
  }
}

// Surface area of node x in double (as the host's cost model computes it).
__device__ __forceinline__ double node_area(const float *lo, const float *hi, uint32_t x) {
  const double ex = (double)hi[3 * (size_t)x] - (double)lo[3 * (size_t)x];
  const double ey = (double)hi[3 * (size_t)x + 1] - (double)lo[3 * (size_t)x + 1];
  const double ez = (double)hi[3 * (size_t)x + 2] - (double)lo[3 * (size_t)x + 2];
  return 2.0 * (ex * ey + ey * ez + ez * ex);
}

// 6. leaf choice bottom-up. A subtree covers a contiguous range of the
//    sorted triangles, so it can become one leaf over that range. With node
//    and triangle test cost 1 (as the host builder), cost(x) = min(area(x) *
//    count(x) if count(x) <= leaf_max, area(x) + cost(left) + cost(right)),
//    a radix leaf costing its area; whole[x] = 1 where the leaf is not
//    dearer. The second child to arrive at a node computes it.
__global__ void leaf_choice_kernel(int n, const uint32_t *__restrict__ left, const uint32_t *__restrict__ right,
                                   const uint32_t *__restrict__ parent, const uint32_t *__restrict__ rlo,
                                   const uint32_t *__restrict__ rhi, const float *__restrict__ nlo,
                                   const float *__restrict__ nhi, uint32_t lmax, double *cost, uint8_t *whole,
                                   uint32_t *arrived) {
  const uint32_t first_leaf = (uint32_t)(n - 1);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint32_t p = parent[first_leaf + k];
    while (p != kNone) {
      __threadfence();
      if (atomicAdd(arrived + p, 1u) == 0u) break;
      const uint32_t l = left[p], r = right[p];
      const double cl = l >= first_leaf ? node_area(nlo, nhi, l) : __ldcg(cost + l);
      const double cr = r >= first_leaf ? node_area(nlo, nhi, r) : __ldcg(cost + r);
      const double a = node_area(nlo, nhi, p);
      const double split = a + cl + cr;
      const uint32_t cnt = rhi[p] - rlo[p] + 1u;
      const double leaf = cnt <= lmax ? a * (double)cnt : __longlong_as_double(0x7ff0000000000000ll);
      const bool w = leaf <= split;
      whole[p] = w ? 1 : 0;
      cost[p] = w ? leaf : split;
      p = parent[p];
    }
  }
}

// device allocations of one build, freed on every exit path
struct Scratch {
  std::vector<void *> ptrs;
  ~Scratch() {
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
};

scion_status fail(cudaError_t e, std::string *err) {
  *err = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SCION_ERR_OOM : SCION_ERR_CUDA;
}

int grid_for(uint64_t n, int threads) {
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + threads - 1) / threads, 152ull * 16));
}

}  // namespace

LbvhTree::~LbvhTree() {
  for (void *p : owned) cudaFree(p);
}

scion_status lbvh_build_tree(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                             uint32_t leaf_max, cudaStream_t s, LbvhTree *out, std::string *err) {
  (void)n_verts;
  out->nv = 0;
  out->gpu_ms = 0.0;
  if (n_tris == 0) return SCION_OK;
  const uint32_t n = (uint32_t)n_tris;
  const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
  const size_t npad = (size_t)tiles * kSortTile;
  Scratch sc;
  float *tlo, *thi;
  uint32_t *keys[2], *vals[2], *hist, *cb, *nvalid;
  cudaError_t e;
#define SCION_LB(call)              \
  do {                              \
    e = (call);                     \
    if (e != cudaSuccess) return fail(e, err); \
  } while (0)
  // tree arrays: owned by the result
  auto keep = [&](auto **p, size_t count) -> cudaError_t {
    void *q = nullptr;
    const cudaError_t r = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(**p));
    if (r == cudaSuccess) out->owned.push_back(q);
    *p = static_cast<std::remove_reference_t<decltype(*p)>>(q);
    return r;
  };
  SCION_LB(sc.get(&tlo, 3 * (size_t)n));
  SCION_LB(sc.get(&thi, 3 * (size_t)n));
  for (int b = 0; b < 2; ++b) {
    SCION_LB(keep(&keys[b], npad));
    SCION_LB(keep(&vals[b], npad));
  }
  SCION_LB(sc.get(&hist, (size_t)kRadix * tiles));
  SCION_LB(sc.get(&cb, 8));
  nvalid = cb + 6;
  cudaEvent_t ev0, ev1;
  SCION_LB(cudaEventCreate(&ev0));
  SCION_LB(cudaEventCreate(&ev1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  SCION_LB(cudaEventRecord(ev0, s));
  SCION_LB(cudaMemsetAsync(cb, 0xFF, 3 * sizeof(uint32_t), s));
  SCION_LB(cudaMemsetAsync(cb + 3, 0, 4 * sizeof(uint32_t), s));
  // padding keys sort after every real key (and after the invalid ones)
  SCION_LB(cudaMemsetAsync(keys[0], 0xFF, npad * sizeof(uint32_t), s));
  SCION_LB(cudaMemsetAsync(vals[0], 0xFF, npad * sizeof(uint32_t), s));
  tri_bounds_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_verts, d_indices, n, tlo, thi, cb, nvalid);
  SCION_LB(cudaGetLastError());
  morton_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_verts, d_indices, tlo, thi, n, cb, keys[0], vals[0]);
  SCION_LB(cudaGetLastError());
  int cur = 0;
  for (int shift = 0; shift < 32; shift += 4) {
    radix_hist_kernel<<<tiles, kSortThreads, 0, s>>>(keys[cur], shift, hist, tiles);
    scan_kernel<<<1, kScanThreads, 0, s>>>(hist, kRadix * tiles);
    radix_scatter_kernel<<<tiles, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], shift,
                                                         hist, tiles);
    SCION_LB(cudaGetLastError());
    cur ^= 1;
  }
  uint32_t nv = 0;
  SCION_LB(cudaMemcpyAsync(&nv, nvalid, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  SCION_LB(cudaStreamSynchronize(s));
  out->ids = vals[cur];
  if (nv == 0) {
    SCION_LB(cudaEventRecord(ev1, s));
    SCION_LB(cudaEventSynchronize(ev1));
    return SCION_OK;
  }
  const size_t nn = 2 * (size_t)nv - 1;
  uint32_t *left, *right, *parent, *arrived, *rlo, *rhi;
  uint8_t *axis, *whole;
  float *nlo, *nhi;
  double *cost;
  SCION_LB(keep(&left, nv));
  SCION_LB(keep(&right, nv));
  SCION_LB(keep(&rlo, nv));
  SCION_LB(keep(&rhi, nv));
  SCION_LB(keep(&axis, nv));
  SCION_LB(keep(&whole, nv));
  SCION_LB(keep(&nlo, 3 * nn));
  SCION_LB(keep(&nhi, 3 * nn));
  SCION_LB(sc.get(&parent, nn));
  SCION_LB(sc.get(&arrived, nv));
  SCION_LB(sc.get(&cost, nv));
  SCION_LB(cudaMemsetAsync(parent, 0xFF, nn * sizeof(uint32_t), s));
  SCION_LB(cudaMemsetAsync(arrived, 0, nv * sizeof(uint32_t), s));
  SCION_LB(cudaMemsetAsync(whole, 0, nv, s));
  if (nv > 1) {
    radix_tree_kernel<<<grid_for(nv - 1, 256), 256, 0, s>>>(keys[cur], (int)nv, left, right, parent, axis, rlo,
                                                             rhi);
    SCION_LB(cudaGetLastError());
  }
  boxes_kernel<<<grid_for(nv, 256), 256, 0, s>>>((int)nv, vals[cur], tlo, thi, left, right, parent, nlo, nhi,
                                                  arrived);
  SCION_LB(cudaGetLastError());
  const uint32_t lmax = leaf_max ? leaf_max : 1u;
  if (nv > 1 && lmax > 1) {
    SCION_LB(cudaMemsetAsync(arrived, 0, nv * sizeof(uint32_t), s));
    leaf_choice_kernel<<<grid_for(nv, 256), 256, 0, s>>>((int)nv, left, right, parent, rlo, rhi, nlo, nhi, lmax,
                                                          cost, whole, arrived);
    SCION_LB(cudaGetLastError());
  }
  SCION_LB(cudaEventRecord(ev1, s));
  SCION_LB(cudaStreamSynchronize(s));
  float ms = 0.f;
  SCION_LB(cudaEventElapsedTime(&ms, ev0, ev1));
  out->gpu_ms = ms;
#undef SCION_LB
  out->nv = nv;
  out->left = left;
  out->right = right;
  out->rlo = rlo;
  out->rhi = rhi;
  out->axis = axis;
  out->whole = whole;
  out->nlo = nlo;
  out->nhi = nhi;
  return SCION_OK;
}

scion_status lbvh_download(const LbvhTree &t, cudaStream_t s, LogicalBVH *out, std::string *err) {
  out->nodes.clear();
  out->prims.clear();
  const uint32_t nv = t.nv;
  if (nv == 0) return SCION_OK;
  const size_t nn = 2 * (size_t)nv - 1;
  std::vector<uint32_t> hl(nv), hr(nv), ids(nv), hrl(nv), hrh(nv);
  std::vector<uint8_t> hax(nv), whole(nv);
  std::vector<float> hlo(3 * nn), hhi(3 * nn);
  cudaError_t e = cudaSuccess;
#define SCION_DL(dst, src, bytes) \
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s)
  SCION_DL(ids.data(), t.ids, nv * sizeof(uint32_t));
  SCION_DL(hl.data(), t.left, nv * sizeof(uint32_t));
  SCION_DL(hr.data(), t.right, nv * sizeof(uint32_t));
  SCION_DL(hax.data(), t.axis, nv);
  SCION_DL(whole.data(), t.whole, nv);
  SCION_DL(hrl.data(), t.rlo, nv * sizeof(uint32_t));
  SCION_DL(hrh.data(), t.rhi, nv * sizeof(uint32_t));
  SCION_DL(hlo.data(), t.nlo, 3 * nn * sizeof(float));
  SCION_DL(hhi.data(), t.nhi, 3 * nn * sizeof(float));
#undef SCION_DL
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e, err);
  // Logical tree, depth first from the root.
  out->prims = std::move(ids);
  out->nodes.reserve(nn);
  struct Item {
    uint32_t src, dst;  // node of the radix tree, node of the logical tree
  };
  std::vector<Item> todo;
  auto box_of = [&](uint32_t x) {
    Box3 b;
    for (int a = 0; a < 3; ++a) {
      b.lo[a] = hlo[3 * (size_t)x + a];
      b.hi[a] = hhi[3 * (size_t)x + a];
    }
    return b;
  };
  auto emit = [&](uint32_t src) {
    LNode d{};
    d.box = box_of(src);
    const uint32_t id = (uint32_t)out->nodes.size();
    if (src + 1 >= nv) {  // a leaf of the radix tree: one triangle
      d.first = src - (nv - 1);
      d.count = 1;
    } else if (whole[src]) {
      d.first = hrl[src];
      d.count = hrh[src] - hrl[src] + 1;
    } else {
      d.axis = hax[src];
      todo.push_back(Item{src, id});
    }
    out->nodes.push_back(d);
    return id;
  };
  emit(0);
  while (!todo.empty()) {
    const Item it = todo.back();
    todo.pop_back();
    const uint32_t l = emit(hl[it.src]);
    const uint32_t r = emit(hr[it.src]);
    out->nodes[it.dst].left = l;
    out->nodes[it.dst].right = r;
  }
  return SCION_OK;
}

scion_status lbvh_build(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                        uint32_t leaf_max, cudaStream_t s, LogicalBVH *out, double *gpu_ms, std::string *err) {
  out->nodes.clear();
  out->prims.clear();
  *gpu_ms = 0.0;
  LbvhTree t;
  scion_status st = lbvh_build_tree(d_verts, n_verts, d_indices, n_tris, leaf_max, s, &t, err);
  if (st != SCION_OK) return st;
  *gpu_ms = t.gpu_ms;
  return lbvh_download(t, s, out, err);
}

}  // namespace scion
