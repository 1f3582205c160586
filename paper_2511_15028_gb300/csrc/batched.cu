// Many scenes in one persistent launch (closest hit).
//
// Every scene keeps its own BVH and layout. Its rays occupy a range of a global
// index space padded to multiples of 32, so each 32-ray chunk a warp takes
// belongs to exactly one scene and the warp dispatches on that scene's node
// family with a warp-uniform switch over the traversal template instances.
// The launch allocates nothing and never synchronises the host, so it can be
// captured in a CUDA graph and replayed; its counters reset themselves.
#include <cuda_runtime.h>

#include "batched.h"
#include "kernels.h"

namespace scion {

namespace {

constexpr int kMaxSharedScenes = 1024;  // scene starts cached in shared memory

template <bool OWN, int W, int PREC, int SOA>
__device__ __forceinline__ void trace_one(const TraceArgs &a, Lane &L, Stack &st, Counts &cnt) {
  while (L.cur != kEmptyRef) {
    if (++L.steps > a.max_steps) {
      L.err = kErrIter;
      L.cur = kEmptyRef;
      break;
    }
    if constexpr (OWN) step_bin<PREC_F32, SOA, REF_DIRECT, false, false>(a, L, st, cnt);
    else step_wide<W, PREC, SOA, REF_DIRECT, false, false>(a, L, st, cnt);
  }
}

__global__ void __launch_bounds__(kMaxThreadsPerBlock)
    batched_kernel(const BatchScene *__restrict__ scenes, uint32_t n_scenes, unsigned long long total,
                   unsigned long long *work, uint32_t *exit_count, uint32_t smem_stack) {
  extern __shared__ uint2 smem[];
  // scene starts (padded global offsets) for the chunk -> scene search
  __shared__ unsigned long long starts[kMaxSharedScenes];
  const uint32_t cached = n_scenes < (uint32_t)kMaxSharedScenes ? n_scenes : (uint32_t)kMaxSharedScenes;
  for (uint32_t i = threadIdx.x; i < cached; i += blockDim.x) starts[i] = scenes[i].begin;
  __syncthreads();
  Stack st;
  st.sh = smem + threadIdx.x;
  st.stride = blockDim.x;
  st.cap_sh = (int)smem_stack;
  st.reset();
  Counts cnt;
  const uint32_t lane = threadIdx.x & 31u;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, 32ull);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (base >= total) break;
    // last scene whose start <= base (binary search, warp-uniform)
    uint32_t lo = 0, hi = n_scenes;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      const unsigned long long sm = mid < cached ? starts[mid] : scenes[mid].begin;
      if (sm <= base) lo = mid;
      else hi = mid;
    }
    const BatchScene &S = scenes[lo];
    const TraceArgs &a = S.a;
    const unsigned long long rid = base - S.begin + lane;
    if (rid >= a.n) continue;
    Lane L;
    L.rid = rid;
    setup_ray(ldg4f(a.rays + 2 * rid), ldg4f(a.rays + 2 * rid + 1), L.r);
    L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_MISS};
    L.steps = 0;
    L.err = 0;
    L.found = false;
    st.reset();
    L.cur = S.family == kFamilyBin ? (a.n_nodes > 0 ? 0u : kEmptyRef) : a.root_ref;
    switch (S.family) {
      case kFamilyBin: trace_one<true, 2, PREC_F32, LAYOUT_AOS>(a, L, st, cnt); break;
      case kFamilyW4F32: trace_one<false, 4, PREC_F32, LAYOUT_SOA>(a, L, st, cnt); break;
      case kFamilyW8F16: trace_one<false, 8, PREC_F16, LAYOUT_SOA>(a, L, st, cnt); break;
      case kFamilyW8U8: trace_one<false, 8, PREC_U8, LAYOUT_AOS>(a, L, st, cnt); break;
      default: L.err = kErrIter; L.cur = kEmptyRef; break;
    }
    if (L.err) {
      atomicCAS(a.status, 0u, L.err);
      L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_ERROR};
    }
    static_cast<uint4 *>(a.out)[rid] =
        make_uint4(__float_as_uint(L.b.t), __float_as_uint(L.b.u), __float_as_uint(L.b.v), L.b.id);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t prev = atomicAdd(exit_count, 1u);
    if (prev == gridDim.x - 1) {
      *work = 0ull;
      *exit_count = 0u;
      __threadfence();
    }
  }
}

}  // namespace

int batched_family(uint32_t own_box, const scion_layout_desc &d) {
  if (d.child_ref != REF_DIRECT) return -1;
  if (own_box) return d.box_layout == LAYOUT_AOS ? (int)kFamilyBin : -1;
  if (d.width == 4 && d.box_prec == PREC_F32 && d.box_layout == LAYOUT_SOA) return (int)kFamilyW4F32;
  if (d.width == 8 && d.box_prec == PREC_F16 && d.box_layout == LAYOUT_SOA) return (int)kFamilyW8F16;
  if (d.width == 8 && d.box_prec == PREC_U8 && d.box_layout == LAYOUT_AOS) return (int)kFamilyW8U8;
  return -1;
}

const void *batched_kernel_ptr() { return (const void *)batched_kernel; }

cudaError_t launch_batched(const BatchScene *d_scenes, uint32_t n_scenes, unsigned long long total,
                           unsigned long long *work, uint32_t *exit_count, uint32_t smem_stack,
                           uint32_t threads, uint32_t grid, cudaStream_t s) {
  const size_t smem = (size_t)threads * smem_stack * sizeof(uint2);
  batched_kernel<<<grid, threads, smem, s>>>(d_scenes, n_scenes, total, work, exit_count, smem_stack);
  return cudaGetLastError();
}

}  // namespace scion
