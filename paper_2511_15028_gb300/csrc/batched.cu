// Many scenes in one persistent launch (closest hit).
//
// Every scene keeps its own BVH and layout. Its rays occupy a range of a global
// index space padded to multiples of 32, so each 32-ray unit a warp takes from
// the global counter belongs to exactly one scene; the warp dispatches on that
// scene's node family with a warp-uniform switch over the traversal template
// instances and stays with the scene while the next units it takes belong to
// it. The scene's fetch mode holds: warp batches (each lane traces its ray of
// the unit to completion, then the warp takes the next unit) or warp refill
// (idle lanes take the next rays as soon as at least rays_per_fetch of them
// are idle, from a new unit when the current one is used up; a unit of
// another scene ends the refill, the warp finishes its rays and moves on).
// The launch allocates nothing and never synchronises the host, so it can be
// captured in a CUDA graph and replayed; its counters reset themselves.
#include <cuda_runtime.h>

#include "batched.h"
#include "kernels.h"

namespace scion {

namespace {

constexpr int kMaxSharedScenes = 1024;  // scene starts cached in shared memory

template <bool OWN, int W, int PREC, int SOA>
__device__ __forceinline__ void step_family(const TraceArgs &a, Lane &L, Stack &st, Counts &cnt) {
  if constexpr (OWN) step_bin<PREC, SOA, REF_DIRECT, false, false>(a, L, st, cnt);
  else step_wide<W, PREC, SOA, REF_DIRECT, false, false>(a, L, st, cnt);
}

// The next 32-ray unit of the global index space (warp-uniform).
__device__ __forceinline__ unsigned long long take_unit(unsigned long long *work) {
  unsigned long long b = 0;
  if ((threadIdx.x & 31u) == 0) b = atomicAdd(work, (unsigned long long)kBatchUnit);
  return __shfl_sync(0xFFFFFFFFu, b, 0);
}

__device__ __forceinline__ void start_lane(const TraceArgs &a, Lane &L, Stack &st, unsigned long long rid, bool own) {
  L.rid = rid;
  setup_ray(ldg4f(a.rays + 2 * rid), ldg4f(a.rays + 2 * rid + 1), L.r);
  L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_MISS};
  L.steps = 0;
  L.err = 0;
  L.found = false;
  st.reset();
  L.cur = own ? (a.n_nodes > 0 ? 0u : kEmptyRef) : a.root_ref;
}

__device__ __forceinline__ void finish_lane(const TraceArgs &a, Lane &L) {
  if (L.err) {
    atomicCAS(a.status, 0u, L.err);
    L.b = Best{__int_as_float(0x7f800000), 0.f, 0.f, SCION_PRIM_ERROR};
  }
  static_cast<uint4 *>(a.out)[L.rid] =
      make_uint4(__float_as_uint(L.b.t), __float_as_uint(L.b.u), __float_as_uint(L.b.v), L.b.id);
}

// Trace the scene's unit at `base` and every following unit the warp takes
// while they belong to the scene; returns the first unit taken that does not
// (another scene's, or >= total). Not inlined: each family's loops get their
// own register allocation (inlined into one switch they spill heavily); the
// call costs once per scene change of a warp.
// The stack is made here, not passed in: an object whose address crosses a
// call lives in local memory, and so would the stack pointer on every step.
template <bool OWN, int W, int PREC, int SOA>
__device__ __noinline__ unsigned long long run_scene(const BatchScene &S, unsigned long long base,
                                                     unsigned long long *work, uint2 *smem_col,
                                                     uint32_t smem_stack) {
  Stack st;
  StackTail<false> tail;
  st.attach(tail);
  st.sh = smem_col;
  st.stride = blockDim.x;
  st.cap_sh = (int)smem_stack;
  st.reset();
  const TraceArgs &a = S.a;
  const unsigned long long s_lo = S.begin, s_hi = S.begin + ((a.n + 31ull) & ~31ull);
  const uint32_t lane = threadIdx.x & 31u;
  Counts cnt;
  Lane L;
  if (a.refill_min == 0) {
    // warp batches: every lane traces its ray of the unit to completion
    while (base >= s_lo && base < s_hi) {
      const unsigned long long rid = base - s_lo + lane;
      if (rid < a.n) {
        start_lane(a, L, st, rid, OWN);
        while (L.cur != kEmptyRef) {
          if (++L.steps > a.max_steps) {
            L.err = kErrIter;
            L.cur = kEmptyRef;
            break;
          }
          step_family<OWN, W, PREC, SOA>(a, L, st, cnt);
        }
        finish_lane(a, L);
      }
      base = take_unit(work);
    }
    return base;
  }
  // warp refill from the rays [next, hi) of the current unit
  const uint32_t k = a.refill_min;
  const uint32_t below = (1u << lane) - 1u;  // lanes ranked before this one
  unsigned long long next = base - s_lo;
  unsigned long long hi = next + kBatchUnit < a.n ? next + kBatchUnit : a.n;
  unsigned long long pending = 0;
  bool mine = true;  // the last unit taken belongs to this scene
  bool has_ray = false;
  L.cur = kEmptyRef;
  while (true) {
    const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !has_ray);
    const uint32_t n_idle = __popc(idle);
    if (n_idle >= k) {
      if (next >= hi && mine) {
        const unsigned long long b = take_unit(work);
        if (b >= s_lo && b < s_hi) {
          next = b - s_lo;
          hi = next + kBatchUnit < a.n ? next + kBatchUnit : a.n;
        } else {
          mine = false;
          pending = b;
        }
      }
      if (next < hi) {
        if (!has_ray) {
          const unsigned long long rid = next + __popc(idle & below);
          if (rid < hi) {
            start_lane(a, L, st, rid, OWN);
            has_ray = true;
          }
        }
        next = next + n_idle < hi ? next + n_idle : hi;
      }
    }
    // a unit of this scene always holds a ray, so with every lane idle the
    // warp either took rays above or has moved past the scene
    if (__ballot_sync(0xFFFFFFFFu, has_ray) == 0u) break;
    if (has_ray && L.cur != kEmptyRef) {
      if (++L.steps > a.max_steps) {
        L.err = kErrIter;
        L.cur = kEmptyRef;
      } else {
        step_family<OWN, W, PREC, SOA>(a, L, st, cnt);
      }
    }
    if (has_ray && L.cur == kEmptyRef) {
      finish_lane(a, L);
      has_ray = false;
    }
  }
  return pending;
}

__global__ void __launch_bounds__(kMaxThreadsPerBlock, kMinBlocksPerSm)
    batched_kernel(const BatchScene *__restrict__ scenes, uint32_t n_scenes, unsigned long long total,
                   unsigned long long *work, uint32_t *exit_count, uint32_t smem_stack) {
  extern __shared__ uint2 smem[];
  // scene starts (padded global offsets) for the unit -> scene search
  __shared__ unsigned long long starts[kMaxSharedScenes];
  const uint32_t cached = n_scenes < (uint32_t)kMaxSharedScenes ? n_scenes : (uint32_t)kMaxSharedScenes;
  for (uint32_t i = threadIdx.x; i < cached; i += blockDim.x) starts[i] = scenes[i].begin;
  __syncthreads();
  uint2 *const col = smem + threadIdx.x;  // this thread's shared-memory stack column
  unsigned long long base = take_unit(work);
  while (base < total) {
    // last scene whose start <= base (binary search, warp-uniform)
    uint32_t lo = 0, hi = n_scenes;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      const unsigned long long sm = mid < cached ? starts[mid] : scenes[mid].begin;
      if (sm <= base) lo = mid;
      else hi = mid;
    }
    const BatchScene &S = scenes[lo];
    switch (S.family) {
      case kFamilyBin: base = run_scene<true, 2, PREC_F32, LAYOUT_AOS>(S, base, work, col, smem_stack); break;
      case kFamilyBinQ16: base = run_scene<true, 2, PREC_Q16, LAYOUT_AOS>(S, base, work, col, smem_stack); break;
      case kFamilyW4F32: base = run_scene<false, 4, PREC_F32, LAYOUT_SOA>(S, base, work, col, smem_stack); break;
      case kFamilyW4F16: base = run_scene<false, 4, PREC_F16, LAYOUT_SOA>(S, base, work, col, smem_stack); break;
      case kFamilyW4U8: base = run_scene<false, 4, PREC_U8, LAYOUT_SOA>(S, base, work, col, smem_stack); break;
      case kFamilyW8F16: base = run_scene<false, 8, PREC_F16, LAYOUT_SOA>(S, base, work, col, smem_stack); break;
      case kFamilyW8U8: base = run_scene<false, 8, PREC_U8, LAYOUT_AOS>(S, base, work, col, smem_stack); break;
      case kFamilyW8U8S: base = run_scene<false, 8, PREC_U8, LAYOUT_SOA>(S, base, work, col, smem_stack); break;
      default: base = take_unit(work); break;  // batch creation admits only the families above
    }
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
  if (own_box) {
    if (d.box_layout != LAYOUT_AOS) return -1;
    if (d.box_prec == PREC_F32) return (int)kFamilyBin;
    if (d.box_prec == PREC_Q16) return (int)kFamilyBinQ16;
    return -1;
  }
  if (d.width == 4 && d.box_layout == LAYOUT_SOA) {
    if (d.box_prec == PREC_F32) return (int)kFamilyW4F32;
    if (d.box_prec == PREC_F16) return (int)kFamilyW4F16;
    if (d.box_prec == PREC_U8) return (int)kFamilyW4U8;
    return -1;
  }
  if (d.width == 8 && d.box_prec == PREC_F16 && d.box_layout == LAYOUT_SOA) return (int)kFamilyW8F16;
  if (d.width == 8 && d.box_prec == PREC_U8) return d.box_layout == LAYOUT_AOS ? (int)kFamilyW8U8 : (int)kFamilyW8U8S;
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
