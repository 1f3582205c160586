// C ABI (include/scion.h, include/scion_debug.h): build, trace, status.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/scion.h"
#include "../../include/scion_debug.h"
#include "backward.h"
#include "batched.h"
#include "builder.h"
#include "gpack.h"
#include "kernels.h"
#include "lbvh.h"
#include "refit.h"

using namespace scion;

namespace {
constexpr uint32_t kStreamSlotCount = 64;  // distinct streams one BVH can be traced on
}

struct scion_bvh_s {
  scion_layout_desc desc;
  bool own_box = false;
  uint32_t n_tris = 0, n_verts = 0;
  bool indexed = false;
  uint32_t n_nodes = 0, node_stride = 0, n_leaf_entries = 0;
  uint32_t root_ref = kEmptyRef, depth = 0, stack_need = 0;
  float frame[9] = {};  // world grid of the quantised own-box codecs
  uint64_t node_bytes = 0, node2_bytes = 0, prim_bytes = 0, idx_bytes = 0, vert_bytes = 0;
  void *d_nodes = nullptr, *d_nodes2 = nullptr, *d_prims = nullptr, *d_prim_ids = nullptr;
  void *d_verts = nullptr, *d_idx = nullptr;
  // device scratch: words 0-3 hold the status word (word 3); then one 16-byte
  // slot per stream that has traced this BVH (u64 work counter, u32 exit
  // counter, pad), so launches on different streams never share a counter
  uint32_t *d_scratch = nullptr;
  std::mutex slot_mu;
  uint32_t n_slots = 0;
  cudaStream_t slot_stream[kStreamSlotCount] = {};
  double build_ms = 0.0, logical_ms = 0.0, pack_ms = 0.0;
  int device = 0;
  // refit scratch, allocated by the first scion_refit
  uint32_t *d_refit_parent = nullptr, *d_refit_pending = nullptr;
  void *d_refit_boxes = nullptr;
  float *d_refit_frame = nullptr;
};

namespace {

// message of the last failing call, per host thread
thread_local std::string g_last_error;
constexpr size_t kScratchBytes = 16 + 16 * kStreamSlotCount;

// scion_trace_params.ordered_children -> kernel order mode
uint32_t order_mode(uint32_t oc) { return oc == 2 ? 0u : (oc == 3 ? 2u : 1u); }

// Counter slot of `stream` for this BVH (assigned on first use), or -1 when
// kStreamSlotCount other streams already hold slots.
int stream_slot(scion_bvh b, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(b->slot_mu);
  for (uint32_t i = 0; i < b->n_slots; ++i)
    if (b->slot_stream[i] == stream) return (int)i;
  if (b->n_slots == kStreamSlotCount) return -1;
  b->slot_stream[b->n_slots] = stream;
  return (int)b->n_slots++;
}

scion_status cuda_fail(cudaError_t e) {
  g_last_error = cudaGetErrorString(e);
  return SCION_ERR_CUDA;
}

#define SCION_CUDA(call)                                      \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) {                                  \
      if (e_ == cudaErrorMemoryAllocation) {                  \
        g_last_error = "out of device memory";                \
        return SCION_ERR_OOM;                                 \
      }                                                       \
      return cuda_fail(e_);                                   \
    }                                                         \
  } while (0)

void free_bvh(scion_bvh b) {
  if (!b) return;
  void *bufs[] = {b->d_nodes,       b->d_nodes2,         b->d_prims,          b->d_prim_ids,
                  b->d_verts,       b->d_idx,            b->d_scratch,        b->d_refit_parent,
                  b->d_refit_pending, b->d_refit_boxes,  b->d_refit_frame};
  for (void *p : bufs)
    if (p) cudaFree(p);
  delete b;
}

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return dev;
}

// Device (or managed) memory that a kernel on the current device may use:
// device memory of another GPU would be a peer access the caller never
// arranged, so it is refused like host memory.
bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == current_device();
}

// The address a kernel uses for a ray or result buffer: device (or managed)
// memory of the current device as given, page-locked host memory through its
// device mapping (the kernel then reads and writes host memory directly, e.g.
// over NVLink-C2C). Pageable host memory and other GPUs' memory are not
// reachable from the kernel: nullptr.
const void *kernel_view(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeDevice) return at.device == current_device() ? p : nullptr;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    // the mapping of the allocation's start, shifted to p
    const char *base = static_cast<const char *>(at.hostPointer);
    return static_cast<const char *>(at.devicePointer) + (static_cast<const char *>(p) - base);
  }
  return nullptr;
}

// The BVH's buffers live on the device it was built on; a call made while
// another device is current would hand them to that device's kernels.
bool on_bvh_device(const scion_bvh b) {
  const int dev = current_device();
  if (dev == b->device) return true;
  g_last_error = "the BVH was built on device " + std::to_string(b->device) + " but device " +
                 std::to_string(dev) + " is current";
  return false;
}

template <typename T>
scion_status upload(void **dst, const std::vector<T> &src, cudaStream_t s, uint64_t *bytes) {
  *bytes = src.size() * sizeof(T);
  if (src.empty()) return SCION_OK;
  SCION_CUDA(cudaMalloc(dst, *bytes));
  SCION_CUDA(cudaMemcpyAsync(*dst, src.data(), *bytes, cudaMemcpyHostToDevice, s));
  return SCION_OK;
}

// The BVH's part of the kernel arguments (buffers, root, codec constants).
void bvh_args(const scion_bvh b, TraceArgs &a) {
  a.nodes = static_cast<const uint4 *>(b->d_nodes);
  a.nodes2 = static_cast<const uint2 *>(b->d_nodes2);
  a.prims = static_cast<const float4 *>(b->d_prims);
  a.prim_ids = static_cast<const uint32_t *>(b->d_prim_ids);
  a.verts = static_cast<const float4 *>(b->d_verts);
  a.tri_idx = static_cast<const uint32_t *>(b->d_idx);
  a.root_ref = b->root_ref;
  a.n_nodes = b->n_nodes;
  a.prim_indirect = b->desc.prim_ref;
  a.node_stride = b->node_stride;
  for (int k = 0; k < 9; ++k) a.frame[k] = b->frame[k];
}

// Dynamic shared memory above this needs the kernel's opt-in attribute (the
// default limit of 48 KB also covers the kernels' static shared memory).
constexpr size_t kSmemOptIn = 32 * 1024;

// Query kinds of launch_trace.
constexpr int kQueryClosest = 0, kQueryAny = 1, kQueryPoint = 2;

// Shared-memory stack entries per thread. The traversal kernels of the
// own-box bvh2 nodes (all but the shared-slab one) and of 2/4-wide nodes keep
// the shared part of the stack as a ring indexed with a mask (StackFor in
// trace.cuh), so for them the count is rounded down to a power of two.
uint32_t stack_entries(scion_bvh b, uint32_t requested, int query) {
  const bool ring = query != kQueryPoint && ((b->own_box && b->desc.box_prec != PREC_SLAB) ||
                                             (!b->own_box && b->desc.width <= 4));
  if (!ring) return requested;
  uint32_t p = 1;
  while (p * 2 <= requested) p *= 2;
  return p;
}

// Warp-batch work of a launch over a.n rays: consecutive 32-ray batches, or
// 8x4 pixel tiles of a row-major image raster_w wide (32 slots per tile).
void set_raster(TraceArgs &a, uint32_t raster_w) {
  a.raster_w = raster_w;
  if (!raster_w) {
    a.n_work = a.n;
    return;
  }
  // up to the last tile holding a ray: ray n-1 is pixel (c, r); every tile of
  // its tile row holds a ray when a row above r lies in that tile row,
  // otherwise only the tiles up to column c do
  const unsigned long long tiles_x = (raster_w + 7ull) / 8, r = (a.n - 1) / raster_w, c = (a.n - 1) % raster_w;
  a.n_work = ((r / 4) * tiles_x + (r % 4 ? tiles_x : c / 8 + 1)) * 32ull;
}


// Shared-memory stack bytes per entry: (ref, entry distance), plus the exit
// distance for the shared-slab layout, whose traversal carries intervals.
size_t stack_entry_bytes(const scion_bvh b, int query) {
  const bool slab = b->own_box && b->desc.box_prec == PREC_SLAB && query != kQueryPoint;
  return sizeof(uint2) + (slab ? sizeof(float) : 0);
}

TraceKernel pick_cpq_kernel(const scion_bvh b, int stats) {
  const scion_layout_desc &d = b->desc;
  const int soa = (int)d.box_layout, cref = (int)d.child_ref;
  if (b->own_box) {
    switch (d.box_prec) {
      case PREC_F32: return cpq_kernels_own_p0(soa, cref, stats);
      case PREC_Q16: return cpq_kernels_own_p3(soa, cref, stats);
      case PREC_EQ10: return cpq_kernels_own_p4(soa, cref, stats);
      case PREC_SLAB: return cpq_kernels_own_p6(soa, cref, stats);
    }
    return nullptr;
  }
  switch (d.width * 10 + d.box_prec) {
    case 20: return cpq_kernels_w2_p0(soa, cref, stats);
    case 21: return cpq_kernels_w2_p1(soa, cref, stats);
    case 22: return cpq_kernels_w2_p2(soa, cref, stats);
    case 40: return cpq_kernels_w4_p0(soa, cref, stats);
    case 41: return cpq_kernels_w4_p1(soa, cref, stats);
    case 42: return cpq_kernels_w4_p2(soa, cref, stats);
    case 80: return cpq_kernels_w8_p0(soa, cref, stats);
    case 81: return cpq_kernels_w8_p1(soa, cref, stats);
    case 82: return cpq_kernels_w8_p2(soa, cref, stats);
    case 25: return cpq_kernels_w2_p5(soa, cref, stats);
    case 45: return cpq_kernels_w4_p5(soa, cref, stats);
    case 85: return cpq_kernels_w8_p5(soa, cref, stats);
  }
  return nullptr;
}

TraceKernel pick_kernel(const scion_bvh b, int query, int stats, uint32_t reg) {
  const scion_layout_desc &d = b->desc;
  const int soa = (int)d.box_layout, cref = (int)d.child_ref;
  if (query == kQueryPoint) return reg == 0 ? pick_cpq_kernel(b, stats) : nullptr;
  const int rg = (int)reg;
  const int any = query == kQueryAny ? 1 : 0;
  if (b->own_box) {
    switch (d.box_prec) {
      case PREC_F32: return kernels_own_p0(soa, cref, any, stats, rg);
      case PREC_Q16: return kernels_own_p3(soa, cref, any, stats, rg);
      case PREC_EQ10: return kernels_own_p4(soa, cref, any, stats, rg);
      case PREC_SLAB: return kernels_own_p6(soa, cref, any, stats, rg);
    }
    return nullptr;
  }
  switch (d.width * 10 + d.box_prec) {
    case 20: return kernels_w2_p0(soa, cref, any, stats, rg);
    case 21: return kernels_w2_p1(soa, cref, any, stats, rg);
    case 22: return kernels_w2_p2(soa, cref, any, stats, rg);
    case 40: return kernels_w4_p0(soa, cref, any, stats, rg);
    case 41: return kernels_w4_p1(soa, cref, any, stats, rg);
    case 42: return kernels_w4_p2(soa, cref, any, stats, rg);
    case 80: return kernels_w8_p0(soa, cref, any, stats, rg);
    case 81: return kernels_w8_p1(soa, cref, any, stats, rg);
    case 82: return kernels_w8_p2(soa, cref, any, stats, rg);
    case 25: return kernels_w2_p5(soa, cref, any, stats, rg);
    case 45: return kernels_w4_p5(soa, cref, any, stats, rg);
    case 85: return kernels_w8_p5(soa, cref, any, stats, rg);
  }
  return nullptr;
}


// Host half of scion_build_many: validate every descriptor (all must share
// leaf_max and sah_bins), build the logical BVH2 once, pack each layout.
scion_status build_host_many(const float *v, uint64_t n_verts, const uint32_t *ix, uint64_t n_tris,
                             const scion_layout_desc *descs, uint32_t n_desc, std::vector<HostBVH> *hbs) {
  if (!descs || n_desc == 0 || (n_tris > 0 && !v)) return SCION_ERR_INVALID_ARG;
  if (n_tris >= kMaxPrims || n_verts >= (1ull << 32)) return SCION_ERR_INVALID_ARG;
  if (!ix && n_verts != 3 * n_tris) return SCION_ERR_INVALID_ARG;
  std::vector<scion_layout_desc> d(n_desc);
  std::vector<bool> own(n_desc);
  for (uint32_t i = 0; i < n_desc; ++i) {
    bool ob = false;
    scion_status st = normalize_desc(descs[i], &d[i], &ob);
    if (st != SCION_OK) return st;
    own[i] = ob;
    if (d[i].leaf_max != d[0].leaf_max || d[i].sah_bins != d[0].sah_bins) {
      g_last_error = "scion_build_many: descriptors differ in leaf_max or sah_bins";
      return SCION_ERR_INVALID_ARG;
    }
  }
  if (ix)
    for (uint64_t i = 0; i < 3 * n_tris; ++i)
      if (ix[i] >= n_verts) return SCION_ERR_INVALID_ARG;
  BuildInput in{v, n_verts, ix, n_tris};
  try {
    const auto t0 = std::chrono::steady_clock::now();
    LogicalBVH lb;
    build_logical(in, d[0].sah_bins, d[0].leaf_max, &lb);
    const double logical_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    hbs->resize(n_desc);
    for (uint32_t i = 0; i < n_desc; ++i) {
      const auto t1 = std::chrono::steady_clock::now();
      std::string err;
      scion_status st = pack_bvh(in, lb, d[i], own[i], &(*hbs)[i], &err);
      if (st != SCION_OK) {
        g_last_error = err;
        return st;
      }
      HostBVH &h = (*hbs)[i];
      h.logical_ms = logical_ms;
      h.pack_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
      h.build_ms = h.logical_ms + h.pack_ms;
    }
  } catch (const std::bad_alloc &) {
    g_last_error = "out of host memory";
    return SCION_ERR_OOM;
  }
  return SCION_OK;
}

// Host half of scion_build: validate, build the logical BVH2, pack.
scion_status build_host(const float *v, uint64_t n_verts, const uint32_t *ix, uint64_t n_tris,
                        const scion_layout_desc *desc, HostBVH *hb) {
  if (!desc || (n_tris > 0 && !v)) return SCION_ERR_INVALID_ARG;
  if (n_tris >= kMaxPrims || n_verts >= (1ull << 32)) return SCION_ERR_INVALID_ARG;
  if (!ix && n_verts != 3 * n_tris) return SCION_ERR_INVALID_ARG;
  scion_layout_desc d;
  bool own_box = false;
  scion_status st = normalize_desc(*desc, &d, &own_box);
  if (st != SCION_OK) return st;
  if (ix)
    for (uint64_t i = 0; i < 3 * n_tris; ++i)
      if (ix[i] >= n_verts) return SCION_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  BuildInput in{v, n_verts, ix, n_tris};
  try {
    LogicalBVH lb;
    build_logical(in, d.sah_bins, d.leaf_max, &lb);
    const auto t1 = std::chrono::steady_clock::now();
    hb->logical_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    std::string err;
    st = pack_bvh(in, lb, d, own_box, hb, &err);
    if (st != SCION_OK) {
      g_last_error = err;
      return st;
    }
    hb->pack_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  } catch (const std::bad_alloc &) {
    g_last_error = "out of host memory";
    return SCION_ERR_OOM;
  }
  hb->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return SCION_OK;
}

uint64_t host_prim_bytes(const HostBVH &hb) {
  return hb.prim_direct.size() * 4 + hb.prim_ids.size() * 4 +
         (hb.desc.prim_ref == REF_INDIRECT ? hb.indices.size() * 4 : 0);
}

struct DevInfo {
  int sms = 0;
};
std::mutex g_dev_mu;
std::vector<DevInfo> g_dev;

int device_sms(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
  if (g_dev[dev].sms == 0) cudaDeviceGetAttribute(&g_dev[dev].sms, cudaDevAttrMultiProcessorCount, dev);
  return g_dev[dev].sms;
}

// Dynamic shared memory above kSmemOptIn needs the kernel's opt-in
// attribute. The attribute belongs to the kernel (per device) and only ever
// grows here: a launch with less shared memory never lowers it below what an
// earlier launch of the same kernel needed.
struct SmemKey {
  const void *k;
  int dev;
  size_t bytes;
};
std::mutex g_smem_mu;
std::vector<SmemKey> g_smem;

scion_status ensure_smem_optin(const void *k, size_t smem, int dev) {
  if (smem <= kSmemOptIn) return SCION_OK;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  for (SmemKey &e : g_smem)
    if (e.k == k && e.dev == dev) {
      if (e.bytes >= smem) return SCION_OK;
      SCION_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      e.bytes = smem;
      return SCION_OK;
    }
  SCION_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  g_smem.push_back(SmemKey{k, dev, smem});
  return SCION_OK;
}

// Resident CTAs per SM of a kernel at a launch shape, per device: the
// occupancy query runs once per (kernel, threads, shared bytes, device), not
// on every trace call.
struct OccKey {
  const void *k;
  uint32_t tpb;
  size_t smem;
  int dev;
  int ctas;
};
std::mutex g_occ_mu;
std::vector<OccKey> g_occ;

scion_status ctas_per_sm(const void *k, uint32_t tpb, size_t smem, int dev, uint32_t *out) {
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (const OccKey &o : g_occ)
      if (o.k == k && o.tpb == tpb && o.smem == smem && o.dev == dev) {
        *out = (uint32_t)o.ctas;
        return SCION_OK;
      }
  }
  int nb = 0;
  SCION_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, (int)tpb, smem));
  nb = std::max(nb, 1);
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ.push_back(OccKey{k, tpb, smem, dev, nb});
  *out = (uint32_t)nb;
  return SCION_OK;
}

// A trace launch ready to go, but for the counters it uses.
struct TraceLaunch {
  TraceKernel k = nullptr;
  TraceArgs a{};
  uint32_t tpb = 0;
  size_t smem = 0;
  uint64_t grid = 0;
  uint32_t ctas_param = 0;  // scion_trace_params.ctas_per_sm (0: from occupancy)
  uint32_t reg_stack = 0;   // register entries at the top of the stack
};

// Checks and set-up shared by every entry point that launches a traversal or
// closest point kernel (scion_trace_closest/_any/_stats,
// scion_query_closest_point, scion_trace_closest_noalloc): arguments,
// alignment, traversal parameters, the device, and the buffers a kernel can
// reach. On success `L` holds everything but the work counters and the
// visit counters; on failure nothing has been issued and g_last_error says
// why. n must be > 0.
scion_status prepare_trace(scion_bvh b, const scion_ray *rays, uint64_t n, void *out,
                           const scion_trace_params *params, int query, TraceLaunch *L) {
  if (!b || !rays || !out) {
    g_last_error = "null BVH, input or result buffer";
    return SCION_ERR_INVALID_ARG;
  }
  const bool out16 = query != kQueryAny;  // scion_hit / scion_closest_point records
  if ((reinterpret_cast<uintptr_t>(rays) & 15u) || (out16 && (reinterpret_cast<uintptr_t>(out) & 15u)) ||
      (!out16 && (reinterpret_cast<uintptr_t>(out) & 3u))) {
    g_last_error = "input records must be 16-byte aligned, results 16-byte (records) or 4-byte (flags) aligned";
    return SCION_ERR_INVALID_ARG;
  }
  scion_trace_params p{};
  if (params) p = *params;
  if (p.reg_stack != 0 && p.reg_stack != 2 && p.reg_stack != kMaxRegStack) {
    g_last_error = "reg_stack must be 0, 2 or 4";
    return SCION_ERR_INVALID_ARG;
  }
  if (query == kQueryPoint && p.reg_stack != 0) {
    g_last_error = "closest point queries keep their stack in memory (reg_stack 0)";
    return SCION_ERR_INVALID_ARG;
  }
  if (p.rays_per_fetch > 32) {
    g_last_error = "rays_per_fetch exceeds 32";
    return SCION_ERR_INVALID_ARG;
  }
  if (p.raster_width != 0 && ((p.rays_per_fetch != 0 && p.rays_per_fetch != 32) || query == kQueryPoint)) {
    g_last_error = "raster_width needs warp batches (rays_per_fetch 0 or 32) and rays";
    return SCION_ERR_INVALID_ARG;
  }
  if (query == kQueryPoint && p.rays_per_fetch != 0 && p.rays_per_fetch != 32) {
    g_last_error = "closest point queries take 32-point warp batches only (rays_per_fetch 0 or 32)";
    return SCION_ERR_INVALID_ARG;
  }
  const uint32_t tpb = p.threads_per_block ? p.threads_per_block : 256;
  if (tpb % 32 || tpb > (uint32_t)kMaxThreadsPerBlock) {
    g_last_error = "threads_per_block must be a multiple of 32 and at most " + std::to_string(kMaxThreadsPerBlock);
    return SCION_ERR_INVALID_ARG;
  }
  uint32_t smem_entries = p.smem_stack ? p.smem_stack : 16;
  if (smem_entries > 64) {
    g_last_error = "smem_stack exceeds 64 entries";
    return SCION_ERR_INVALID_ARG;
  }
  smem_entries = stack_entries(b, smem_entries, query);
  if (p.ordered_children > 3) {
    g_last_error = "ordered_children must be 0..3";
    return SCION_ERR_INVALID_ARG;
  }
  if (!on_bvh_device(b)) return SCION_ERR_INVALID_ARG;
  TraceKernel k = pick_kernel(b, query, 0, p.reg_stack);
  if (!k) {
    g_last_error = "this query is not offered for the BVH's layout";
    return SCION_ERR_UNSUPPORTED_LAYOUT;
  }
  const void *k_rays = kernel_view(rays), *k_out = kernel_view(out);
  if (!k_rays || !k_out) {
    g_last_error = "input and result buffers must be device memory of the current device or page-locked host memory";
    return SCION_ERR_INVALID_ARG;
  }
  L->k = k;
  L->tpb = tpb;
  L->smem = (size_t)tpb * smem_entries * stack_entry_bytes(b, query);
  TraceArgs &a = L->a;
  bvh_args(b, a);
  a.rays = reinterpret_cast<const float4 *>(k_rays);
  a.out = const_cast<void *>(k_out);
  a.n = n;
  a.max_steps = p.max_steps ? p.max_steps : 2u * (b->n_nodes + b->n_leaf_entries) + 64u;
  a.ordered = order_mode(p.ordered_children);
  a.smem_stack = smem_entries;
  a.refill_min = p.rays_per_fetch < 32 ? p.rays_per_fetch : 0u;
  set_raster(a, p.raster_width);
  a.status = b->d_scratch + 3;
  a.stats = nullptr;
  a.work = nullptr;
  a.exit_count = nullptr;
  L->ctas_param = p.ctas_per_sm;
  L->reg_stack = p.reg_stack;
  return SCION_OK;
}

// Grid of a prepared launch (persistent CTAs per SM x SMs, at most one CTA
// per tpb rays) and the launch itself.
scion_status issue_trace(TraceLaunch &L, cudaStream_t stream, TraceKernel k) {
  const int dev = current_device();
  scion_status st = ensure_smem_optin((const void *)k, L.smem, dev);
  if (st != SCION_OK) return st;
  uint32_t ctas = L.ctas_param;
  if (ctas == 0) {
    st = ctas_per_sm((const void *)k, L.tpb, L.smem, dev, &ctas);
    if (st != SCION_OK) return st;
  }
  L.grid = std::min<uint64_t>((uint64_t)ctas * device_sms(dev), (L.a.n + L.tpb - 1) / L.tpb);
  void *args[] = {&L.a};
  SCION_CUDA(cudaLaunchKernel((const void *)k, dim3((unsigned)L.grid), dim3(L.tpb), args, L.smem, stream));
  return SCION_OK;
}

scion_status launch_trace(scion_bvh b, const scion_ray *rays, uint64_t n, void *out,
                          const scion_trace_params *params, cudaStream_t stream, int query,
                          unsigned long long *stats = nullptr) {
  if (!b) return SCION_ERR_INVALID_ARG;
  if (n == 0) return SCION_OK;
  TraceLaunch L;
  scion_status st = prepare_trace(b, rays, n, out, params, query, &L);
  if (st != SCION_OK) return st;
  TraceKernel k = L.k;
  if (stats) {
    k = pick_kernel(b, query, 1, 0);
    if (!k) return SCION_ERR_UNSUPPORTED_LAYOUT;
  }
  const int slot = stream_slot(b, stream);
  if (slot < 0) {
    g_last_error = "more than 64 streams have traced this BVH";
    return SCION_ERR_INVALID_ARG;
  }
  uint32_t *sl = b->d_scratch + 4 + 4 * slot;
  L.a.work = reinterpret_cast<unsigned long long *>(sl);
  L.a.exit_count = sl + 2;
  L.a.stats = stats;
  return issue_trace(L, stream, k);
}



// Upload one packed BVH; on failure everything is freed and *out stays null.
scion_status upload_bvh(HostBVH &hb, uint64_t n_tris, uint64_t n_verts, bool indexed, cudaStream_t s,
                        scion_bvh *out) {
  scion_bvh b = new (std::nothrow) scion_bvh_s();
  if (!b) return SCION_ERR_OOM;
  b->desc = hb.desc;
  b->own_box = hb.own_box;
  b->n_tris = (uint32_t)n_tris;
  b->n_verts = (uint32_t)n_verts;
  b->indexed = indexed;
  b->n_nodes = hb.n_nodes;
  b->node_stride = hb.node_stride;
  b->n_leaf_entries = hb.n_leaf_entries;
  b->root_ref = hb.root_ref;
  b->depth = hb.depth;
  b->stack_need = hb.stack_need;
  for (int k = 0; k < 9; ++k) b->frame[k] = hb.frame[k];
  b->build_ms = hb.build_ms;
  b->logical_ms = hb.logical_ms;
  b->pack_ms = hb.pack_ms;
  cudaGetDevice(&b->device);
  uint64_t pb = 0, pi = 0;
  scion_status us = SCION_OK;
  if (us == SCION_OK) us = upload(&b->d_nodes, hb.nodes, s, &b->node_bytes);
  if (us == SCION_OK) us = upload(&b->d_nodes2, hb.nodes2, s, &b->node2_bytes);
  if (us == SCION_OK) us = upload(&b->d_prims, hb.prim_direct, s, &pb);
  if (us == SCION_OK) us = upload(&b->d_prim_ids, hb.prim_ids, s, &pi);
  if (us == SCION_OK) us = upload(&b->d_verts, hb.verts4, s, &b->vert_bytes);
  if (us == SCION_OK) us = upload(&b->d_idx, hb.indices, s, &b->idx_bytes);
  if (us == SCION_OK) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->d_scratch), kScratchBytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_scratch, 0, kScratchBytes, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) us = e == cudaErrorMemoryAllocation ? SCION_ERR_OOM : cuda_fail(e);
  }
  if (us != SCION_OK) {
    free_bvh(b);
    return us;
  }
  b->prim_bytes = host_prim_bytes(hb);
  *out = b;
  return SCION_OK;
}

// A BVH around buffers packed on the device (gpu_pack); takes them over.
scion_status adopt_bvh(DevicePacked &dp, const scion_layout_desc &desc, bool own_box, uint64_t n_tris,
                       uint64_t n_verts, bool indexed, cudaStream_t s, scion_bvh *out) {
  auto release = [&]() {
    void *bufs[] = {dp.nodes, dp.nodes2, dp.prims, dp.prim_ids, dp.verts4, dp.idx};
    for (void *p : bufs)
      if (p) cudaFree(p);
    dp = DevicePacked{};
  };
  scion_bvh b = new (std::nothrow) scion_bvh_s();
  if (!b) {
    release();
    return SCION_ERR_OOM;
  }
  b->desc = desc;
  b->own_box = own_box;
  b->n_tris = (uint32_t)n_tris;
  b->n_verts = (uint32_t)n_verts;
  b->indexed = indexed;
  b->n_nodes = dp.n_nodes;
  b->node_stride = dp.node_stride;
  b->n_leaf_entries = dp.n_leaf_entries;
  b->root_ref = dp.root_ref;
  b->depth = dp.depth;
  b->stack_need = dp.stack_need;
  for (int k = 0; k < 9; ++k) b->frame[k] = dp.frame[k];
  b->device = current_device();
  b->d_nodes = dp.nodes;
  b->d_nodes2 = dp.nodes2;
  b->d_prims = dp.prims;
  b->d_prim_ids = dp.prim_ids;
  b->d_verts = dp.verts4;
  b->d_idx = dp.idx;
  b->node_bytes = dp.node_bytes;
  b->node2_bytes = dp.node2_bytes;
  b->vert_bytes = dp.vert_bytes;
  b->idx_bytes = dp.idx_bytes;
  b->prim_bytes = dp.prim_direct_bytes + dp.prim_id_bytes + (desc.prim_ref == REF_INDIRECT ? dp.idx_bytes : 0);
  dp = DevicePacked{};  // the BVH owns the buffers now
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->d_scratch), kScratchBytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_scratch, 0, kScratchBytes, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_bvh(b);
    return e == cudaErrorMemoryAllocation ? SCION_ERR_OOM : cuda_fail(e);
  }
  *out = b;
  return SCION_OK;
}

// Host copies of device-resident inputs (a device-to-host boundary).
scion_status host_inputs(const float *verts, uint64_t n_verts, const uint32_t *indices, uint64_t n_tris,
                         cudaStream_t s, std::vector<float> *hv, std::vector<uint32_t> *hi,
                         const float **v, const uint32_t **ix) {
  *v = verts;
  *ix = indices;
  if (verts && is_device_ptr(verts)) {
    hv->resize(3 * n_verts);
    SCION_CUDA(cudaMemcpyAsync(hv->data(), verts, hv->size() * 4, cudaMemcpyDeviceToHost, s));
    SCION_CUDA(cudaStreamSynchronize(s));
    *v = hv->data();
  }
  if (indices && is_device_ptr(indices)) {
    hi->resize(3 * n_tris);
    SCION_CUDA(cudaMemcpyAsync(hi->data(), indices, hi->size() * 4, cudaMemcpyDeviceToHost, s));
    SCION_CUDA(cudaStreamSynchronize(s));
    *ix = hi->data();
  }
  return SCION_OK;
}

}  // namespace

extern "C" {

const char *scion_status_string(scion_status s) {
  switch (s) {
    case SCION_OK: return "ok";
    case SCION_ERR_INVALID_ARG: return "invalid argument";
    case SCION_ERR_UNSUPPORTED_LAYOUT: return "unsupported layout";
    case SCION_ERR_OOM: return "out of memory";
    case SCION_ERR_CUDA: return "CUDA error";
    case SCION_ERR_STACK_OVERFLOW: return "traversal stack overflow";
    case SCION_ERR_ITER_LIMIT: return "traversal step limit";
    case SCION_ERR_BAD_INPUT: return "bad input";
  }
  return "unknown status";
}

const char *scion_last_error(void) { return g_last_error.c_str(); }

scion_status scion_build(const float *verts, uint64_t n_verts, const uint32_t *indices,
                         uint64_t n_tris, const scion_layout_desc *desc, scion_stream stream,
                         scion_bvh *out) {
  if (!out) return SCION_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || (n_tris > 0 && !verts)) return SCION_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<float> hv;
  std::vector<uint32_t> hi;
  const float *v;
  const uint32_t *ix;
  scion_status st = host_inputs(verts, n_verts, indices, n_tris, s, &hv, &hi, &v, &ix);
  if (st != SCION_OK) return st;
  HostBVH hb;
  st = build_host(v, n_verts, ix, n_tris, desc, &hb);
  if (st != SCION_OK) return st;
  return upload_bvh(hb, n_tris, n_verts, ix != nullptr, s, out);
}

}  // extern "C"

namespace {

// GPU construction with packing on the host (the path for the layouts the
// GPU packer does not build, and a debug entry point that compares the two).
scion_status build_gpu_host_pack(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                                 const scion_layout_desc &d, bool own_box, cudaStream_t s, scion_bvh *out) {
  const auto t0 = std::chrono::steady_clock::now();
  HostBVH hb;
  try {
    // host copies for the packers (direct triangles, vertex tables) and the
    // index check, which must pass before any kernel reads through the indices
    std::vector<float> hv;
    std::vector<uint32_t> hi;
    const float *v;
    const uint32_t *ix;
    scion_status st = host_inputs(d_verts, n_verts, d_indices, n_tris, s, &hv, &hi, &v, &ix);
    if (st != SCION_OK) return st;
    if (ix)
      for (uint64_t i = 0; i < 3 * n_tris; ++i)
        if (ix[i] >= n_verts) return SCION_ERR_INVALID_ARG;
    LogicalBVH lb;
    double gpu_ms = 0.0;
    std::string err;
    st = lbvh_build(d_verts, n_verts, d_indices, n_tris, d.leaf_max, s, &lb, &gpu_ms, &err);
    if (st != SCION_OK) {
      g_last_error = err;
      return st;
    }
    const auto t1 = std::chrono::steady_clock::now();
    st = pack_bvh(BuildInput{v, n_verts, ix, n_tris}, lb, d, own_box, &hb, &err);
    if (st != SCION_OK) {
      g_last_error = err;
      return st;
    }
    hb.logical_ms = gpu_ms;
    hb.pack_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  } catch (const std::bad_alloc &) {
    g_last_error = "out of host memory";
    return SCION_ERR_OOM;
  }
  hb.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return upload_bvh(hb, n_tris, n_verts, d_indices != nullptr, s, out);
}

// Arguments of scion_build_gpu and its debug twin; fills the normalized
// descriptor.
scion_status check_build_gpu(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                             const scion_layout_desc *desc, scion_bvh *out, scion_layout_desc *d, bool *own_box) {
  if (!out) return SCION_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || (n_tris > 0 && !d_verts)) return SCION_ERR_INVALID_ARG;
  if (n_tris >= kMaxPrims || n_verts >= (1ull << 32)) return SCION_ERR_INVALID_ARG;
  if (!d_indices && n_verts != 3 * n_tris) return SCION_ERR_INVALID_ARG;
  if (n_tris > 0 && (!is_device_ptr(d_verts) || (d_indices && !is_device_ptr(d_indices)))) {
    g_last_error = "scion_build_gpu: vertices and indices must be device memory of the current device";
    return SCION_ERR_INVALID_ARG;
  }
  return normalize_desc(*desc, d, own_box);
}

}  // namespace

extern "C" {

scion_status scion_build_gpu(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices,
                             uint64_t n_tris, const scion_layout_desc *desc, scion_stream stream,
                             scion_bvh *out) {
  scion_layout_desc d;
  bool own_box = false;
  scion_status st = check_build_gpu(d_verts, n_verts, d_indices, n_tris, desc, out, &d, &own_box);
  if (st != SCION_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!gpu_pack_supported(d, own_box)) return build_gpu_host_pack(d_verts, n_verts, d_indices, n_tris, d, own_box, s, out);
  std::string err;
  bool in_range = true;
  st = gpu_indices_in_range(d_indices, n_tris, n_verts, s, &in_range, &err);
  if (st != SCION_OK) {
    g_last_error = err;
    return st;
  }
  if (!in_range) {
    g_last_error = "scion_build_gpu: a vertex index is out of range";
    return SCION_ERR_INVALID_ARG;
  }
  LbvhTree t;
  st = lbvh_build_tree(d_verts, n_verts, d_indices, n_tris, d.leaf_max, s, &t, &err);
  if (st != SCION_OK) {
    g_last_error = err;
    return st;
  }
  const auto t1 = std::chrono::steady_clock::now();
  DevicePacked dp;
  st = gpu_pack(t, d_verts, n_verts, d_indices, n_tris, d, own_box, s, &dp, &err);
  if (st != SCION_OK) {
    g_last_error = err;
    return st;
  }
  const double pack_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  st = adopt_bvh(dp, d, own_box, n_tris, n_verts, d_indices != nullptr, s, out);
  if (st != SCION_OK) return st;
  (*out)->logical_ms = t.gpu_ms;
  (*out)->pack_ms = pack_ms;
  (*out)->build_ms = t.gpu_ms + pack_ms;
  return SCION_OK;
}

scion_status scion_debug_build_gpu_host_pack(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices,
                                             uint64_t n_tris, const scion_layout_desc *desc, scion_stream stream,
                                             scion_bvh *out) {
  scion_layout_desc d;
  bool own_box = false;
  scion_status st = check_build_gpu(d_verts, n_verts, d_indices, n_tris, desc, out, &d, &own_box);
  if (st != SCION_OK) return st;
  return build_gpu_host_pack(d_verts, n_verts, d_indices, n_tris, d, own_box, reinterpret_cast<cudaStream_t>(stream),
                             out);
}

scion_status scion_debug_bvh_bytes(scion_bvh b, void *nodes, uint64_t nodes_cap, void *nodes2, uint64_t nodes2_cap,
                                   void *prims, uint64_t prims_cap, uint64_t *sizes) {
  if (!b || !sizes) return SCION_ERR_INVALID_ARG;
  const uint64_t pb = b->desc.prim_ref == REF_DIRECT ? 48ull * b->n_leaf_entries : 4ull * b->n_leaf_entries;
  sizes[0] = b->node_bytes;
  sizes[1] = b->node2_bytes;
  sizes[2] = pb;
  if ((nodes && nodes_cap < b->node_bytes) || (nodes2 && nodes2_cap < b->node2_bytes) || (prims && prims_cap < pb))
    return SCION_ERR_INVALID_ARG;
  if (!on_bvh_device(b)) return SCION_ERR_INVALID_ARG;
  const void *src = b->desc.prim_ref == REF_DIRECT ? b->d_prims : b->d_prim_ids;
  cudaError_t e = cudaSuccess;
  if (nodes && b->node_bytes) e = cudaMemcpy(nodes, b->d_nodes, b->node_bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && nodes2 && b->node2_bytes) e = cudaMemcpy(nodes2, b->d_nodes2, b->node2_bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && prims && pb) e = cudaMemcpy(prims, src, pb, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  return SCION_OK;
}

scion_status scion_refit(scion_bvh bvh, const float *d_verts, uint64_t n_verts, scion_stream stream) {
  if (!bvh || n_verts != bvh->n_verts || (n_verts > 0 && !d_verts)) return SCION_ERR_INVALID_ARG;
  if (n_verts > 0 && !is_device_ptr(d_verts)) {
    g_last_error = "scion_refit: vertices must be device memory";
    return SCION_ERR_INVALID_ARG;
  }
  if (!on_bvh_device(bvh)) return SCION_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  scion_bvh b = bvh;
  if (!b->d_refit_parent && b->n_nodes > 0) {
    const size_t n = b->n_nodes;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->d_refit_parent), n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_refit_pending), n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_refit_boxes, n * 6 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_refit_frame), 16 * sizeof(float));
    if (e != cudaSuccess) {
      cudaFree(b->d_refit_parent);
      cudaFree(b->d_refit_pending);
      cudaFree(b->d_refit_boxes);
      cudaFree(b->d_refit_frame);
      b->d_refit_parent = b->d_refit_pending = nullptr;
      b->d_refit_boxes = nullptr;
      b->d_refit_frame = nullptr;
      return e == cudaErrorMemoryAllocation ? SCION_ERR_OOM : cuda_fail(e);
    }
  }
  RefitBuffers rb;
  rb.nodes = b->d_nodes;
  rb.nodes2 = b->d_nodes2;
  rb.prims = b->d_prims;
  rb.verts4 = b->d_verts;
  rb.prim_ids = static_cast<const uint32_t *>(b->d_prim_ids);
  rb.tri_idx = static_cast<const uint32_t *>(b->d_idx);
  rb.n_nodes = b->n_nodes;
  rb.node_stride = b->node_stride;
  rb.n_leaf_entries = b->n_leaf_entries;
  rb.n_verts = b->n_verts;
  rb.own_box = b->own_box;
  rb.desc = b->desc;
  rb.parent = b->d_refit_parent;
  rb.pending = b->d_refit_pending;
  rb.boxes = b->d_refit_boxes;
  rb.frame = b->d_refit_frame;
  rb.status = b->d_scratch + 3;
  SCION_CUDA(refit_launch(rb, d_verts, s));
  if (prec_has_frame(b->desc.box_prec) && b->n_nodes > 0) {
    // the traversal takes the grid as a launch argument: read it back
    SCION_CUDA(cudaMemcpyAsync(b->frame, b->d_refit_frame, 9 * sizeof(float), cudaMemcpyDeviceToHost, s));
    SCION_CUDA(cudaStreamSynchronize(s));
  }
  return SCION_OK;
}

scion_status scion_bvh_build_times(scion_bvh bvh, double *logical_ms, double *pack_ms) {
  if (!bvh) return SCION_ERR_INVALID_ARG;
  if (logical_ms) *logical_ms = bvh->logical_ms;
  if (pack_ms) *pack_ms = bvh->pack_ms;
  return SCION_OK;
}

scion_status scion_build_many(const float *verts, uint64_t n_verts, const uint32_t *indices,
                              uint64_t n_tris, const scion_layout_desc *descs, uint32_t n_desc,
                              scion_stream stream, scion_bvh *out) {
  if (!out || !descs || n_desc == 0) return SCION_ERR_INVALID_ARG;
  for (uint32_t i = 0; i < n_desc; ++i) out[i] = nullptr;
  if (n_tris > 0 && !verts) return SCION_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<float> hv;
  std::vector<uint32_t> hi;
  const float *v;
  const uint32_t *ix;
  scion_status st = host_inputs(verts, n_verts, indices, n_tris, s, &hv, &hi, &v, &ix);
  if (st != SCION_OK) return st;
  std::vector<HostBVH> hbs;
  st = build_host_many(v, n_verts, ix, n_tris, descs, n_desc, &hbs);
  if (st != SCION_OK) return st;
  for (uint32_t i = 0; i < n_desc; ++i) {
    st = upload_bvh(hbs[i], n_tris, n_verts, ix != nullptr, s, &out[i]);
    if (st != SCION_OK) {
      for (uint32_t j = 0; j < i; ++j) {
        free_bvh(out[j]);
        out[j] = nullptr;
      }
      return st;
    }
    hbs[i] = HostBVH();  // release host memory early
  }
  return SCION_OK;
}

scion_status scion_bvh_info(scion_bvh b, uint64_t *node_bytes, uint64_t *prim_bytes, uint32_t *depth,
                            uint32_t *n_nodes) {
  if (!b) return SCION_ERR_INVALID_ARG;
  if (node_bytes) *node_bytes = b->node_bytes + b->node2_bytes;
  if (prim_bytes) *prim_bytes = b->prim_bytes;
  if (depth) *depth = b->depth;
  if (n_nodes) *n_nodes = b->n_nodes;
  return SCION_OK;
}

scion_status scion_trace_closest(scion_bvh b, const scion_ray *d_rays, uint64_t n, scion_hit *d_hits,
                                 const scion_trace_params *params, scion_stream stream) {
  return launch_trace(b, d_rays, n, d_hits, params, reinterpret_cast<cudaStream_t>(stream), kQueryClosest);
}

scion_status scion_trace_any(scion_bvh b, const scion_ray *d_rays, uint64_t n, uint32_t *d_occluded,
                             const scion_trace_params *params, scion_stream stream) {
  return launch_trace(b, d_rays, n, d_occluded, params, reinterpret_cast<cudaStream_t>(stream), kQueryAny);
}

scion_status scion_query_closest_point(scion_bvh b, const scion_point *d_points, uint64_t n,
                                      scion_closest_point *d_out, const scion_trace_params *params,
                                      scion_stream stream) {
  return launch_trace(b, reinterpret_cast<const scion_ray *>(d_points), n, d_out, params,
                      reinterpret_cast<cudaStream_t>(stream), kQueryPoint);
}

scion_status scion_trace_stats(scion_bvh b, const scion_ray *d_rays, uint64_t n, uint32_t query,
                              void *d_out, const scion_trace_params *params, scion_stream stream,
                              uint64_t *d_counters) {
  if (!d_counters || query > 2 || (reinterpret_cast<uintptr_t>(d_counters) & 7u)) return SCION_ERR_INVALID_ARG;
  if (n > 0 && !is_device_ptr(d_counters)) {  // the kernels add to them with device atomics
    g_last_error = "d_counters must be device memory";
    return SCION_ERR_INVALID_ARG;
  }
  return launch_trace(b, d_rays, n, d_out, params, reinterpret_cast<cudaStream_t>(stream), (int)query,
                      reinterpret_cast<unsigned long long *>(d_counters));
}

scion_status scion_trace_backward(scion_bvh b, const scion_ray *d_rays, const scion_hit *d_hits,
                                  const float *d_grad_tuv, uint64_t n, float *d_grad_verts,
                                  scion_ray *d_grad_rays, scion_stream stream) {
  if (!b || (n > 0 && (!d_rays || !d_hits || !d_grad_tuv || !d_grad_verts))) return SCION_ERR_INVALID_ARG;
  if (n == 0) return SCION_OK;
  if ((reinterpret_cast<uintptr_t>(d_rays) & 15u) || (reinterpret_cast<uintptr_t>(d_hits) & 15u) ||
      (reinterpret_cast<uintptr_t>(d_grad_rays) & 15u) || (reinterpret_cast<uintptr_t>(d_grad_tuv) & 3u) ||
      (reinterpret_cast<uintptr_t>(d_grad_verts) & 3u)) {
    g_last_error = "scion_trace_backward: misaligned buffer";
    return SCION_ERR_INVALID_ARG;
  }
  if (!on_bvh_device(b)) return SCION_ERR_INVALID_ARG;
  // the kernel scatters into the gradients with device atomics: device memory only
  if (!is_device_ptr(d_rays) || !is_device_ptr(d_hits) || !is_device_ptr(d_grad_tuv) ||
      !is_device_ptr(d_grad_verts) || (d_grad_rays && !is_device_ptr(d_grad_rays))) {
    g_last_error = "scion_trace_backward takes device buffers";
    return SCION_ERR_INVALID_ARG;
  }
  BackwardArgs a;
  a.rays = reinterpret_cast<const float *>(d_rays);
  a.hits = reinterpret_cast<const uint32_t *>(d_hits);
  a.grad_tuv = d_grad_tuv;
  a.verts = static_cast<const float4 *>(b->d_verts);
  a.tri_idx = static_cast<const uint32_t *>(b->d_idx);
  a.grad_verts = d_grad_verts;
  a.grad_rays = reinterpret_cast<float *>(d_grad_rays);
  a.n = n;
  a.n_tris = b->n_tris;
  int dev = 0;
  cudaGetDevice(&dev);
  SCION_CUDA(launch_backward(a, device_sms(dev), reinterpret_cast<cudaStream_t>(stream)));
  return SCION_OK;
}

// ---------------------------------------------------------------- batched
struct scion_batch_s {
  BatchScene *d_scenes = nullptr;   // scene table (device)
  uint32_t *d_counters = nullptr;   // u64 work counter + u32 exit counter
  uint32_t n_scenes = 0;            // scenes in the multi-family launch
  unsigned long long total = 0;     // padded global ray count
  uint32_t threads = 256, smem_stack = 16, grid = 0;
  // scenes whose layout the batched kernel does not handle: plain launches
  std::vector<scion_bvh> rest_bvh;
  std::vector<const scion_ray *> rest_rays;
  std::vector<uint64_t> rest_n;
  std::vector<scion_hit *> rest_hits;
  std::vector<scion_trace_params> rest_params;
};

scion_status scion_batch_create(const scion_bvh *bvhs, const scion_ray *const *d_rays, const uint64_t *n,
                                scion_hit *const *d_hits, uint32_t n_scenes,
                                const scion_trace_params *per_scene, scion_stream stream, scion_batch *out) {
  if (!out) return SCION_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_scenes > 0 && (!bvhs || !d_rays || !n || !d_hits)) return SCION_ERR_INVALID_ARG;
  scion_batch bt = new (std::nothrow) scion_batch_s();
  if (!bt) return SCION_ERR_OOM;
  std::vector<BatchScene> table;
  unsigned long long total = 0;
  if (per_scene) {
    bt->threads = per_scene[0].threads_per_block ? per_scene[0].threads_per_block : 256;
    bt->smem_stack = per_scene[0].smem_stack ? per_scene[0].smem_stack : 16;
  }
  if (bt->threads % 32 || bt->threads > (uint32_t)kMaxThreadsPerBlock || bt->smem_stack > 64) {
    delete bt;
    return SCION_ERR_INVALID_ARG;
  }
  for (uint32_t i = 0; i < n_scenes; ++i) {
    scion_bvh b = bvhs[i];
    scion_trace_params p{};
    if (per_scene) p = per_scene[i];
    if (!b || (n[i] > 0 && (!d_rays[i] || !d_hits[i])) || p.ordered_children > 3 || p.rays_per_fetch > 32 ||
        (reinterpret_cast<uintptr_t>(d_rays[i]) & 15u) || (reinterpret_cast<uintptr_t>(d_hits[i]) & 15u)) {
      g_last_error = "scion_batch_create: scene " + std::to_string(i) + ": bad argument";
      delete bt;
      return SCION_ERR_INVALID_ARG;
    }
    if (p.raster_width != 0 || p.reg_stack != 0) {
      g_last_error = "scion_batch_create: raster_width and reg_stack are plain-launch parameters (scene " +
                     std::to_string(i) + ")";
      delete bt;
      return SCION_ERR_INVALID_ARG;
    }
    if (n[i] == 0) continue;
    if (!on_bvh_device(b)) {
      delete bt;
      return SCION_ERR_INVALID_ARG;
    }
    const void *k_rays = kernel_view(d_rays[i]), *k_hits = kernel_view(d_hits[i]);
    if (!k_rays || !k_hits) {
      g_last_error = "ray and result buffers must be device memory or page-locked host memory";
      delete bt;
      return SCION_ERR_INVALID_ARG;
    }
    const int fam = batched_family(b->own_box ? 1u : 0u, b->desc);
    if (fam < 0) {
      bt->rest_bvh.push_back(b);
      bt->rest_rays.push_back(d_rays[i]);
      bt->rest_n.push_back(n[i]);
      bt->rest_hits.push_back(d_hits[i]);
      bt->rest_params.push_back(p);
      continue;
    }
    BatchScene sc{};
    TraceArgs &a = sc.a;
    bvh_args(b, a);
    a.rays = reinterpret_cast<const float4 *>(k_rays);
    a.out = const_cast<void *>(k_hits);
    a.n = n[i];
    a.max_steps = p.max_steps ? p.max_steps : 2u * (b->n_nodes + b->n_leaf_entries) + 64u;
    a.ordered = order_mode(p.ordered_children);
    a.smem_stack = bt->smem_stack;
    a.refill_min = p.rays_per_fetch < 32 ? p.rays_per_fetch : 0u;
    a.status = b->d_scratch + 3;
    sc.begin = total;
    sc.family = (uint32_t)fam;
    total += (n[i] + kBatchUnit - 1) / kBatchUnit * kBatchUnit;
    table.push_back(sc);
  }
  bt->n_scenes = (uint32_t)table.size();
  bt->total = total;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&bt->d_counters), 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->d_counters, 0, 16, s);
  if (e == cudaSuccess && !table.empty()) {
    e = cudaMalloc(reinterpret_cast<void **>(&bt->d_scenes), table.size() * sizeof(BatchScene));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bt->d_scenes, table.data(), table.size() * sizeof(BatchScene), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && !table.empty()) {
    const size_t smem = (size_t)bt->threads * bt->smem_stack * sizeof(uint2);
    int nb = 0;
    int dev = current_device();
    const scion_status so = ensure_smem_optin(batched_kernel_ptr(), smem, dev);
    if (so != SCION_OK) {
      if (bt->d_counters) cudaFree(bt->d_counters);
      if (bt->d_scenes) cudaFree(bt->d_scenes);
      delete bt;
      return so;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_kernel_ptr(), (int)bt->threads, smem);
    // one unit per warp at a time: more CTAs than units would only idle
    const uint64_t per_cta = (uint64_t)kBatchUnit * (bt->threads / 32);
    const uint64_t want = ((uint64_t)total + per_cta - 1) / per_cta;
    bt->grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)std::max(nb, 1) * device_sms(dev), want));
  }
  if (e != cudaSuccess) {
    if (bt->d_counters) cudaFree(bt->d_counters);
    if (bt->d_scenes) cudaFree(bt->d_scenes);
    delete bt;
    if (e == cudaErrorMemoryAllocation) return SCION_ERR_OOM;
    return cuda_fail(e);
  }
  *out = bt;
  return SCION_OK;
}

scion_status scion_batch_launch(scion_batch bt, scion_stream stream) {
  if (!bt) return SCION_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (bt->n_scenes > 0)
    SCION_CUDA(launch_batched(bt->d_scenes, bt->n_scenes, bt->total,
                              reinterpret_cast<unsigned long long *>(bt->d_counters), bt->d_counters + 2,
                              bt->smem_stack, bt->threads, bt->grid, s));
  for (size_t i = 0; i < bt->rest_bvh.size(); ++i) {
    scion_status st = launch_trace(bt->rest_bvh[i], bt->rest_rays[i], bt->rest_n[i], bt->rest_hits[i],
                                   &bt->rest_params[i], s, kQueryClosest);
    if (st != SCION_OK) return st;
  }
  return SCION_OK;
}

void scion_batch_destroy(scion_batch bt) {
  if (!bt) return;
  if (bt->d_counters) cudaFree(bt->d_counters);
  if (bt->d_scenes) cudaFree(bt->d_scenes);
  delete bt;
}

scion_status scion_batch_info(scion_batch bt, uint32_t *batched_scenes, uint32_t *plain_scenes) {
  if (!bt) return SCION_ERR_INVALID_ARG;
  if (batched_scenes) *batched_scenes = bt->n_scenes;
  if (plain_scenes) *plain_scenes = (uint32_t)bt->rest_bvh.size();
  return SCION_OK;
}

scion_status scion_trace_batched(const scion_bvh *bvhs, const scion_ray *const *d_rays, const uint64_t *n,
                                 scion_hit *const *d_hits, uint32_t n_scenes,
                                 const scion_trace_params *per_scene, scion_stream stream) {
  scion_batch bt = nullptr;
  scion_status st = scion_batch_create(bvhs, d_rays, n, d_hits, n_scenes, per_scene, stream, &bt);
  if (st != SCION_OK) return st;
  st = scion_batch_launch(bt, stream);
  // the table must outlive the launch: wait for it before releasing
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  scion_batch_destroy(bt);
  if (st != SCION_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e);
  return SCION_OK;
}

scion_status scion_get_status(scion_bvh b, scion_stream stream, scion_status *device_status) {
  if (!b || !device_status) return SCION_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  SCION_CUDA(cudaMemcpyAsync(&v, b->d_scratch + 3, 4, cudaMemcpyDeviceToHost, s));
  SCION_CUDA(cudaStreamSynchronize(s));
  if (v) {
    SCION_CUDA(cudaMemsetAsync(b->d_scratch + 3, 0, 4, s));
    SCION_CUDA(cudaStreamSynchronize(s));
  }
  *device_status = (scion_status)v;
  return SCION_OK;
}

void scion_destroy(scion_bvh b) { free_bvh(b); }

// ---------------------------------------------------------------- debug ABI
struct scion_host_bvh_s {
  HostBVH hb;
};

scion_status scion_debug_build_host(const float *verts, uint64_t n_verts, const uint32_t *indices,
                                    uint64_t n_tris, const scion_layout_desc *desc, scion_host_bvh *out) {
  if (!out) return SCION_ERR_INVALID_ARG;
  *out = nullptr;
  scion_host_bvh h = new (std::nothrow) scion_host_bvh_s();
  if (!h) return SCION_ERR_OOM;
  scion_status st = build_host(verts, n_verts, indices, n_tris, desc, &h->hb);
  if (st != SCION_OK) {
    delete h;
    return st;
  }
  *out = h;
  return SCION_OK;
}

scion_status scion_debug_host_stats(scion_host_bvh h, scion_debug_info *info) {
  if (!h || !info) return SCION_ERR_INVALID_ARG;
  const HostBVH &b = h->hb;
  info->n_nodes = b.n_nodes;
  info->node_stride = b.node_stride;
  info->n_leaf_entries = b.n_leaf_entries;
  info->root_ref = b.root_ref;
  info->depth = b.depth;
  info->stack_need = b.stack_need;
  info->own_box = b.own_box ? 1u : 0u;
  info->node2_bytes = (uint32_t)b.nodes2.size();
  info->node_bytes = b.nodes.size() + b.nodes2.size();
  info->prim_bytes = host_prim_bytes(b);
  info->vert_bytes = b.verts4.size() * 4;
  info->build_ms = b.build_ms;
  return SCION_OK;
}

scion_status scion_debug_host_decode(scion_host_bvh h, uint32_t *kind, uint32_t *a, uint32_t *c,
                                     float *boxes, float *own_boxes, uint32_t *leaf_ids) {
  if (!h || !kind || !a || !c || !boxes || !own_boxes || !leaf_ids) return SCION_ERR_INVALID_ARG;
  const HostBVH &hb = h->hb;
  for (uint32_t i = 0; i < hb.n_nodes; ++i) {
    DecodedChild ch[8];
    Box3 own{};
    std::memset(ch, 0, sizeof(ch));
    const int nc = decode_node(hb, i, ch, &own);
    for (int k = 0; k < 8; ++k) {
      const size_t o = (size_t)i * 8 + k;
      kind[o] = k < nc ? (uint32_t)ch[k].kind : 0u;
      a[o] = ch[k].kind == 1 ? ch[k].node : ch[k].first;
      c[o] = ch[k].kind == 2 ? ch[k].count : 0u;
      for (int q = 0; q < 3; ++q) {
        boxes[o * 6 + q] = ch[k].box.lo[q];
        boxes[o * 6 + 3 + q] = ch[k].box.hi[q];
      }
    }
    for (int q = 0; q < 3; ++q) {
      own_boxes[(size_t)i * 6 + q] = own.lo[q];
      own_boxes[(size_t)i * 6 + 3 + q] = own.hi[q];
    }
  }
  if (hb.desc.box_prec == PREC_SLAB && hb.n_nodes > 0) {
    // carried boxes top-down (parents precede children in every node order):
    // the root's is the frame, a child's is its parent's with one plane moved
    for (int q = 0; q < 6; ++q) own_boxes[q] = hb.frame[q];
    for (uint32_t i = 0; i < hb.n_nodes; ++i) {
      if (kind[(size_t)i * 8] != 1) continue;
      const uint8_t *p = hb.nodes.data() + (size_t)i * kSlabNodeBytes;
      const uint32_t ax = bin_meta_axis(get_u32(p + 12));
      const uint32_t l = a[(size_t)i * 8], r = a[(size_t)i * 8 + 1];
      for (int q = 0; q < 6; ++q) {
        own_boxes[(size_t)l * 6 + q] = own_boxes[(size_t)i * 6 + q];
        own_boxes[(size_t)r * 6 + q] = own_boxes[(size_t)i * 6 + q];
      }
      own_boxes[(size_t)l * 6 + 3 + ax] = get_f32(p);
      own_boxes[(size_t)r * 6 + ax] = get_f32(p + 4);
    }
  }
  for (uint32_t i = 0; i < hb.n_leaf_entries; ++i) {
    if (hb.desc.prim_ref == REF_DIRECT) std::memcpy(&leaf_ids[i], &hb.prim_direct[(size_t)i * 12 + 3], 4);
    else leaf_ids[i] = hb.prim_ids[i];
  }
  return SCION_OK;
}

scion_status scion_debug_set_bvh_device(scion_bvh b, int device) {
  if (!b || device < 0) return SCION_ERR_INVALID_ARG;
  b->device = device;
  return SCION_OK;
}

uint64_t scion_debug_raster_slots(uint64_t n, uint32_t raster_width) {
  if (n == 0) return 0;
  TraceArgs a{};
  a.n = n;
  set_raster(a, raster_width);
  return a.n_work;
}

scion_status scion_debug_host_raw(scion_host_bvh h, void *nodes, uint64_t nodes_cap, void *nodes2,
                                  uint64_t nodes2_cap, float *frame) {
  if (!h || !frame) return SCION_ERR_INVALID_ARG;
  const HostBVH &hb = h->hb;
  if (nodes_cap < hb.nodes.size() || nodes2_cap < hb.nodes2.size()) return SCION_ERR_INVALID_ARG;
  if ((!hb.nodes.empty() && !nodes) || (!hb.nodes2.empty() && !nodes2)) return SCION_ERR_INVALID_ARG;
  if (!hb.nodes.empty()) std::memcpy(nodes, hb.nodes.data(), hb.nodes.size());
  if (!hb.nodes2.empty()) std::memcpy(nodes2, hb.nodes2.data(), hb.nodes2.size());
  for (int k = 0; k < 9; ++k) frame[k] = hb.frame[k];
  return SCION_OK;
}

void scion_debug_host_destroy(scion_host_bvh h) { delete h; }

uint32_t scion_debug_f16_round(float x, int dir) {
  return dir < 0 ? f32_to_f16_down(x) : f32_to_f16_up(x);
}

float scion_debug_f16_decode(uint32_t h) { return f16_to_f32((uint16_t)h); }

}  // extern "C"

// ---------------------------------------------------------------- allocation-free closest hit
// Some callers must not allocate device memory while they trace: a host
// application that hands all device memory to its own arena up front and
// forbids any later allocation, or a latency-bound thread that must not enter
// the driver's allocator (cudaMalloc can synchronize the device).
// scion_trace_closest_noalloc serves them: the traversal's per-launch work
// counters live in the fixed array below, reserved once when the library's
// device code is loaded, instead of in memory that scion_build allocated with
// the BVH. The kernel itself is the same closest-hit kernel.
namespace {
constexpr size_t kStaticScratchBytes = 256;          // reserved per device until exit
constexpr size_t kStaticScratchUsed = 16;            // u64 work counter + u32 exit counter
constexpr uint64_t kStaticMaxRays = 1ull << 62;      // the 64-bit counter must not wrap
static_assert(kStaticScratchUsed <= kStaticScratchBytes, "static scratch too small");
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once
// per device; in host code the symbol itself is only a host-side stand-in).
scion_status static_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) {
    g_last_error = "device ordinal out of range for the static scratch table";
    return SCION_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SCION_OK;
}
}  // namespace

extern "C" scion_status scion_trace_closest_noalloc(scion_bvh b, const scion_ray *rays, uint64_t n,
                                                    scion_hit *hits, const scion_trace_params *params,
                                                    scion_stream stream) {
  if (!b) return SCION_ERR_INVALID_ARG;
  if (n >= kStaticMaxRays) {
    g_last_error = "scion_trace_closest_noalloc: n exceeds the static scratch counter range (2^62 rays)";
    return SCION_ERR_INVALID_ARG;
  }
  if (n == 0) return SCION_OK;
  // the same checks and set-up as scion_trace_closest, then the counters of
  // the static array instead of the BVH's
  TraceLaunch L;
  scion_status st = prepare_trace(b, rays, n, hits, params, kQueryClosest, &L);
  if (st != SCION_OK) return st;
  void *scratch = nullptr;
  st = static_scratch(&scratch);
  if (st != SCION_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the counters must start at zero; they keep the previous call's values
  SCION_CUDA(cudaMemsetAsync(scratch, 0, kStaticScratchUsed, s));
  L.a.work = static_cast<unsigned long long *>(scratch);
  L.a.exit_count = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(scratch) + 8);
  return issue_trace(L, s, L.k);  // device errors still go to the BVH's status word
}
