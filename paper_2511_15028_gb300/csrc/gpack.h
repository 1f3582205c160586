// Packing on the GPU: the layout build (Section 5.1's second phase, the
// count-then-fill constructor of App. F) applied to the logical BVH2 that the
// GPU builder leaves in device memory, so a GPU build never moves the tree
// through host memory. The packed bytes are those of the host packer
// (builder.cpp) for the same logical tree: the same greedy collapse to width
// W, the same node orders and the same host/device codecs (codec.h).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "builder.h"
#include "lbvh.h"

namespace scion {

// A packed BVH in device memory. The buffers belong to the caller once
// gpu_pack returns SCION_OK (cudaFree each); on error gpu_pack frees them.
struct DevicePacked {
  void *nodes = nullptr, *nodes2 = nullptr, *prims = nullptr, *prim_ids = nullptr;
  void *verts4 = nullptr, *idx = nullptr;
  uint64_t node_bytes = 0, node2_bytes = 0, prim_direct_bytes = 0, prim_id_bytes = 0, vert_bytes = 0,
           idx_bytes = 0;
  uint32_t n_nodes = 0, node_stride = 0, n_leaf_entries = 0, root_ref = kEmptyRef, depth = 0, stack_need = 0;
  float frame[9] = {};
  double pack_ms = 0.0;  // device time of the packing kernels
};

// Whether every index of the device array d_indices (u32[n_tris][3]) is
// below n_verts, checked on the GPU (before any kernel reads through them).
scion_status gpu_indices_in_range(const uint32_t *d_indices, uint64_t n_tris, uint64_t n_verts, cudaStream_t stream,
                                  bool *ok, std::string *err);

// Layouts gpu_pack builds: every width, box precision, box layout and child
// and primitive reference of the children-in-parent nodes and of the
// own-box f32 / q16 / eq10 nodes, in DFS or BFS order. The treelet order and
// the shared-slab node are packed on the host.
bool gpu_pack_supported(const scion_layout_desc &d, bool own_box);

// Pack the device tree `t` (over the triangles of d_verts / d_indices, device
// memory) into the normalized layout `d` on `stream`; synchronises it before
// returning. Errors: as the host packer for the same tree (UNSUPPORTED_LAYOUT
// for an order that breaks the child reference encoding or too many nodes
// for a quantised node, BAD_INPUT for a code that cannot enclose its box,
// INVALID_ARG for too many nodes), OOM, CUDA; *err says which.
scion_status gpu_pack(const LbvhTree &t, const float *d_verts, uint64_t n_verts, const uint32_t *d_indices,
                      uint64_t n_tris, const scion_layout_desc &d, bool own_box, cudaStream_t stream,
                      DevicePacked *out, std::string *err);

}  // namespace scion
