// GPU construction of the logical BVH2 (the "construction" phase that the
// paper keeps apart from the layout build, Section 5 footnote and Section 5.1
// two-phase construction; Section 2: topology is orthogonal to layout).
//
// Linear BVH: triangles are ordered along a 30-bit Morton curve of their box
// centres (Lauterbach et al. 2009), the binary radix tree over the sorted
// codes is built with one thread per interior node (Karras 2012), and boxes
// are computed bottom-up. A subtree of at most leaf_max triangles (a
// contiguous range of the sorted order) becomes one leaf where the surface
// area heuristic prefers it to the subtree's best split. The result is the
// same LogicalBVH the host SAH builder produces, so every packer and layout
// applies unchanged.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "builder.h"

namespace scion {

// The logical BVH2 as the GPU builds it, left in device memory: the binary
// radix tree over the nv valid triangles in Morton order. Interior node i in
// [0, nv-2] has children left[i], right[i]; node ids >= nv-1 are radix
// leaves (leaf k = node nv-1+k holds the sorted triangle ids[k]). An
// interior node with whole[i] = 1 is a logical leaf over the sorted
// triangles rlo[i]..rhi[i]; the logical tree is what is reachable from node
// 0 without entering such a node. Boxes nlo/nhi: 3 floats per node (2nv-1
// nodes). Node 0 is the root (a radix leaf when nv = 1). Owns its device
// memory; freed with the object.
struct LbvhTree {
  uint32_t nv = 0;
  const uint32_t *ids = nullptr;
  const uint32_t *left = nullptr, *right = nullptr, *rlo = nullptr, *rhi = nullptr;
  const uint8_t *axis = nullptr, *whole = nullptr;
  const float *nlo = nullptr, *nhi = nullptr;
  double gpu_ms = 0.0;  // device time of the build kernels
  std::vector<void *> owned;
  LbvhTree() = default;
  LbvhTree(const LbvhTree &) = delete;
  LbvhTree &operator=(const LbvhTree &) = delete;
  ~LbvhTree();
};

// Build from device vertex (float[n_verts][3]) and optional device index
// (u32[n_tris][3]) arrays. Triangles with a non-finite vertex are left out.
// Synchronises `stream` before returning.
scion_status lbvh_build_tree(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                             uint32_t leaf_max, cudaStream_t stream, LbvhTree *out, std::string *err);

// The tree in host memory, as the host packers take it.
scion_status lbvh_download(const LbvhTree &t, cudaStream_t stream, LogicalBVH *out, std::string *err);

// Both steps. *gpu_ms receives the device time of the build kernels (bounds,
// codes, sort, tree, boxes, leaf choice), without the download.
scion_status lbvh_build(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                        uint32_t leaf_max, cudaStream_t stream, LogicalBVH *out, double *gpu_ms, std::string *err);

}  // namespace scion
