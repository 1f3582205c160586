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

#include "builder.h"

namespace scion {

// Build from device vertex (float[n_verts][3]) and optional device index
// (u32[n_tris][3]) arrays. Triangles with a non-finite vertex are left out.
// Device scratch is allocated and freed inside; the call synchronises
// `stream` before returning. *gpu_ms receives the device time of the build
// kernels (bounds, codes, sort, tree, boxes), without the download.
scion_status lbvh_build(const float *d_verts, uint64_t n_verts, const uint32_t *d_indices, uint64_t n_tris,
                        uint32_t leaf_max, cudaStream_t stream, LogicalBVH *out, double *gpu_ms, std::string *err);

}  // namespace scion
