// Refit of a packed BVH to new vertex positions (same triangles, same tree):
// boxes are recomputed bottom-up on the GPU and re-encoded in place in the
// BVH's own layout with the codecs the host packer uses (codec.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/scion.h"

namespace scion {

struct RefitBuffers {
  void *nodes, *nodes2, *prims, *verts4;  // the BVH's device buffers
  const uint32_t *prim_ids, *tri_idx;
  uint32_t n_nodes, node_stride, n_leaf_entries;
  uint64_t n_verts;
  bool own_box;
  scion_layout_desc desc;
  // refit scratch (device): n_nodes parents and counters, n_nodes boxes of
  // 24 bytes, 12 floats of world grid (q16/eq10)
  uint32_t *parent, *pending;
  void *boxes;
  float *frame;
  uint32_t *status;  // the BVH's device status word (encoding failures)
};

// Enqueue the refit kernels on `s`; new vertices: DEVICE float[n_verts][3].
cudaError_t refit_launch(const RefitBuffers &b, const float *d_new_verts, cudaStream_t s);

}  // namespace scion
