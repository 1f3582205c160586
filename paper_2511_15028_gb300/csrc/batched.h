// Multi-scene persistent closest-hit launch (see batched.cu).
#pragma once

#include <cuda_runtime.h>

#include "../../include/scion.h"
#include "trace.cuh"

namespace scion {

// Node families the batched kernel dispatches on (direct child references;
// direct or indirect triangles): the width-2 own-box node with f32 or q16
// boxes (AoS), 4-wide SoA nodes with f32, f16 or u8 boxes, 8-wide SoA f16,
// 8-wide u8 AoS and SoA.
enum : uint32_t {
  kFamilyBin = 0,
  kFamilyBinQ16 = 1,
  kFamilyW4F32 = 2,
  kFamilyW4F16 = 3,
  kFamilyW4U8 = 4,
  kFamilyW8F16 = 5,
  kFamilyW8U8 = 6,
  kFamilyW8U8S = 7
};

// Rays a warp takes per atomic from the global counter; every scene's range
// in the global index space is padded to a multiple of it.
constexpr uint32_t kBatchUnit = 32;

struct alignas(16) BatchScene {
  TraceArgs a;               // the scene's trace arguments (rays, hits, BVH buffers)
  unsigned long long begin;  // first index of the scene in the padded global range
  uint32_t family;
  uint32_t pad;
};

// Family of a layout, or -1 if the batched kernel does not handle it.
int batched_family(uint32_t own_box, const scion_layout_desc &d);
const void *batched_kernel_ptr();
cudaError_t launch_batched(const BatchScene *d_scenes, uint32_t n_scenes, unsigned long long total,
                           unsigned long long *work, uint32_t *exit_count, uint32_t smem_stack,
                           uint32_t threads, uint32_t grid, cudaStream_t s);

}  // namespace scion
