// Multi-scene persistent closest-hit launch (see batched.cu).
#pragma once

#include <cuda_runtime.h>

#include "../../include/scion.h"
#include "trace.cuh"

namespace scion {

// Node families the batched kernel dispatches on (direct child references;
// direct or indirect triangles).
enum : uint32_t { kFamilyBin = 0, kFamilyW4F32 = 1, kFamilyW8F16 = 2, kFamilyW8U8 = 3 };

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
