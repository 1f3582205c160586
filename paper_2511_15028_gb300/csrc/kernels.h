// Kernel table: one persistent traversal kernel per (node codec, query).
#pragma once

#include "trace.cuh"

namespace scion {

typedef void (*TraceKernel)(TraceArgs);

// Defined by trace_inst.cu, compiled once per node family:
//   own-box binary node       : kernels_own_p<prec>(soa, cref, any, stats, reg),
//                               prec 0 f32, 3 q16, 4 eq10, 6 shared slab
//   wide node of width W, prec: kernels_w<W>_p<prec>(soa, cref, any, stats, reg)
// stats = 1 selects the counting variant (visit counters, same results);
// reg = register entries at the top of the traversal stack (0, 2 or 4; other
// values give null).
TraceKernel kernels_own_p0(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_own_p3(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_own_p4(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_own_p6(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w2_p0(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w2_p1(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w2_p2(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w4_p0(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w4_p1(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w4_p2(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w8_p0(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w8_p1(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w8_p2(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w2_p5(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w4_p5(int soa, int cref, int any, int stats, int reg);
TraceKernel kernels_w8_p5(int soa, int cref, int any, int stats, int reg);
// closest point query kernels of the same families
TraceKernel cpq_kernels_own_p0(int soa, int cref, int stats);
TraceKernel cpq_kernels_own_p3(int soa, int cref, int stats);
TraceKernel cpq_kernels_own_p4(int soa, int cref, int stats);
TraceKernel cpq_kernels_own_p6(int soa, int cref, int stats);  // null: not supported
TraceKernel cpq_kernels_w2_p0(int soa, int cref, int stats);
TraceKernel cpq_kernels_w2_p1(int soa, int cref, int stats);
TraceKernel cpq_kernels_w2_p2(int soa, int cref, int stats);
TraceKernel cpq_kernels_w4_p0(int soa, int cref, int stats);
TraceKernel cpq_kernels_w4_p1(int soa, int cref, int stats);
TraceKernel cpq_kernels_w4_p2(int soa, int cref, int stats);
TraceKernel cpq_kernels_w8_p0(int soa, int cref, int stats);
TraceKernel cpq_kernels_w8_p1(int soa, int cref, int stats);
TraceKernel cpq_kernels_w8_p2(int soa, int cref, int stats);
TraceKernel cpq_kernels_w2_p5(int soa, int cref, int stats);
TraceKernel cpq_kernels_w4_p5(int soa, int cref, int stats);
TraceKernel cpq_kernels_w8_p5(int soa, int cref, int stats);

constexpr int kMaxThreadsPerBlock = 256;
constexpr uint32_t kMaxRegStack = 4;  // largest register tier of the traversal stack
// Four 256-thread CTAs per SM: caps a traversal kernel at 64 registers so 32
// warps per SM keep dependent node loads in flight (the 8-wide f16/u8 kernels
// otherwise take 74-80 registers, and 24 warps). The 8-wide f32 node (48
// floats of boxes) would spill heavily under the cap and keeps its own count.
#if defined(SCION_W) && SCION_W == 8 && SCION_PREC == 0
constexpr int kMinBlocksPerSm = 1;
#else
constexpr int kMinBlocksPerSm = 4;
#endif

}  // namespace scion
