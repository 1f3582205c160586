// Kernel table: one persistent traversal kernel per (node codec, query).
#pragma once

#include "trace.cuh"

namespace scion {

typedef void (*TraceKernel)(TraceArgs);

// Defined by trace_inst.cu, compiled once per node family:
//   own-box binary node       : kernels_own(soa, cref, any, stats)
//   wide node of width W, prec: kernels_w<W>_p<prec>(soa, cref, any, stats)
// stats = 1 selects the counting variant (visit counters, same results).
TraceKernel kernels_own(int soa, int cref, int any, int stats);
TraceKernel kernels_w2_p0(int soa, int cref, int any, int stats);
TraceKernel kernels_w2_p1(int soa, int cref, int any, int stats);
TraceKernel kernels_w2_p2(int soa, int cref, int any, int stats);
TraceKernel kernels_w4_p0(int soa, int cref, int any, int stats);
TraceKernel kernels_w4_p1(int soa, int cref, int any, int stats);
TraceKernel kernels_w4_p2(int soa, int cref, int any, int stats);
TraceKernel kernels_w8_p0(int soa, int cref, int any, int stats);
TraceKernel kernels_w8_p1(int soa, int cref, int any, int stats);
TraceKernel kernels_w8_p2(int soa, int cref, int any, int stats);

constexpr int kMaxThreadsPerBlock = 256;

}  // namespace scion
