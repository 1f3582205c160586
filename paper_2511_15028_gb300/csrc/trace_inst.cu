// Instantiates the traversal kernels of one node family. Compiled several
// times with -DSCION_OWN=1 -DSCION_PREC=<0|3|4|6> (own-box node with f32, q16
// or eq10 boxes, or the shared-slab node), or -DSCION_W=<2|4|8> -DSCION_PREC=<0|1|2|5>, so the families
// build in parallel.
#include "cpq.cuh"
#include "kernels.h"

#define SCION_CAT_(a, b) a##b
#define SCION_CAT(a, b) SCION_CAT_(a, b)

namespace scion {

#if defined(SCION_OWN)
#define SCION_FAMILY_OWN true
#define SCION_W 2
#define SCION_GETTER SCION_CAT(kernels_own_p, SCION_PREC)
#define SCION_CPQ_GETTER SCION_CAT(cpq_kernels_own_p, SCION_PREC)
#else
#define SCION_FAMILY_OWN false
#define SCION_GETTER SCION_CAT(SCION_CAT(SCION_CAT(kernels_w, SCION_W), _p), SCION_PREC)
#define SCION_CPQ_GETTER SCION_CAT(SCION_CAT(SCION_CAT(cpq_kernels_w, SCION_W), _p), SCION_PREC)
#endif

// The register tier of the stack spills under the 64-register cap of four
// CTAs per SM; measured, that costs less than giving up a CTA per SM.
template <int SOA, int CREF, bool ANY, bool STATS, int REG>
__global__ void __launch_bounds__(kMaxThreadsPerBlock, kMinBlocksPerSm) trace_kernel(TraceArgs a) {
  trace_kernel_body<SCION_FAMILY_OWN, SCION_W, SCION_PREC, SOA, CREF, ANY, STATS, REG>(a);
}

// reg: register entries at the top of the stack, 0, 2 or 4 (the counting
// variants visit the same nodes whatever the stack: they exist for reg 0)
TraceKernel SCION_GETTER(int soa, int cref, int any, int stats, int reg) {
  static const TraceKernel counting[2][2][2] = {
      {{trace_kernel<0, 0, false, true, 0>, trace_kernel<0, 0, true, true, 0>},
       {trace_kernel<0, 1, false, true, 0>, trace_kernel<0, 1, true, true, 0>}},
      {{trace_kernel<1, 0, false, true, 0>, trace_kernel<1, 0, true, true, 0>},
       {trace_kernel<1, 1, false, true, 0>, trace_kernel<1, 1, true, true, 0>}}};
  static const TraceKernel plain[3][2][2][2] = {
      {{{trace_kernel<0, 0, false, false, 0>, trace_kernel<0, 0, true, false, 0>},
        {trace_kernel<0, 1, false, false, 0>, trace_kernel<0, 1, true, false, 0>}},
       {{trace_kernel<1, 0, false, false, 0>, trace_kernel<1, 0, true, false, 0>},
        {trace_kernel<1, 1, false, false, 0>, trace_kernel<1, 1, true, false, 0>}}},
      {{{trace_kernel<0, 0, false, false, 2>, trace_kernel<0, 0, true, false, 2>},
        {trace_kernel<0, 1, false, false, 2>, trace_kernel<0, 1, true, false, 2>}},
       {{trace_kernel<1, 0, false, false, 2>, trace_kernel<1, 0, true, false, 2>},
        {trace_kernel<1, 1, false, false, 2>, trace_kernel<1, 1, true, false, 2>}}},
      {{{trace_kernel<0, 0, false, false, 4>, trace_kernel<0, 0, true, false, 4>},
        {trace_kernel<0, 1, false, false, 4>, trace_kernel<0, 1, true, false, 4>}},
       {{trace_kernel<1, 0, false, false, 4>, trace_kernel<1, 0, true, false, 4>},
        {trace_kernel<1, 1, false, false, 4>, trace_kernel<1, 1, true, false, 4>}}}};
  if (stats) return counting[soa & 1][cref & 1][any & 1];
  const int ri = reg == 4 ? 2 : (reg == 2 ? 1 : 0);
  if (reg != 0 && reg != 2 && reg != 4) return nullptr;
  return plain[ri][soa & 1][cref & 1][any & 1];
}


#if SCION_FAMILY_OWN && SCION_PREC == 6
// the shared-slab node carries ray intervals, not boxes: no closest point query
TraceKernel SCION_CPQ_GETTER(int, int, int) { return nullptr; }
#else
template <int SOA, int CREF, bool STATS>
__global__ void __launch_bounds__(kMaxThreadsPerBlock, kMinBlocksPerSm) cpq_kernel(TraceArgs a) {
  cpq_kernel_body<SCION_FAMILY_OWN, SCION_W, SCION_PREC, SOA, CREF, STATS>(a);
}
TraceKernel SCION_CPQ_GETTER(int soa, int cref, int stats) {
  static const TraceKernel table[2][2][2] = {
      {{cpq_kernel<0, 0, false>, cpq_kernel<0, 0, true>}, {cpq_kernel<0, 1, false>, cpq_kernel<0, 1, true>}},
      {{cpq_kernel<1, 0, false>, cpq_kernel<1, 0, true>}, {cpq_kernel<1, 1, false>, cpq_kernel<1, 1, true>}}};
  return table[soa & 1][cref & 1][stats & 1];
}
#endif

}  // namespace scion
