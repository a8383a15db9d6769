// noc_run_variant.cu -- one variant of the cycle kernel per compilation: the
// build compiles this file once for each (per-cycle hash record, drain record,
// L1 way bound, L2 way bound) combination it ships, and the plain loop twice
// more per way bound: without the options beyond the paper's workloads
// (-DNOC_BASE=1), and specialised to the interleaved L2 in cache mode with
// exactly those way counts (-DNOC_FIXED_POLICY=0 -DNOC_FIXED_MODE=0
// -DNOC_EXACT_WAYS=1).
#include "noc_kernel.cuh"

#if !defined(NOC_HASH) || !defined(NOC_DRAIN) || !defined(NOC_W1) || !defined(NOC_W2)
#error "compile with -DNOC_HASH= -DNOC_DRAIN= -DNOC_W1= -DNOC_W2="
#endif
#if defined(NOC_FIXED_POLICY)
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC il
#elif defined(NOC_BASE)
#define NOC_POLV (-2)
#define NOC_SPEC base
#else
#define NOC_POLV (-1)
#define NOC_SPEC gen
#endif

#define NOC_PASTE6(a, b, c, d, e, f) a##_##b##_##c##_##d##_##e##_##f
#define NOC_NAME(a, b, c, d, e, f) NOC_PASTE6(a, b, c, d, e, f)

namespace noc {

cudaError_t NOC_NAME(launch_run, NOC_HASH, NOC_DRAIN, NOC_W1, NOC_W2, NOC_SPEC)(const Params& P,
                                                                              const RunArgs& A,
                                                                              cudaStream_t s) {
  return launch_run_t<NOC_HASH != 0, NOC_DRAIN != 0, NOC_W1, NOC_W2, NOC_POLV>(P, A, s);
}

#if NOC_HASH == 0 && NOC_DRAIN == 0
cudaError_t NOC_NAME(max_coresident_run, 0, 0, NOC_W1, NOC_W2, NOC_SPEC)(int threads, int* out) {
  return max_coresident_run_t<NOC_W1, NOC_W2, NOC_POLV>(threads, out);
}
#endif

}  // namespace noc
