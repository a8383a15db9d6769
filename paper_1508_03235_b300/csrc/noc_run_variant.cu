// noc_run_variant.cu -- one variant of the cycle kernel per compilation: the
// build compiles this file once for each (per-cycle hash record, drain record,
// L1 way bound, L2 way bound) combination it ships.
#include "noc_kernel.cuh"

#if !defined(NOC_HASH) || !defined(NOC_DRAIN) || !defined(NOC_W1) || !defined(NOC_W2)
#error "compile with -DNOC_HASH= -DNOC_DRAIN= -DNOC_W1= -DNOC_W2="
#endif

#define NOC_PASTE5(a, b, c, d, e) a##_##b##_##c##_##d##_##e
#define NOC_NAME(a, b, c, d, e) NOC_PASTE5(a, b, c, d, e)

namespace noc {

cudaError_t NOC_NAME(launch_run, NOC_HASH, NOC_DRAIN, NOC_W1, NOC_W2)(const Params& P,
                                                                    const RunArgs& A,
                                                                    cudaStream_t s) {
  return launch_run_t<NOC_HASH != 0, NOC_DRAIN != 0, NOC_W1, NOC_W2>(P, A, s);
}

#if NOC_HASH == 0 && NOC_DRAIN == 0
cudaError_t NOC_NAME(max_coresident_run, 0, 0, NOC_W1, NOC_W2)(int threads, int* out) {
  return max_coresident_run_t<NOC_W1, NOC_W2>(threads, out);
}
#endif

}  // namespace noc
