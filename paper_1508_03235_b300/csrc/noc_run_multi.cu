// noc_run_multi.cu -- the capacity loop (two tiles per thread, noc_multi.cuh):
// compiled once per way-bound class with every policy, mode and option.
#include "noc_multi.cuh"

#if !defined(NOC_W1) || !defined(NOC_W2)
#error "compile with -DNOC_W1= -DNOC_W2="
#endif
#define NOC_PASTE3(a, b, c) a##_##b##_##c
#define NOC_NAME(a, b, c) NOC_PASTE3(a, b, c)

namespace noc {

cudaError_t NOC_NAME(launch_multi, NOC_W1, NOC_W2)(const Params& P, const RunArgs& A, cudaStream_t s) {
  return launch_multi_t<NOC_W1, NOC_W2, -3>(P, A, s);
}

cudaError_t NOC_NAME(max_coresident_multi, NOC_W1, NOC_W2)(int threads, int* out) {
  return max_coresident_multi_t<NOC_W1, NOC_W2, -3>(threads, out);
}

}  // namespace noc
