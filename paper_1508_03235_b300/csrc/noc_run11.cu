// noc_run11.cu -- cycle kernel recording both
#include "noc_kernel.cuh"

namespace noc {

cudaError_t launch_run11(const Params& P, const RunArgs& A, cudaStream_t s) {
  return launch_run_t<true, true>(P, A, s);
}

}  // namespace noc
