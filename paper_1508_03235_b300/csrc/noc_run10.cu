// noc_run10.cu -- cycle kernel recording the per-cycle state hash
#include "noc_kernel.cuh"

namespace noc {

cudaError_t launch_run10(const Params& P, const RunArgs& A, cudaStream_t s) {
  return launch_run_t<true, false>(P, A, s);
}

}  // namespace noc
