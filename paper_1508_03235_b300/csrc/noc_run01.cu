// noc_run01.cu -- cycle kernel recording per-cycle quiescence (drain)
#include "noc_kernel.cuh"

namespace noc {

cudaError_t launch_run01(const Params& P, const RunArgs& A, cudaStream_t s) {
  return launch_run_t<false, true>(P, A, s);
}

}  // namespace noc
