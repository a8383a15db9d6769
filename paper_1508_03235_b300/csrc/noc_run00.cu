// noc_run00.cu -- the cycle kernel as the bench and the product run it (no per-cycle records)
#include "noc_kernel.cuh"

namespace noc {


cudaError_t launch_run00(const Params& P, const RunArgs& A, cudaStream_t s) {
  return launch_run_t<false, false>(P, A, s);
}

cudaError_t max_coresident_ctas(int threads, int* out) {
  cudaError_t e = prepare_run<false, false>();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, run_kernel<false, false>, threads,
                                                    run_smem_bytes_impl(threads));
  if (e != cudaSuccess) return e;
  *out = per * sms;
  return cudaSuccess;
}


size_t run_smem_bytes(int threads) { return run_smem_bytes_impl(threads); }

int block_threads(int W, int H, int gx, int gy) { return block_threads_impl(W, H, gx, gy); }

}  // namespace noc
