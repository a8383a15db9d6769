// noc_batch.cu -- the batch engine's persistent work-queue kernel (compiled once
// per L1/L2 way bound, and more per bound specialised like the plain cycle
// loop: -DNOC_BASE=1, and -DNOC_FIXED_POLICY=<p> -DNOC_FIXED_MODE=0
// -DNOC_EXACT_WAYS=1 for p = 0, 1, 2)
// the batch's rectangles are small and mostly edge: one poll in flight
#define NOC_POLL_STAGE 0
#define NOC_PREFETCH_HOME 0
#include "noc_kernel.cuh"

#if !defined(NOC_W1) || !defined(NOC_W2)
#error "compile with -DNOC_W1= -DNOC_W2="
#endif
#if defined(NOC_FIXED_POLICY) && NOC_FIXED_POLICY == 1
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC local
#elif defined(NOC_FIXED_POLICY) && NOC_FIXED_POLICY == 2
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC migrate
#elif defined(NOC_FIXED_POLICY)
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC il
#elif defined(NOC_BASE)
#define NOC_POLV (-2)
#define NOC_SPEC base
#else
#define NOC_POLV (-1)
#define NOC_SPEC gen
#endif
#define NOC_PASTE4(a, b, c, d) a##_##b##_##c##_##d
#define NOC_NAME(a, b, c, d) NOC_PASTE4(a, b, c, d)

namespace noc {

// ---------------------------------------------------------------- batch kernel
// Persistent CTAs pop (instance, rectangle) items from a device work queue in
// order.  All rectangles of one instance are consecutive in the queue; a CTA
// that pops one waits until every rectangle of its instance has been popped
// (so the instance's neighbour waits start together), then runs it to the end
// of the instance's cycles.  Items are popped in order, so every instance
// before the current one is already running to completion: the waits end.
template <int W1, int W2, int POLV>
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 1) batch_kernel(const __grid_constant__ BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Params sP;
  __shared__ RunArgs sA;
  __shared__ int s_item, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(B.next_item, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= B.n_items) break;
    const int inst = B.item_inst[item];
    if (threadIdx.x == 0) {
      atomicAdd(&B.claimed[inst], 1u);
      int w = wait_ge(&B.claimed[inst], (unsigned)B.need[inst], B.args[inst].abort_flag, B.gang_ns);
      if (w == 0) {
        atomicExch(B.args[inst].abort_flag, 1u);
        set_error(B.params[inst], 0, ERR_TIMEOUT);
      }
      s_ok = w > 0;
    }
    // this instance's parameters into shared memory
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&B.params[inst]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sP);
      for (int k = threadIdx.x; k < (int)(sizeof(Params) / 4); k += blockDim.x) dst[k] = src[k];
      const uint32_t* srca = reinterpret_cast<const uint32_t*>(&B.args[inst]);
      uint32_t* dsta = reinterpret_cast<uint32_t*>(&sA);
      for (int k = threadIdx.x; k < (int)(sizeof(RunArgs) / 4); k += blockDim.x) dsta[k] = srca[k];
    }
    __syncthreads();
    if (s_ok) run_rect_warps<W1, W2>(sP, sA, B.item_rect[item], smem_raw);
    __syncthreads();
  }
}

#define NOC_BATCH_KERNEL batch_kernel<NOC_W1, NOC_W2, NOC_POLV>

cudaError_t NOC_NAME(launch_batch, NOC_W1, NOC_W2, NOC_SPEC)(const BatchArgs& B, int grid, int threads,
                                                            cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(NOC_BATCH_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)run_smem_bytes_impl(BATCH_MAX_THREADS, false));
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&B};
  return cudaLaunchCooperativeKernel((const void*)NOC_BATCH_KERNEL, dim3(grid), dim3(threads), args,
                                     run_smem_bytes_impl(threads, false), s);
}

cudaError_t NOC_NAME(max_coresident_batch, NOC_W1, NOC_W2, NOC_SPEC)(int threads, int* out) {
  cudaError_t e = cudaFuncSetAttribute(NOC_BATCH_KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)run_smem_bytes_impl(BATCH_MAX_THREADS, false));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, NOC_BATCH_KERNEL, threads, run_smem_bytes_impl(threads, false));
  if (e != cudaSuccess) return e;
  *out = per * sms;
  return cudaSuccess;
}


}  // namespace noc
