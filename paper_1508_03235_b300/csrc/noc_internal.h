// noc_internal.h -- declarations shared by the kernels (noc_kernel.cu) and the
// host side of the C ABI (noc_api.cu).  Not installed; not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include "noc_model.cuh"

namespace noc {

// global cycle flags per CTA rectangle: one per warp (the plain cycle loop),
// slot 0 for the CTA as a whole (the traced and draining loops)
constexpr int FLAG_SLOTS = 16;

// per-launch arguments of the cycle kernel
struct RunArgs {
  uint32_t t0, n;        // first cycle and number of cycles of this launch
  int draining;          // 1: no new references (drain)
  int gx, gy;            // CTA rectangle grid
  unsigned long long* hash_trace;  // per-cycle dynamic hash (nullptr: off)
  unsigned int* busy;              // per-cycle count of non-quiet tiles (drain)
  unsigned int* abort_flag;        // set when a wait ran out; all CTAs stop
  long long wait_ns;               // limit of each device-side wait
  int silent_cta;                  // test fault: this CTA never publishes
  int thread_map;                  // tile-to-thread order inside a rectangle (MAP_*)
  // per-phase SM clocks of the plain loop, summed over warps (the profiled
  // build only; nullptr otherwise): waiting, routing, publishing, Phase 3,
  // Phase 1, and the number of warp-cycles
  unsigned long long* prof;
  // 1: run the plain loop on the checked build (noc_set_checks)
  int checked;
};

// batch work queue: per-instance parameters, and items (instance, rectangle)
// ordered instance by instance
struct BatchArgs {
  const Params* params;
  const RunArgs* args;
  const int* item_inst;
  const int* item_rect;
  const int* need;          // rectangles per instance
  unsigned int* claimed;    // rectangles popped per instance
  unsigned int* next_item;  // queue head
  int n_items;
  long long gang_ns;        // limit of the wait for an instance's rectangles
};
// kind: which specialisation of the device code runs -- KIND_IL, KIND_LOCAL
// and KIND_MIGRATE (one L2 policy -- interleaved, LSPD with local placement,
// LSPD with migration -- in cache mode with exactly the way counts of the
// class of (l1_ways, l2_ways), no packet, write-back, directory-node or age
// option), KIND_BASE (every policy and mode, none of those options) or
// KIND_GEN (everything); variant_kind(P) is the narrowest one a configuration
// may run on
enum { KIND_GEN = 0, KIND_BASE = 1, KIND_IL = 2, KIND_LOCAL = 3, KIND_MIGRATE = 4 };
// batch kernel-variant groups (noc_batch_group)
constexpr int NOC_BATCH_GROUPS = 11;
int variant_kind(const Params& P);
cudaError_t launch_batch(const BatchArgs& B, int grid, int threads, int l1_ways, int l2_ways, int kind,
                         cudaStream_t s);
cudaError_t max_coresident_batch(int l1_ways, int l2_ways, int kind, int threads, int* out);
int batch_way_class(int l1_ways, int l2_ways);

// geometry of the launch for a gx x gy rectangle grid
int block_threads(int W, int H, int gx, int gy);
size_t run_smem_bytes(int threads);

cudaError_t launch_run(const Params& P, const RunArgs& A, cudaStream_t s);
cudaError_t max_coresident_ctas(const Params& P, int threads, int* out);
cudaError_t launch_dyn_hash(const Params& P, uint32_t cycle, unsigned long long* out,
                            cudaStream_t s);
cudaError_t launch_state_hash(const Params& P, uint32_t cycle, unsigned long long* out,
                              cudaStream_t s);
cudaError_t launch_reduce_stats(const Params& P, int tile, unsigned long long* out,
                                cudaStream_t s);
cudaError_t launch_count_busy(const Params& P, uint32_t cycle, unsigned int* out,
                              cudaStream_t s);
cudaError_t launch_gen_refs(const Params& P, uint32_t t0, uint32_t n, cudaStream_t s);
cudaError_t launch_fill_u32(unsigned int* p, unsigned int v, size_t n, cudaStream_t s);

}  // namespace noc
