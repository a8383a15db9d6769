// noc_host.h -- host-side helpers shared by the C ABI's translation units
// (noc_api.cu, noc_static.cu, noc_kernel.cu).  Not installed; not part of the
// ABI; no device code reads it.
#pragma once
#include "noc.h"
#include "noc_internal.h"

namespace noc {

// the C ABI's error reporting: stores the formatted message that
// noc_last_error() returns (thread-local) and returns code
int fail(int code, const char* fmt, ...);
// check a configuration exactly as noc_create does (NOC_ERR_ARG with the
// reason set through fail() when invalid) and fill every model field of P;
// the device pointers of P are left null
int configure(int mesh_w, int mesh_h, const noc_cache_cfg* c, int l2_policy, const noc_traffic* tr,
              uint64_t seed, Params& P);
// the build of the cycle kernel launch_run picks for (P, A): loop << 8 |
// kind << 4 | way class, with loop 1 for the traced / draining loop, kind a
// KIND_* value and way class 0 = (4, 8), 1 = (4, 16), 2 = (16, 16) bounds
int run_variant(const Params& P, const RunArgs& A);
// the most threads a CTA of the one-tile loop may have (MAX_THREADS of the
// device code; one CTA per SM at the wide builds' register cap)
constexpr int RUN_MAX_THREADS = 448;
// and of its per-phase profiled build (PROF_THREADS of the device code)
constexpr int RUN_PROF_THREADS = 384;
// the launch bound (most threads per CTA) of the build launch_run picks
int run_launch_bound(const Params& P, const RunArgs& A);
// co-resident CTAs of the plain loop's checked build at `threads` per CTA
cudaError_t max_coresident_checked(const Params& P, int threads, int* out);
// co-resident CTAs of the plain loop's profiled build at `threads` per CTA
cudaError_t max_coresident_prof(const Params& P, int threads, int* out);
// the capacity loop (two tiles per thread, plain cycles only): launch, its
// co-resident CTAs at `threads` per CTA, threads per CTA of a gx x gy
// rectangle grid, and its run_variant() code (loop 2)
constexpr int MULTI_MAX_THREADS = 256;
cudaError_t launch_multi(const Params& P, const RunArgs& A, cudaStream_t s);
cudaError_t max_coresident_multi(const Params& P, int threads, int* out);
int multi_threads(int W, int H, int gx, int gy);
int multi_variant(const Params& P);

}  // namespace noc
