// noc_run_variant.cu -- one variant of the cycle kernel per compilation: the
// build compiles this file once for each (per-cycle hash record, drain record,
// L1 way bound, L2 way bound) combination it ships, and the plain loop twice
// more per way bound: without the options beyond the paper's workloads
// (-DNOC_BASE=1), and specialised to one L2 policy in cache mode with exactly
// those way counts (-DNOC_FIXED_POLICY=<p> -DNOC_FIXED_MODE=0
// -DNOC_EXACT_WAYS=1: p = 0 interleaved, 1 LSPD with local placement, 2 LSPD
// with migration); the plain-loop builds once more each with -DNOC_NARROW=1,
// for CTAs of at most NARROW_THREADS threads, and with -DNOC_XL=1, for CTAs of
// more than WIDE_THREADS; the general plain loop once more with -DNOC_CHECKS=1.
#include "noc_kernel.cuh"

#if !defined(NOC_HASH) || !defined(NOC_DRAIN) || !defined(NOC_W1) || !defined(NOC_W2)
#error "compile with -DNOC_HASH= -DNOC_DRAIN= -DNOC_W1= -DNOC_W2="
#endif
#if defined(NOC_FIXED_POLICY) && NOC_FIXED_POLICY == 1
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC0 local
#elif defined(NOC_FIXED_POLICY) && NOC_FIXED_POLICY == 2
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC0 migrate
#elif defined(NOC_FIXED_POLICY)
#define NOC_POLV NOC_FIXED_POLICY
#define NOC_SPEC0 il
#elif defined(NOC_BASE)
#define NOC_POLV (-2)
#define NOC_SPEC0 base
#else
#define NOC_POLV (-1)
#define NOC_SPEC0 gen
#endif
// -DNOC_NARROW=1: the build for CTAs of at most NARROW_THREADS threads
#define NOC_PASTE2(a, b) a##_##b
#define NOC_CAT2(a, b) NOC_PASTE2(a, b)
#if NOC_CHECKS
// -DNOC_CHECKS=1: the plain loop with the single-writer checks, for every CTA size
#define NOC_LB MAX_THREADS
#define NOC_SPEC NOC_CAT2(NOC_SPEC0, checked)
#elif defined(NOC_NARROW) && NOC_NARROW
#define NOC_LB NARROW_THREADS
#define NOC_SPEC NOC_CAT2(NOC_SPEC0, narrow)
#elif NOC_PHASE_PROFILE
// -DNOC_PHASE_PROFILE=1: the plain loop with per-phase clock reads
#define NOC_LB PROF_THREADS
#define NOC_SPEC NOC_CAT2(NOC_SPEC0, prof)
#elif defined(NOC_XL) && NOC_XL
// -DNOC_XL=1: the plain loop for CTAs of up to MAX_THREADS threads
#define NOC_LB MAX_THREADS
#define NOC_SPEC NOC_CAT2(NOC_SPEC0, xl)
#elif NOC_HASH || NOC_DRAIN
// the traced and draining loops take every CTA size the plain loop does
#define NOC_LB MAX_THREADS
#define NOC_SPEC NOC_SPEC0
#else
#define NOC_LB WIDE_THREADS
#define NOC_SPEC NOC_SPEC0
#endif

#define NOC_PASTE6(a, b, c, d, e, f) a##_##b##_##c##_##d##_##e##_##f
#define NOC_NAME(a, b, c, d, e, f) NOC_PASTE6(a, b, c, d, e, f)

namespace noc {

cudaError_t NOC_NAME(launch_run, NOC_HASH, NOC_DRAIN, NOC_W1, NOC_W2, NOC_SPEC)(const Params& P,
                                                                              const RunArgs& A,
                                                                              cudaStream_t s) {
  return launch_run_t<NOC_HASH != 0, NOC_DRAIN != 0, NOC_W1, NOC_W2, NOC_POLV, NOC_LB>(P, A, s);
}

#if NOC_HASH == 0 && NOC_DRAIN == 0
cudaError_t NOC_NAME(max_coresident_run, 0, 0, NOC_W1, NOC_W2, NOC_SPEC)(int threads, int* out) {
  return max_coresident_run_t<NOC_W1, NOC_W2, NOC_POLV, NOC_LB>(threads, out);
}
#endif

}  // namespace noc
