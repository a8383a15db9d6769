// noc_kernel.cu -- state-hash, statistics and drain helper kernels, and the
// dispatch to the cycle-kernel variants.
#include "noc_host.h"
#include "noc_kernel.cuh"

namespace noc {

static_assert(RUN_MAX_THREADS == MAX_THREADS && RUN_PROF_THREADS == PROF_THREADS,
              "host and device thread limits agree");

// ---------------------------------------------------------------- dispatch
// Kernel variants shipped: the per-cycle hash record or the drain's busy
// record on (the traced / draining loop) or neither (the plain loop), and the
// compile-time way bounds (L1, L2) of the cache-set code: (4, 8), (4, 16) and
// the general (16, 16).  The plain loop also comes as "base" (every policy and
// mode, the packet, write-back, directory-node and age options compiled out) and as
// "il", "local" and "migrate", each specialised to one L2 policy (interleaved,
// LSPD with local placement, LSPD with migration) in cache mode with the
// class's exact way counts (the other policies' code compiled out, the way
// loops of fixed length).  The per-phase profiled builds exist for gen, base
// and il; a local or migrate configuration is profiled on the base build.
#define NOC_DECL_RUN(h, d, w1, w2, sp) \
  cudaError_t launch_run_##h##_##d##_##w1##_##w2##_##sp(const Params&, const RunArgs&, cudaStream_t);
#define NOC_DECL_WAYS(w1, w2)                                                   \
  NOC_DECL_RUN(0, 0, w1, w2, gen)                                               \
  NOC_DECL_RUN(1, 0, w1, w2, gen)                                               \
  NOC_DECL_RUN(0, 1, w1, w2, gen)                                               \
  NOC_DECL_RUN(0, 0, w1, w2, il)                                                \
  NOC_DECL_RUN(0, 0, w1, w2, base)                                              \
  NOC_DECL_RUN(0, 0, w1, w2, gen_narrow)                                        \
  NOC_DECL_RUN(0, 0, w1, w2, il_narrow)                                         \
  NOC_DECL_RUN(0, 0, w1, w2, base_narrow)                                       \
  NOC_DECL_RUN(0, 0, w1, w2, gen_prof)                                          \
  NOC_DECL_RUN(0, 0, w1, w2, il_prof)                                           \
  NOC_DECL_RUN(0, 0, w1, w2, base_prof)                                         \
  NOC_DECL_RUN(0, 0, w1, w2, local)                                             \
  NOC_DECL_RUN(0, 0, w1, w2, migrate)                                           \
  NOC_DECL_RUN(0, 0, w1, w2, local_narrow)                                      \
  NOC_DECL_RUN(0, 0, w1, w2, gen_xl)                                            \
  NOC_DECL_RUN(0, 0, w1, w2, gen_checked)                                       \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_gen_checked(int threads, int* out); \
  NOC_DECL_RUN(0, 0, w1, w2, base_xl)                                           \
  NOC_DECL_RUN(0, 0, w1, w2, il_xl)                                             \
  NOC_DECL_RUN(0, 0, w1, w2, local_xl)                                          \
  NOC_DECL_RUN(0, 0, w1, w2, migrate_xl)                                        \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_gen_xl(int threads, int* out);     \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_base_xl(int threads, int* out);    \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_il_xl(int threads, int* out);      \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_local_xl(int threads, int* out);   \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_migrate_xl(int threads, int* out); \
  NOC_DECL_RUN(0, 0, w1, w2, migrate_narrow)                                    \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_local(int threads, int* out);        \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_migrate(int threads, int* out);      \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_local_narrow(int threads, int* out); \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_migrate_narrow(int threads, int* out); \
  cudaError_t launch_batch_##w1##_##w2##_local(const BatchArgs&, int, int, cudaStream_t); \
  cudaError_t launch_batch_##w1##_##w2##_migrate(const BatchArgs&, int, int, cudaStream_t); \
  cudaError_t max_coresident_batch_##w1##_##w2##_local(int threads, int* out);            \
  cudaError_t max_coresident_batch_##w1##_##w2##_migrate(int threads, int* out);          \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_gen_prof(int threads, int* out);  \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_il_prof(int threads, int* out);   \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_base_prof(int threads, int* out); \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_gen(int threads, int* out);  \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_il(int threads, int* out);   \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_base(int threads, int* out); \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_gen_narrow(int threads, int* out);  \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_il_narrow(int threads, int* out);   \
  cudaError_t max_coresident_run_0_0_##w1##_##w2##_base_narrow(int threads, int* out); \
  cudaError_t launch_batch_##w1##_##w2##_gen(const BatchArgs&, int, int, cudaStream_t); \
  cudaError_t launch_batch_##w1##_##w2##_il(const BatchArgs&, int, int, cudaStream_t);  \
  cudaError_t launch_batch_##w1##_##w2##_base(const BatchArgs&, int, int, cudaStream_t); \
  cudaError_t max_coresident_batch_##w1##_##w2##_gen(int threads, int* out);             \
  cudaError_t max_coresident_batch_##w1##_##w2##_il(int threads, int* out);              \
  cudaError_t max_coresident_batch_##w1##_##w2##_base(int threads, int* out);
NOC_DECL_WAYS(4, 8)
NOC_DECL_WAYS(4, 16)
NOC_DECL_WAYS(16, 16)
#define NOC_DECL_MULTI(w1, w2)                                                                  \
  cudaError_t launch_multi_##w1##_##w2(const Params&, const RunArgs&, cudaStream_t);           \
  cudaError_t max_coresident_multi_##w1##_##w2(int threads, int* out);
NOC_DECL_MULTI(4, 8)
NOC_DECL_MULTI(4, 16)
NOC_DECL_MULTI(16, 16)

// way-bound class of a configuration: 0 = (4, 8), 1 = (4, 16), 2 = (16, 16)
static int way_class(int l1_ways, int l2_ways) {
  if (l1_ways > 4) return 2;
  return l2_ways <= 8 ? 0 : 1;
}
// the plain loop has variants specialised to one L2 policy in cache mode with
// exactly the way counts of its class and none of the options
static bool exact_cache(const Params& P) {
  static const int exact[3][2] = {{4, 8}, {4, 16}, {16, 16}};
  const int c = way_class(P.l1_ways, P.l2_ways);
  return P.mode == MODE_CACHE && !P.packet_mode && !P.l1_write_back && !P.age_mode &&
         P.l1_ways == exact[c][0] && P.l2_ways == exact[c][1];
}
// the plain-loop variant a configuration runs on (the interleaved L2 keeps no
// directory, so the directory node makes no difference to it)
int variant_kind(const Params& P) {
  if (exact_cache(P)) {
    if (P.policy == POL_INTERLEAVED) return KIND_IL;
    if (!P.dir_central) return P.policy == POL_LOCAL ? KIND_LOCAL : KIND_MIGRATE;
  }
  if (!P.packet_mode && !P.l1_write_back && !P.dir_central && !P.age_mode) return KIND_BASE;
  return KIND_GEN;
}
// the kind whose profiled build a configuration runs on
static int prof_kind(int kind) { return kind == KIND_LOCAL || kind == KIND_MIGRATE ? KIND_BASE : kind; }

#define NOC_PICK_RUN(h, d, sp)                                    \
  switch (way_class(P.l1_ways, P.l2_ways)) {                      \
    case 0: return launch_run_##h##_##d##_4_8_##sp(P, A, s);      \
    case 1: return launch_run_##h##_##d##_4_16_##sp(P, A, s);     \
    default: return launch_run_##h##_##d##_16_16_##sp(P, A, s);   \
  }

int run_variant(const Params& P, const RunArgs& A) {
  const int traced = (A.hash_trace || A.busy) ? 1 : 0;
  const int kind = traced || A.checked ? KIND_GEN : A.prof ? prof_kind(variant_kind(P)) : variant_kind(P);
  return (traced << 8) | (kind << 4) | way_class(P.l1_ways, P.l2_ways);
}

// the plain loop's launch bound for CTAs of `threads`: the smallest that fits
static int plain_bound(int threads) {
  return threads <= NARROW_THREADS ? NARROW_THREADS : threads <= WIDE_THREADS ? WIDE_THREADS : MAX_THREADS;
}

int run_launch_bound(const Params& P, const RunArgs& A) {
  if (A.hash_trace || A.busy || A.checked) return MAX_THREADS;
  if (A.prof) return PROF_THREADS;
  return plain_bound(block_threads_impl(P.W, P.H, A.gx, A.gy));
}

int multi_variant(const Params& P) { return (2 << 8) | (KIND_GEN << 4) | way_class(P.l1_ways, P.l2_ways); }

cudaError_t launch_multi(const Params& P, const RunArgs& A, cudaStream_t s) {
  switch (way_class(P.l1_ways, P.l2_ways)) {
    case 0: return launch_multi_4_8(P, A, s);
    case 1: return launch_multi_4_16(P, A, s);
    default: return launch_multi_16_16(P, A, s);
  }
}

cudaError_t max_coresident_multi(const Params& P, int threads, int* out) {
  switch (way_class(P.l1_ways, P.l2_ways)) {
    case 0: return max_coresident_multi_4_8(threads, out);
    case 1: return max_coresident_multi_4_16(threads, out);
    default: return max_coresident_multi_16_16(threads, out);
  }
}

int multi_threads(int W, int H, int gx, int gy) {
  const int bw = (W + gx - 1) / gx, bh = (H + gy - 1) / gy;
  const int per = (bw * bh + 1) / 2;
  return ((per + 31) / 32) * 32;
}

cudaError_t launch_run(const Params& P, const RunArgs& A, cudaStream_t s) {
  // a drain records its busy counts, never a hash trace
  if (A.hash_trace && A.busy) return cudaErrorInvalidValue;
  if (A.hash_trace) { NOC_PICK_RUN(1, 0, gen) }
  if (A.busy) { NOC_PICK_RUN(0, 1, gen) }
  // the plain loop: the checked build when asked for, the profiled build when
  // asked for, else the build of the smallest launch bound the CTAs fit
  if (A.checked) { NOC_PICK_RUN(0, 0, gen_checked) }
  if (A.prof) {
    switch (prof_kind(variant_kind(P))) {
      case KIND_IL: NOC_PICK_RUN(0, 0, il_prof)
      case KIND_BASE: NOC_PICK_RUN(0, 0, base_prof)
      default: NOC_PICK_RUN(0, 0, gen_prof)
    }
  }
  const int bound = plain_bound(block_threads_impl(P.W, P.H, A.gx, A.gy));
  if (bound == MAX_THREADS) {
    switch (variant_kind(P)) {
      case KIND_IL: NOC_PICK_RUN(0, 0, il_xl)
      case KIND_LOCAL: NOC_PICK_RUN(0, 0, local_xl)
      case KIND_MIGRATE: NOC_PICK_RUN(0, 0, migrate_xl)
      case KIND_BASE: NOC_PICK_RUN(0, 0, base_xl)
      default: NOC_PICK_RUN(0, 0, gen_xl)
    }
  }
  if (bound == NARROW_THREADS) {
    switch (variant_kind(P)) {
      case KIND_IL: NOC_PICK_RUN(0, 0, il_narrow)
      case KIND_LOCAL: NOC_PICK_RUN(0, 0, local_narrow)
      case KIND_MIGRATE: NOC_PICK_RUN(0, 0, migrate_narrow)
      case KIND_BASE: NOC_PICK_RUN(0, 0, base_narrow)
      default: NOC_PICK_RUN(0, 0, gen_narrow)
    }
  }
  switch (variant_kind(P)) {
    case KIND_IL: NOC_PICK_RUN(0, 0, il)
    case KIND_LOCAL: NOC_PICK_RUN(0, 0, local)
    case KIND_MIGRATE: NOC_PICK_RUN(0, 0, migrate)
    case KIND_BASE: NOC_PICK_RUN(0, 0, base)
    default: NOC_PICK_RUN(0, 0, gen)
  }
}

#define NOC_PICK_KIND(fn, kind, w1, w2, ...)                                    \
  switch (kind) {                                                                \
    case KIND_IL: return fn##_##w1##_##w2##_il(__VA_ARGS__);                     \
    case KIND_LOCAL: return fn##_##w1##_##w2##_local(__VA_ARGS__);               \
    case KIND_MIGRATE: return fn##_##w1##_##w2##_migrate(__VA_ARGS__);           \
    case KIND_BASE: return fn##_##w1##_##w2##_base(__VA_ARGS__);                 \
    default: return fn##_##w1##_##w2##_gen(__VA_ARGS__);                        \
  }

#define NOC_PICK_KIND_NARROW(fn, kind, w1, w2, ...)                             \
  switch (kind) {                                                                \
    case KIND_IL: return fn##_##w1##_##w2##_il_narrow(__VA_ARGS__);              \
    case KIND_LOCAL: return fn##_##w1##_##w2##_local_narrow(__VA_ARGS__);        \
    case KIND_MIGRATE: return fn##_##w1##_##w2##_migrate_narrow(__VA_ARGS__);    \
    case KIND_BASE: return fn##_##w1##_##w2##_base_narrow(__VA_ARGS__);          \
    default: return fn##_##w1##_##w2##_gen_narrow(__VA_ARGS__);                  \
  }

#define NOC_PICK_KIND_XL(fn, kind, w1, w2, ...)                                 \
  switch (kind) {                                                                \
    case KIND_IL: return fn##_##w1##_##w2##_il_xl(__VA_ARGS__);                  \
    case KIND_LOCAL: return fn##_##w1##_##w2##_local_xl(__VA_ARGS__);            \
    case KIND_MIGRATE: return fn##_##w1##_##w2##_migrate_xl(__VA_ARGS__);        \
    case KIND_BASE: return fn##_##w1##_##w2##_base_xl(__VA_ARGS__);              \
    default: return fn##_##w1##_##w2##_gen_xl(__VA_ARGS__);                      \
  }

// co-resident CTAs of the plain loop at `threads` per CTA, for the build a
// launch of that size uses
#define NOC_PICK_KIND_PROF(fn, kind, w1, w2, ...)                               \
  switch (kind) {                                                                \
    case KIND_IL: return fn##_##w1##_##w2##_il_prof(__VA_ARGS__);                \
    case KIND_BASE: return fn##_##w1##_##w2##_base_prof(__VA_ARGS__);            \
    default: return fn##_##w1##_##w2##_gen_prof(__VA_ARGS__);                    \
  }

cudaError_t max_coresident_checked(const Params& P, int threads, int* out) {
  switch (way_class(P.l1_ways, P.l2_ways)) {
    case 0: return max_coresident_run_0_0_4_8_gen_checked(threads, out);
    case 1: return max_coresident_run_0_0_4_16_gen_checked(threads, out);
    default: return max_coresident_run_0_0_16_16_gen_checked(threads, out);
  }
}

cudaError_t max_coresident_prof(const Params& P, int threads, int* out) {
  const int kind = prof_kind(variant_kind(P));
  switch (way_class(P.l1_ways, P.l2_ways)) {
    case 0: NOC_PICK_KIND_PROF(max_coresident_run_0_0, kind, 4, 8, threads, out)
    case 1: NOC_PICK_KIND_PROF(max_coresident_run_0_0, kind, 4, 16, threads, out)
    default: NOC_PICK_KIND_PROF(max_coresident_run_0_0, kind, 16, 16, threads, out)
  }
}

cudaError_t max_coresident_ctas(const Params& P, int threads, int* out) {
  const int kind = variant_kind(P);
  if (plain_bound(threads) == MAX_THREADS) {
    switch (way_class(P.l1_ways, P.l2_ways)) {
      case 0: NOC_PICK_KIND_XL(max_coresident_run_0_0, kind, 4, 8, threads, out)
      case 1: NOC_PICK_KIND_XL(max_coresident_run_0_0, kind, 4, 16, threads, out)
      default: NOC_PICK_KIND_XL(max_coresident_run_0_0, kind, 16, 16, threads, out)
    }
  }
  if (threads <= NARROW_THREADS) {
    switch (way_class(P.l1_ways, P.l2_ways)) {
      case 0: NOC_PICK_KIND_NARROW(max_coresident_run_0_0, kind, 4, 8, threads, out)
      case 1: NOC_PICK_KIND_NARROW(max_coresident_run_0_0, kind, 4, 16, threads, out)
      default: NOC_PICK_KIND_NARROW(max_coresident_run_0_0, kind, 16, 16, threads, out)
    }
  }
  switch (way_class(P.l1_ways, P.l2_ways)) {
    case 0: NOC_PICK_KIND(max_coresident_run_0_0, kind, 4, 8, threads, out)
    case 1: NOC_PICK_KIND(max_coresident_run_0_0, kind, 4, 16, threads, out)
    default: NOC_PICK_KIND(max_coresident_run_0_0, kind, 16, 16, threads, out)
  }
}

int batch_way_class(int l1_ways, int l2_ways) { return way_class(l1_ways, l2_ways); }

cudaError_t launch_batch(const BatchArgs& B, int grid, int threads, int l1_ways, int l2_ways, int kind,
                         cudaStream_t s) {
  switch (way_class(l1_ways, l2_ways)) {
    case 0: NOC_PICK_KIND(launch_batch, kind, 4, 8, B, grid, threads, s)
    case 1: NOC_PICK_KIND(launch_batch, kind, 4, 16, B, grid, threads, s)
    default: NOC_PICK_KIND(launch_batch, kind, 16, 16, B, grid, threads, s)
  }
}

cudaError_t max_coresident_batch(int l1_ways, int l2_ways, int kind, int threads, int* out) {
  switch (way_class(l1_ways, l2_ways)) {
    case 0: NOC_PICK_KIND(max_coresident_batch, kind, 4, 8, threads, out)
    case 1: NOC_PICK_KIND(max_coresident_batch, kind, 4, 16, threads, out)
    default: NOC_PICK_KIND(max_coresident_batch, kind, 16, 16, threads, out)
  }
}

size_t run_smem_bytes(int threads) { return run_smem_bytes_impl(threads); }

int block_threads(int W, int H, int gx, int gy) { return block_threads_impl(W, H, gx, gy); }

static int grid_for(size_t n, int threads) {
  size_t g = (n + threads - 1) / threads;
  if (g > 4096) g = 4096;
  return (int)(g ? g : 1);
}

// ---------------------------------------------------------------- references
// Draw ahead, for every tile, the references it can issue in cycles
// [t0, t0 + n): those eligible by cycle t0 + n - 1 from its next_ref on, at most
// refcap.  One thread per (tile, slot), so the Philox work runs at full width
// instead of on the cycle kernel's serial path.
// One warp per tile: the window of references the tile's core may issue in
// cycles [t0, t0 + n), at most refcap, and no more than twice what the core
// took from its previous window plus 32 (a core that runs behind schedule
// takes far fewer than the schedule allows; past the window the cycle kernel
// draws in place, so the window's size never changes a result).  A window
// that still holds twice what the core took since it was drawn, plus 8, is
// kept as it is, so such cores redraw only every few launches.  Lanes draw
// consecutive references, so the window's stores are coalesced.
__global__ void gen_refs_kernel(const Params P, uint32_t t0, uint32_t n) {
  const size_t N = (size_t)P.N;
  const uint32_t lane = threadIdx.x & 31u;
  const size_t warps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t c = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < N; c += warps) {
    const uint32_t k0 = P.core[C_NEXT * N + c];
    uint32_t cnt = 0;
    if (P.period > 0 && P.mode != MODE_TRACE) {
      const unsigned long long last = (unsigned long long)(t0 + n - 1) / (unsigned)P.period;
      if (last + 1 > k0) cnt = (uint32_t)min(last + 1 - k0, (unsigned long long)P.refcap);
      const uint32_t prev_cnt = P.refcnt[c], prev_k0 = P.refk0[c];
      if (prev_cnt > 0 && k0 >= prev_k0) {
        const unsigned long long used = k0 - prev_k0;
        // the window drawn earlier still holds twice what the core took
        // since then, and a margin: keep it (warp-uniform)
        if ((unsigned long long)prev_k0 + prev_cnt >= k0 + 2 * used + 8) continue;
        cnt = (uint32_t)min((unsigned long long)cnt, 2 * used + 32);
      }
    }
    __syncwarp();
    if (lane == 0) {
      P.refk0[c] = k0;
      P.refcnt[c] = cnt;
    }
    for (uint32_t j = lane; j < cnt; j += 32) {
      uint32_t raw;
      if (draw_ref(P, (uint32_t)c, k0 + j, raw)) P.refbuf[c * (size_t)P.refcap + j] = raw;
    }
  }
}

cudaError_t launch_gen_refs(const Params& P, uint32_t t0, uint32_t n, cudaStream_t s) {
  gen_refs_kernel<<<grid_for((size_t)P.N * 32, 256), 256, 0, s>>>(P, t0, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- hashes
__global__ void dyn_hash_kernel(const Params P, uint32_t cycle, unsigned long long* out) {
  __shared__ unsigned long long red[32];
  unsigned long long acc = 0;
  const size_t N = (size_t)P.N;
  const uint32_t par = (cycle - 1u) & 1u;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < (uint32_t)P.N;
       r += gridDim.x * blockDim.x) {
    Tile T;
    load_tile(P, r, T);
    uint4 o[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) o[d] = P.glink[((size_t)par * 4 + d) * N + r];
    acc += tile_hash(P, T, o) + rob_hash(P, r);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

__device__ __forceinline__ void flit_words(const Params& P, uint4 f, unsigned long long& w0,
                                           unsigned long long& w1, unsigned long long& w2) {
  uint32_t ty = ftype(f);
  w0 = w1 = w2 = 0;
  if (!ty) return;
  w0 = (unsigned long long)ty | ((unsigned long long)fsrc(f) << 16) |
       ((unsigned long long)fdst(f) << 32) | ((unsigned long long)fa(f) << 48);
  w1 = (unsigned long long)fline(f) | ((unsigned long long)finject(P, f) << 32);
  w2 = (unsigned long long)fe(f) | ((unsigned long long)fage(P, f) << 32);
}

// full-state terms other than the dynamic hash: fold(0x18, cycle) plus one fold
// per valid L1 way (0x11), valid L2 way (0x12), core / service queue entry
// (0x13 / 0x14), memory-FIFO entry (0x15), directory entry (0x16) and
// forward entry (0x17)
__global__ void state_terms_kernel(const Params P, uint32_t cycle, unsigned long long* out) {
  __shared__ unsigned long long red[32];
  unsigned long long acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t N = (size_t)P.N;
  if (tid == 0) acc += hfold(hstart(0x18), cycle);
  // L1 ways
  const size_t n1 = N * P.l1_sets * P.l1_ways;
  for (size_t k = tid; k < n1; k += stride) {
    uint32_t v = P.l1[k];
    if (!(v & W_VALID)) continue;
    size_t way = k % P.l1_ways, set = (k / P.l1_ways) % P.l1_sets, r = k / ((size_t)P.l1_ways * P.l1_sets);
    unsigned long long h = hstart(0x11);
    h = hfold(h, r);
    h = hfold(h, set);
    h = hfold(h, way);
    h = hfold(h, (v & W_LINE) | ((unsigned long long)((v & W_DIRTY) ? 1 : 0) << 31));
    h = hfold(h, P.l1own[k]);
    h = hfold(h, wrank(v));
    acc += h;
  }
  // L2 ways
  const size_t n2 = N * P.l2_sets * P.l2_ways;
  for (size_t k = tid; k < n2; k += stride) {
    uint32_t v = P.l2[k];
    if (!(v & W_VALID)) continue;
    size_t way = k % P.l2_ways, set = (k / P.l2_ways) % P.l2_sets, r = k / ((size_t)P.l2_ways * P.l2_sets);
    unsigned long long h = hstart(0x12);
    h = hfold(h, r);
    h = hfold(h, set);
    h = hfold(h, way);
    h = hfold(h, v & W_LINE);
    h = hfold(h, (v & W_DIRTY) ? 1u : 0u);
    h = hfold(h, wrank(v));
    h = hfold(h, P.policy != POL_INTERLEAVED ? P.l2ep[k] : 0u);
    uint32_t mig = 0, hn = 0;
    const uint16_t* hp = nullptr;
    if (P.policy == POL_MIGRATE) {
      hp = P.l2hist + k * (size_t)P.hist_stride;
      hn = hp[0];
      mig = hp[1];
    }
    h = hfold(h, mig);
    h = hfold(h, hn);
    for (uint32_t j = 0; j < hn; ++j) h = hfold(h, hp[2 + j]);
    acc += h;
  }
  // core and service queues
  for (int qi = 0; qi < 2; ++qi) {
    const int cap = qi == 0 ? P.core_q : P.svc_q;
    const uint4* buf = qi == 0 ? P.cq : P.sq;
    const int field = qi == 0 ? C_CQ : C_SQ;
    const size_t nq = N * cap;
    for (size_t k = tid; k < nq; k += stride) {
      size_t r = k / cap, slot = k % cap;
      uint32_t q = P.core[field * N + r], head = q & 0xFFFFu, len = q >> 16;
      uint32_t pos = (uint32_t)((slot + cap - head) % cap);
      if (pos >= len) continue;
      unsigned long long w0, w1, w2;
      flit_words(P, buf[k], w0, w1, w2);
      unsigned long long h = hstart(0x13 + qi);
      h = hfold(h, r);
      h = hfold(h, pos);
      h = hfold(h, w0);
      h = hfold(h, w1);
      h = hfold(h, w2);
      acc += h;
    }
  }
  // memory-return FIFOs
  {
    const size_t nq = N * P.mem_q;
    for (size_t k = tid; k < nq; k += stride) {
      size_t r = k / P.mem_q, slot = k % P.mem_q;
      uint32_t q = P.core[C_MQ * N + r], head = q & 0xFFFFu, len = q >> 16;
      uint32_t pos = (uint32_t)((slot + P.mem_q - head) % P.mem_q);
      if (pos >= len) continue;
      uint4 m = P.mq[k];
      unsigned long long h = hstart(0x15);
      h = hfold(h, r);
      h = hfold(h, pos);
      h = hfold(h, m.x);
      h = hfold(h, m.y);
      h = hfold(h, m.z);
      acc += h;
    }
  }
  // directory
  if (P.policy != POL_INTERLEAVED)
    for (size_t k = tid; k < P.total_lines; k += stride) {
      uint32_t D = P.dir[k];
      if (D == DIR_NONE) continue;
      unsigned long long h = hstart(0x16);
      h = hfold(h, k);
      h = hfold(h, D & 0xFFFFu);
      h = hfold(h, D >> 16);
      acc += h;
    }
  // forward tables
  if (P.policy == POL_MIGRATE) {
    const size_t nf = N * P.fwd_cap;
    for (size_t k = tid; k < nf; k += stride) {
      size_t r = k / P.fwd_cap, slot = k % P.fwd_cap;
      uint32_t q = P.core[C_FWD * N + r], next = q & 0xFFFFu, n = q >> 16;
      uint32_t pos = (uint32_t)((next + 2 * P.fwd_cap - 1 - slot) % P.fwd_cap);
      if (pos >= n) continue;
      unsigned long long h = hstart(0x17);
      h = hfold(h, r);
      h = hfold(h, pos);
      h = hfold(h, P.fwd[k * 2]);
      h = hfold(h, P.fwd[k * 2 + 1]);
      acc += h;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}


cudaError_t launch_dyn_hash(const Params& P, uint32_t cycle, unsigned long long* out,
                            cudaStream_t s) {
  dyn_hash_kernel<<<grid_for(P.N, 256), 256, 0, s>>>(P, cycle, out);
  return cudaGetLastError();
}

cudaError_t launch_state_hash(const Params& P, uint32_t cycle, unsigned long long* out,
                              cudaStream_t s) {
  dyn_hash_kernel<<<grid_for(P.N, 256), 256, 0, s>>>(P, cycle, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  size_t n = (size_t)P.N * P.l2_sets * P.l2_ways;
  state_terms_kernel<<<grid_for(n, 256), 256, 0, s>>>(P, cycle, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- statistics
// block k reduces counter k over all tiles (a maximum for the latency max)
__global__ void reduce_stats_kernel(const Params P, int tile, unsigned long long* out) {
  __shared__ unsigned long long red[32];
  const int k = blockIdx.x;
  const size_t N = (size_t)P.N;
  unsigned long long acc = 0;
  if (tile >= 0) {
    if (threadIdx.x == 0) out[k] = P.stats[k * N + tile];
    return;
  }
  for (size_t r = threadIdx.x; r < N; r += blockDim.x) {
    unsigned long long v = P.stats[k * N + r];
    acc = k == S_LATMAX ? (v > acc ? v : acc) : acc + v;
  }
  if (k == S_LATMAX) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long u = __shfl_xor_sync(0xFFFFFFFFu, acc, o);
      acc = u > acc ? u : acc;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
      out[k] = m;
    }
    return;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[k] = acc;
}

cudaError_t launch_reduce_stats(const Params& P, int tile, unsigned long long* out,
                                cudaStream_t s) {
  reduce_stats_kernel<<<NSTAT, 256, 0, s>>>(P, tile, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- drain helpers
__global__ void count_busy_kernel(const Params P, uint32_t cycle, unsigned int* out) {
  __shared__ unsigned long long red[32];
  const size_t N = (size_t)P.N;
  const uint32_t par = (cycle - 1u) & 1u;
  unsigned long long c = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < (uint32_t)P.N;
       r += gridDim.x * blockDim.x) {
    Tile T;
    load_tile(P, r, T);
    uint4 o[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) o[d] = P.glink[((size_t)par * 4 + d) * N + r];
    c += tile_quiet(T, o) ? 0 : 1;
  }
  c = block_sum(c, red);
  if (threadIdx.x == 0 && c) atomicAdd(out, (unsigned)c);
}

cudaError_t launch_count_busy(const Params& P, uint32_t cycle, unsigned int* out, cudaStream_t s) {
  count_busy_kernel<<<grid_for(P.N, 256), 256, 0, s>>>(P, cycle, out);
  return cudaGetLastError();
}

__global__ void fill_u32_kernel(unsigned int* p, unsigned int v, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    p[k] = v;
}

cudaError_t launch_fill_u32(unsigned int* p, unsigned int v, size_t n, cudaStream_t s) {
  fill_u32_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
  return cudaGetLastError();
}

}  // namespace noc
