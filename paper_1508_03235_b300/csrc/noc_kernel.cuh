// noc_kernel.cuh -- the persistent cooperative cycle kernel (templates shared by
// the translation units noc_run*.cu and noc_batch.cu that instantiate them).
//
// Mapping (B300, sm_103a): the mesh is cut into gx x gy rectangles, one CTA
// each, one thread per tile.  A launch runs many simulated cycles.  Links
// between tiles of the same rectangle are exchanged through shared memory;
// links that cross a rectangle edge go through an L2-resident global buffer,
// and each CTA waits only for its (up to four) neighbouring CTAs to publish the
// previous cycle -- a neighbour-flag barrier instead of a grid-wide one.  The
// tile's own work of the next cycle (Phase 3 of this cycle, Phase 1 of the
// next) runs before that wait, so cache latency and barrier latency overlap.
#pragma once
#include <cstdio>

#include "noc_internal.h"

namespace noc {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait until *flag >= target (cycle counts, wrap-safe).  Returns 1 on success,
// 0 when the time limit ran out, -1 when another CTA already gave up.  The
// iteration count is bounded as well, so the wait always ends.
static __device__ int wait_ge(const unsigned* flag, unsigned target, const unsigned* abort_flag,
                       long long limit_ns) {
  const unsigned long long start = global_ns();
  for (unsigned it = 0; it < (1u << 28); ++it) {
    if ((int)(ld_acquire_u32(flag) - target) >= 0) return 1;
    if ((it & 31u) == 31u) {
      if (ld_acquire_u32(abort_flag)) return -1;
      if ((long long)(global_ns() - start) > limit_ns) return 0;
    }
  }
  return 0;
}

// ---------------------------------------------------------------- tile state I/O
static __device__ void load_tile(const Params& P, uint32_t r, Tile& T) {
  const size_t N = (size_t)P.N;
  const uint32_t* C = P.core;
  T.r = r;
  T.x = r % (uint32_t)P.W;
  T.y = r / (uint32_t)P.W;
  T.next_ref = C[C_NEXT * N + r];
  uint32_t b = C[C_FSMB * N + r];
  T.fsm = b & 0xFFu;
  T.fsm_write = (b >> 8) & 0xFFu;
  T.om_kind = (b >> 16) & 0xFFu;
  T.om_write = b >> 24;
  T.fsm_line = C[C_FLINE * N + r];
  T.fsm_timer = C[C_FTIMER * N + r];
  T.fsm_start = C[C_FSTART * N + r];
  T.om_line = C[C_OLINE * N + r];
  T.om_start = C[C_OSTART * N + r];
  T.om_timer = C[C_OTIMER * N + r];
  uint32_t e = C[C_EPOCH * N + r];
  T.epoch = e & 0xFFFFu;
  T.om_epoch = e >> 16;
  uint32_t q = C[C_CQ * N + r];
  T.cq_head = q & 0xFFFFu;
  T.cq_len = q >> 16;
  q = C[C_SQ * N + r];
  T.sq_head = q & 0xFFFFu;
  T.sq_len = q >> 16;
  q = C[C_MQ * N + r];
  T.mq_head = q & 0xFFFFu;
  T.mq_len = q >> 16;
  q = C[C_FWD * N + r];
  T.fwd_next = q & 0xFFFFu;
  T.fwd_n = q >> 16;
  const uint4 z = make_uint4(0, 0, 0, 0);
  T.cq_front = T.cq_len ? P.cq[(size_t)r * P.core_q + T.cq_head] : z;
  T.sq_front = T.sq_len ? P.sq[(size_t)r * P.svc_q + T.sq_head] : z;
  T.mq_front = T.mq_len ? P.mq[(size_t)r * P.mem_q + T.mq_head] : z;
  T.ej = z;
  T.rk0 = P.refbuf ? P.refk0[r] : 0;
  T.rcnt = P.refbuf ? P.refcnt[r] : 0;
  prefetch_next_ref(P, T);
  T.inj = P.stats[S_INJ * N + r];
  T.ejc = P.stats[S_EJ * N + r];
  T.defl = P.stats[S_DEFL * N + r];
  T.latsum = P.stats[S_LATSUM * N + r];
  T.latmax = P.stats[S_LATMAX * N + r];
  T.l2lsum = 0;
#pragma unroll
  for (int k = 0; k < NSMALL; ++k) T.sm[k] = 0;
}

static __device__ void store_tile(const Params& P, const Tile& T) {
  const size_t N = (size_t)P.N;
  const uint32_t r = T.r;
  uint32_t* C = P.core;
  C[C_NEXT * N + r] = T.next_ref;
  C[C_FSMB * N + r] = T.fsm | (T.fsm_write << 8) | (T.om_kind << 16) | (T.om_write << 24);
  C[C_FLINE * N + r] = T.fsm_line;
  C[C_FTIMER * N + r] = T.fsm_timer;
  C[C_FSTART * N + r] = T.fsm_start;
  C[C_OLINE * N + r] = T.om_line;
  C[C_OSTART * N + r] = T.om_start;
  C[C_OTIMER * N + r] = T.om_timer;
  C[C_EPOCH * N + r] = T.epoch | (T.om_epoch << 16);
  C[C_CQ * N + r] = T.cq_head | (T.cq_len << 16);
  C[C_SQ * N + r] = T.sq_head | (T.sq_len << 16);
  C[C_MQ * N + r] = T.mq_head | (T.mq_len << 16);
  C[C_FWD * N + r] = T.fwd_next | (T.fwd_n << 16);
  P.stats[S_INJ * N + r] = T.inj;
  P.stats[S_EJ * N + r] = T.ejc;
  P.stats[S_DEFL * N + r] = T.defl;
  P.stats[S_LATSUM * N + r] = T.latsum;
  P.stats[S_LATMAX * N + r] = T.latmax;
  if (T.l2lsum) P.stats[S_L2LSUM * N + r] += T.l2lsum;
#pragma unroll
  for (int k = 0; k < NSMALL; ++k)
    if (k + S_REFS != S_L2LSUM && T.sm[k]) P.stats[(size_t)(k + S_REFS) * N + r] += T.sm[k];
}

__device__ __forceinline__ bool tile_quiet(const Tile& T, const uint4 (&out)[4]) {
  bool q = T.cq_len == 0 && T.sq_len == 0 && T.mq_len == 0 && T.fsm == FSM_IDLE &&
           T.om_kind == OM_NONE;
#pragma unroll
  for (int d = 0; d < 4; ++d) q = q && ftype(out[d]) == T_NONE;
  return q;
}

// sum a 64-bit value over the CTA; the result is valid in thread 0
static __device__ unsigned long long block_sum(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  unsigned long long s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------- cycle kernel
// The cycle kernel runs CTAs of up to MAX_THREADS threads, one CTA per SM.
// The plain loop is built for three launch bounds: NARROW_THREADS (320; the
// 208x208 workload's 104x3 strips), where the compiler keeps 166 registers a
// thread; WIDE_THREADS (384, 154-166 registers); and MAX_THREADS (448, "xl").
// Each of an SM's four sub-partitions holds 16,384 registers and a CTA of
// more than 12 warps puts four warps on some of them, so the xl builds keep
// 128 registers a thread (and spill a little): with them every mesh of up to
// 148 x 448 tiles -- beyond the 65,535 that 16-bit tile indices allow -- fits
// one co-resident launch with one tile per thread.  A launch takes the
// smallest bound its CTAs fit, since more registers run faster (about 10 %
// between the 384 and 448 builds).  The traced and draining loops are built
// for MAX_THREADS, the per-phase profiled plain loop for PROF_THREADS (161
// registers, close to the production builds' timing).  The batch kernel's
// CTAs hold at most BATCH_MAX_THREADS threads (rectangles of at most 19 x 19).
constexpr int MAX_THREADS = 448;
constexpr int WIDE_THREADS = 384;
constexpr int NARROW_THREADS = 320;
constexpr int PROF_THREADS = 384;
constexpr int BATCH_MAX_THREADS = 384;

// The plain cycle loop polls the tagged slots of the links entering its
// rectangle either with one poll in flight (plain loads; NOC_POLL_STAGE 0, the
// batch kernel) or with two (NOC_POLL_STAGE 1, the single-simulation kernels):
// each round copies the needed slots into a per-thread shared-memory stage
// with cp.async while the previous copy is read, so a flit written by another
// SM is seen about half a global round trip sooner.  Rectangles that are all
// edge (two tiles thin) pay for the doubled polling, so the batch kernel, whose
// 8x8 rectangles are mostly edge, keeps one poll.  The stage starts on a
// 16-byte boundary, as cp.async needs: the bytes before it are a multiple of 16.
#ifndef NOC_POLL_STAGE
#define NOC_POLL_STAGE 1
#endif
// With the staged polls, the first copy of the next cycle's edge slots is
// issued between this warp's Phase 3 and Phase 1 (NOC_EARLY_POLL 1), so that
// its L2 round trip overlaps Phase 1 instead of following it.  Issued at the
// publish instead, the copy samples the neighbours' slots earlier and finds
// the flit less often: 1.5 % slower per cycle at 208 x 208 and 1.7 % at
// 64 x 64 than after Phase 3, but still 0.6 % faster than no early copy.
#ifndef NOC_EARLY_POLL
#define NOC_EARLY_POLL 1
#endif
// The profiled build of the plain loop (-DNOC_PHASE_PROFILE=1) reads the SM
// clock at each phase boundary, after the warp has reconverged, and adds each
// phase's clocks to A.prof at the end of the launch.
#ifndef NOC_PHASE_PROFILE
#define NOC_PHASE_PROFILE 0
#endif
#if NOC_PHASE_PROFILE
#define NOC_PROF_MARK(k)                   \
  do {                                     \
    __syncwarp();                          \
    const long long now_ = clock64();      \
    prof_[k] += (unsigned long long)(now_ - prof_t_); \
    prof_t_ = now_;                        \
  } while (0)
#else
#define NOC_PROF_MARK(k) \
  do {                   \
  } while (0)
#endif

// shared memory before the poll stage: links [2 parity][4 port][threads],
// histograms, reduction words
__host__ __device__ inline size_t run_smem_base_bytes(int threads) {
  return (size_t)threads * 8 * sizeof(uint4) + (2 * HIST_BINS + 2) * sizeof(uint32_t) +
         32 * sizeof(unsigned long long);
}
// the poll stage: [threads][2 buffers][4 ports][2 halves] tagged slots
__host__ __device__ inline size_t run_smem_bytes_impl(int threads, bool stage = NOC_POLL_STAGE != 0) {
  return run_smem_base_bytes(threads) + (stage ? (size_t)threads * 16 * sizeof(uint4) : 0);
}

inline int block_threads_impl(int W, int H, int gx, int gy) {
  int bw = (W + gx - 1) / gx, bh = (H + gy - 1) / gy;
  int a = bw * bh;
  return ((a + 31) / 32) * 32;
}

// Tiles on the perimeter of a bw x bh rectangle (only they have links that
// leave it); rectangles with a side <= 2 are all perimeter.
__device__ __forceinline__ int perim_count(int bw, int bh) {
  return (bw <= 2 || bh <= 2) ? bw * bh : 2 * bw + 2 * (bh - 2);
}
// Tile-to-thread order inside a bw x bh rectangle (thread i runs tile
// (lx, ly)): perimeter first (the top row, the side columns pairwise, the
// bottom row, then the interior row by row, so the few warps that touch the
// links leaving the rectangle are the first ones), row-major, or
// column-major.  Rectangles two tiles thin or less are row-major in all three.
enum : int { MAP_PERIMETER = 0, MAP_ROWS = 1, MAP_COLUMNS = 2 };
__device__ __forceinline__ int tile_index(int lx, int ly, int bw, int bh, int map) {
  if (map == MAP_COLUMNS && bw > 2 && bh > 2) return lx * bh + ly;
  if (map == MAP_ROWS || bw <= 2 || bh <= 2) return ly * bw + lx;
  if (ly == 0) return lx;
  if (ly == bh - 1) return bw + 2 * (bh - 2) + lx;
  if (lx == 0) return bw + 2 * (ly - 1);
  if (lx == bw - 1) return bw + 2 * (ly - 1) + 1;
  return perim_count(bw, bh) + (ly - 1) * (bw - 2) + (lx - 1);
}
__device__ __forceinline__ void tile_of(int i, int bw, int bh, int map, int& lx, int& ly) {
  if (map == MAP_COLUMNS && bw > 2 && bh > 2) {
    lx = i / bh;
    ly = i % bh;
    return;
  }
  if (map == MAP_ROWS || bw <= 2 || bh <= 2) {
    lx = i % bw;
    ly = i / bw;
    return;
  }
  const int np = perim_count(bw, bh);
  if (i < bw) {
    lx = i;
    ly = 0;
  } else if (i < bw + 2 * (bh - 2)) {
    const int j = i - bw;
    ly = 1 + j / 2;
    lx = (j & 1) ? bw - 1 : 0;
  } else if (i < np) {
    lx = i - bw - 2 * (bh - 2);
    ly = bh - 1;
  } else {
    const int j = i - np;
    ly = 1 + j / (bw - 2);
    lx = 1 + j % (bw - 2);
  }
}

// One CTA runs rectangle b of one simulation for A.n cycles.
template <bool HASH, bool DRAIN, int W1, int W2>
__device__ __forceinline__ void run_rect(const Params& P, const RunArgs& A, const int b,
                                         unsigned char* smem_raw) {
  const int nt = blockDim.x;
  uint4* sl = reinterpret_cast<uint4*>(smem_raw);  // [2 parity][4 port][nt]
  uint32_t* sh_hist = reinterpret_cast<uint32_t*>(sl + 8 * nt);
  unsigned long long* sh_red = reinterpret_cast<unsigned long long*>(sh_hist + 2 * HIST_BINS + 2);
  __shared__ int sh_abort;

  const int cx = b % A.gx, cy = b / A.gx;
  const int X0 = cx * P.W / A.gx, X1 = (cx + 1) * P.W / A.gx;
  const int Y0 = cy * P.H / A.gy, Y1 = (cy + 1) * P.H / A.gy;
  const int bw = X1 - X0, bh = Y1 - Y0;
  const int i = threadIdx.x;
  const bool active = i < bw * bh;
  int lx = 0, ly = 0;
  if (active) tile_of(i, bw, bh, A.thread_map, lx, ly);
  // shared-memory slots (thread indices) of the in-rectangle neighbours
  const int in_n = ly > 0 ? tile_index(lx, ly - 1, bw, bh, A.thread_map) : 0;
  const int in_s = ly < bh - 1 ? tile_index(lx, ly + 1, bw, bh, A.thread_map) : 0;
  const int in_e = lx < bw - 1 ? tile_index(lx + 1, ly, bw, bh, A.thread_map) : 0;
  const int in_w = lx > 0 ? tile_index(lx - 1, ly, bw, bh, A.thread_map) : 0;
  // the warps that hold the perimeter, which publish the cycle on their own
  // the warps holding perimeter tiles: the first ones in perimeter-first
  // order, any of them otherwise
  const int edge_threads = A.thread_map == MAP_PERIMETER ? ((perim_count(bw, bh) + 31) / 32) * 32 : nt;
  const bool edge_warp = i < edge_threads;
  const uint32_t x = X0 + lx, y = Y0 + ly, r = y * P.W + x;
  const size_t N = (size_t)P.N;
  const uint32_t exists = (y > 0 ? 1u << P_N : 0u) | (y + 1 < (uint32_t)P.H ? 1u << P_S : 0u) |
                          (x + 1 < (uint32_t)P.W ? 1u << P_E : 0u) | (x > 0 ? 1u << P_W : 0u);
  // links that leave the rectangle also go to the global buffer
  const uint32_t boundary = exists & ((ly == 0 ? 1u << P_N : 0u) | (ly == bh - 1 ? 1u << P_S : 0u) |
                                      (lx == bw - 1 ? 1u << P_E : 0u) | (lx == 0 ? 1u << P_W : 0u));
  // neighbouring CTA on each side (N, S, E, W), or -1
  const int nbr[4] = {cy > 0 ? b - A.gx : -1, cy + 1 < A.gy ? b + A.gx : -1,
                      cx + 1 < A.gx ? b + 1 : -1, cx > 0 ? b - 1 : -1};
  const bool alone = A.gx * A.gy == 1;

  for (int k = i; k < 2 * HIST_BINS; k += nt) sh_hist[k] = 0;
  if (i == 0) sh_abort = 0;

  Tile T;
  uint4 out[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) out[d] = make_uint4(0, 0, 0, 0);
  const uint32_t t0 = A.t0, tend = A.t0 + A.n;
  if (active) {
    load_tile(P, r, T);
    const uint32_t pin = (t0 - 1u) & 1u;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      out[d] = P.glink[((size_t)pin * 4 + d) * N + r];
      sl[(pin * 4 + d) * nt + i] = out[d];
    }
  }
  __syncthreads();
  if (active) phase1<W1, W2>(P, T, t0, A.draining != 0, sh_hist);

  uint32_t t = t0;
  for (; t < tend; ++t) {
    const uint32_t pin = (t - 1u) & 1u, pout = t & 1u;
    // ---- Phase 2: gather arrivals, route, publish outputs
    if (active) {
      uint4 in[4];
      const uint4 z = make_uint4(0, 0, 0, 0);
      const uint4* sp = sl + pin * 4 * nt;
      const uint4* gl = P.glink + (size_t)pin * 4 * N;
      in[P_N] = !(exists & (1u << P_N)) ? z
                : (ly > 0 ? sp[P_S * nt + in_n] : __ldcg(&gl[P_S * N + r - P.W]));
      in[P_S] = !(exists & (1u << P_S)) ? z
                : (ly < bh - 1 ? sp[P_N * nt + in_s] : __ldcg(&gl[P_N * N + r + P.W]));
      in[P_E] = !(exists & (1u << P_E)) ? z
                : (lx < bw - 1 ? sp[P_W * nt + in_e] : __ldcg(&gl[P_W * N + r + 1]));
      in[P_W] = !(exists & (1u << P_W)) ? z
                : (lx > 0 ? sp[P_E * nt + in_w] : __ldcg(&gl[P_E * N + r - 1]));
      route(P, T, t, in, exists, sl + pout * 4 * nt + i, nt, P.glink + (size_t)pout * 4 * N + r, N,
            boundary);
    }
    // publish: the perimeter warps meet at a named barrier, then one release
    // store orders all their link stores before the flag; the interior warps
    // go on without waiting
    if (!alone && edge_warp) {
      asm volatile("bar.sync 1, %0;" ::"r"(edge_threads) : "memory");
      if (i == 0 && b != A.silent_cta) st_release_u32(&P.flags[b * FLAG_SLOTS], t + 1);
    }
    // ---- Phase 3 of this cycle
    if (active) phase3<W1, W2>(P, T, t, sh_hist);
    if (HASH || DRAIN) {
#pragma unroll
      for (int d = 0; d < 4; ++d) out[d] = sl[(pout * 4 + d) * nt + i];
    }
    if (HASH) {
      unsigned long long h = active ? tile_hash(P, T, out) + rob_hash(P, r) : 0ull;
      h = block_sum(h, sh_red);
      if (i == 0) atomicAdd(&A.hash_trace[t - t0], h);
    }
    if (DRAIN) {
      unsigned long long q = (active && (!tile_quiet(T, out) || !rob_empty(P, r))) ? 1ull : 0ull;
      q = block_sum(q, sh_red);
      if (i == 0 && q) atomicAdd(&A.busy[t - t0], (unsigned)q);
    }
    if (t + 1 == tend) break;
    // ---- Phase 1 of the next cycle, then the neighbours' outputs of this one
    if (active) phase1<W1, W2>(P, T, t + 1, A.draining != 0, sh_hist);
    // lanes 0..3 each wait for one neighbouring CTA (N, S, E, W)
    if (i < 4 && nbr[i] >= 0) {
      int w = wait_ge(&P.flags[nbr[i] * FLAG_SLOTS], t + 1, A.abort_flag, A.wait_ns);
      if (w <= 0) {
        if (w == 0) {
          atomicExch(A.abort_flag, 1u);
          set_error(P, t + 1, ERR_TIMEOUT);
        }
        sh_abort = 1;
      }
    }
    __syncthreads();
    if (sh_abort) break;
  }

  // ---- end of launch: full link state of the last cycle, tile state, counters
  if (active) {
    const uint32_t plast = (t - (t == tend ? 1u : 0u)) & 1u;
#pragma unroll
    for (int d = 0; d < 4; ++d) P.glink[((size_t)plast * 4 + d) * N + r] = sl[(plast * 4 + d) * nt + i];
    store_tile(P, T);
  }
  __syncthreads();
  for (int k = i; k < 2 * HIST_BINS; k += nt)
    if (sh_hist[k]) atomicAdd(&P.hist[k], (unsigned long long)sh_hist[k]);
}

// ---------------------------------------------------------------- warp-flag loop
constexpr int WARPS_PER_CTA = MAX_THREADS / 32;

__device__ __forceinline__ void st_release_cta_shared(unsigned* p, unsigned v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v)
               : "memory");
}
__device__ __forceinline__ unsigned ld_volatile_shared(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}
__device__ __forceinline__ uint4 ld_volatile_shared_v4(const uint4* p) {
  uint4 v;
  asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p)))
               : "memory");
  return v;
}
// 16 bytes global -> shared through L2 (cp.async.cg), and the group controls
__device__ __forceinline__ void cp_async16_cg(uint4* smem, const uint4* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most the newest group is still in flight
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// One CTA runs rectangle b of one simulation for A.n cycles, with no CTA-wide
// barrier per cycle.  Inside the rectangle every warp publishes the cycle it
// has routed in a shared-memory flag and, before routing the next cycle, waits
// only for the warps that hold its tiles' neighbours.  Links that leave the
// rectangle go through tagged global slots (tag_store): the reader polls the
// slot itself until it carries the previous cycle's tag, so neither side
// needs a flag or a fence.  A warp is never more than one cycle ahead of a
// warp or tile that reads its outputs or writes its inputs (every link has a
// twin in the other direction, which the writer must have read first), which
// is all the double-buffered links need.  Threads map to tiles perimeter
// first, so the warps that touch global links are few.
template <int W1, int W2>
__device__ __forceinline__ void run_rect_warps(const Params& P, const RunArgs& A, const int b,
                                               unsigned char* smem_raw) {
  const int nt = blockDim.x;
  uint4* sl = reinterpret_cast<uint4*>(smem_raw);  // [2 parity][4 port][nt]
  uint32_t* sh_hist = reinterpret_cast<uint32_t*>(sl + 8 * nt);
  __shared__ unsigned wflag[WARPS_PER_CTA];
#if NOC_POLL_STAGE
  // this thread's poll stage: [2 buffers][4 ports][2 halves]
  uint4* stg = reinterpret_cast<uint4*>(smem_raw + run_smem_base_bytes(nt)) + (size_t)threadIdx.x * 16;
#endif

  const int cx = b % A.gx, cy = b / A.gx;
  const int X0 = cx * P.W / A.gx, X1 = (cx + 1) * P.W / A.gx;
  const int Y0 = cy * P.H / A.gy, Y1 = (cy + 1) * P.H / A.gy;
  const int bw = X1 - X0, bh = Y1 - Y0;
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
  const bool active = i < bw * bh;
  int lx = 0, ly = 0;
  if (active) tile_of(i, bw, bh, A.thread_map, lx, ly);
  const int in_n = ly > 0 ? tile_index(lx, ly - 1, bw, bh, A.thread_map) : 0;
  const int in_s = ly < bh - 1 ? tile_index(lx, ly + 1, bw, bh, A.thread_map) : 0;
  const int in_e = lx < bw - 1 ? tile_index(lx + 1, ly, bw, bh, A.thread_map) : 0;
  const int in_w = lx > 0 ? tile_index(lx - 1, ly, bw, bh, A.thread_map) : 0;
  const uint32_t x = X0 + lx, y = Y0 + ly, r = y * P.W + x;
  const size_t N = (size_t)P.N;
  const bool draining = A.draining != 0;
  const uint32_t exists = !active ? 0u
                          : (y > 0 ? 1u << P_N : 0u) | (y + 1 < (uint32_t)P.H ? 1u << P_S : 0u) |
                                (x + 1 < (uint32_t)P.W ? 1u << P_E : 0u) | (x > 0 ? 1u << P_W : 0u);
  // links that cross the rectangle's edge, in and out
  const uint32_t boundary = exists & ((ly == 0 ? 1u << P_N : 0u) | (ly == bh - 1 ? 1u << P_S : 0u) |
                                      (lx == bw - 1 ? 1u << P_E : 0u) | (lx == 0 ? 1u << P_W : 0u));
  // the silent rectangle (a test of the bounded waits) never writes its edges
  const uint32_t edge_out = b == A.silent_cta ? 0u : boundary;

  // the warps of this CTA that hold in-rectangle neighbours of this warp's
  // tiles; lane l < WARPS_PER_CTA polls warp l's flag
  unsigned lm = 0;
  if (active) {
    if (ly > 0) lm |= 1u << (in_n >> 5);
    if (ly < bh - 1) lm |= 1u << (in_s >> 5);
    if (lx < bw - 1) lm |= 1u << (in_e >> 5);
    if (lx > 0) lm |= 1u << (in_w >> 5);
  }
  lm = __reduce_or_sync(0xFFFFFFFFu, lm) & ~(1u << warp);
  const bool poll_local = lane < WARPS_PER_CTA && ((lm >> lane) & 1u);
  // tagged slot (in uint4) of this tile's input across each edge, parity 0:
  // the neighbour's output port facing this tile
  const size_t pstride = 2 * 4 * N;  // uint4 per parity
  uint32_t rin[4] = {0, 0, 0, 0};
  if (boundary & (1u << P_N)) rin[P_N] = (P_S * (uint32_t)N + r - P.W) * 2;
  if (boundary & (1u << P_S)) rin[P_S] = (P_N * (uint32_t)N + r + P.W) * 2;
  if (boundary & (1u << P_E)) rin[P_E] = (P_W * (uint32_t)N + r + 1) * 2;
  if (boundary & (1u << P_W)) rin[P_W] = (P_E * (uint32_t)N + r - 1) * 2;

  for (int k = i; k < 2 * HIST_BINS; k += nt) sh_hist[k] = 0;
  const uint32_t t0 = A.t0, tend = A.t0 + A.n;
  if (i < WARPS_PER_CTA) wflag[i] = t0;

  Tile T;
  if (active) {
    load_tile(P, r, T);
    const uint32_t pin = (t0 - 1u) & 1u;
#pragma unroll
    for (int d = 0; d < 4; ++d) sl[(pin * 4 + d) * nt + i] = P.glink[((size_t)pin * 4 + d) * N + r];
  }
  __syncthreads();
  if (active) phase1<W1, W2>(P, T, t0, draining, sh_hist);
#if NOC_PHASE_PROFILE
  unsigned long long prof_[5] = {0, 0, 0, 0, 0};
  long long prof_t_ = clock64();
#endif

  uint32_t t = t0;
  for (; t < tend; ++t) {
    const uint32_t pin = (t - 1u) & 1u, pout = t & 1u;
    // the injection candidate needs only this tile's state: taken before the wait
    const InjCand ic = active ? inj_candidate(P, T) : InjCand{make_uint4(0, 0, 0, 0), 0u, 0};
    uint4 in[4];
    const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int d = 0; d < 4; ++d) in[d] = z;
    if (t == t0) {
      // the previous launch's last outputs, complete in the global links
      const uint4* gl = P.glink + (size_t)pin * 4 * N;
      if (boundary & (1u << P_N)) in[P_N] = __ldcg(&gl[P_S * N + r - P.W]);
      if (boundary & (1u << P_S)) in[P_S] = __ldcg(&gl[P_N * N + r + P.W]);
      if (boundary & (1u << P_E)) in[P_E] = __ldcg(&gl[P_W * N + r + 1]);
      if (boundary & (1u << P_W)) in[P_W] = __ldcg(&gl[P_E * N + r - 1]);
    } else {
      // wait for the neighbours' outputs of cycle t-1: flags of the warps
      // inside the rectangle, the tagged slots themselves across its edges
      const uint32_t tag = link_tag(t - 1);
      const uint4* gt = P.gtag + pin * pstride;
      uint32_t need = boundary;
      // the clock is read at the first periodic check, not on every cycle's
      // entry: the wait's limit then runs from that check
      unsigned long long start = 0;
      bool aborted = false;
#if NOC_POLL_STAGE
      // two polls in flight: each round issues the next copy of the needed
      // slots into one stage buffer and then reads the copy in the other.  A
      // copy still in flight when the wait ends lands in the buffer that the
      // next cycle's first round writes; it holds the other parity's tags,
      // which never match, and cp.async.wait_group retires it first.
#if NOC_EARLY_POLL
      if (t == t0 + 1)   // later cycles issued their first copy after Phase 3
#endif
      {
#pragma unroll
        for (int d = 0; d < 4; ++d)
          if (need & (1u << d)) {
            cp_async16_cg(stg + d * 2, gt + rin[d]);
            cp_async16_cg(stg + d * 2 + 1, gt + rin[d] + 1);
          }
        cp_async_commit();
      }
#endif
      for (unsigned it = 0;; ++it) {
#if NOC_POLL_STAGE
        const uint32_t bo = (it & 1u) * 8, bn = 8 - bo;
#pragma unroll
        for (int d = 0; d < 4; ++d)
          if (need & (1u << d)) {
            cp_async16_cg(stg + bn + d * 2, gt + rin[d]);
            cp_async16_cg(stg + bn + d * 2 + 1, gt + rin[d] + 1);
          }
        cp_async_commit();
        cp_async_wait1();
#pragma unroll
        for (int d = 0; d < 4; ++d)
          if (need & (1u << d)) {
            const uint4 a = ld_volatile_shared_v4(stg + bo + d * 2);
            const uint4 c = ld_volatile_shared_v4(stg + bo + d * 2 + 1);
            if (tag_decode(a, c, tag, in[d])) need &= ~(1u << d);
          }
#else
#pragma unroll
        for (int d = 0; d < 4; ++d)
          if (need & (1u << d)) {
            const uint4 a = ld_relaxed_v4(gt + rin[d]), c = ld_relaxed_v4(gt + rin[d] + 1);
            if (tag_decode(a, c, tag, in[d])) need &= ~(1u << d);
          }
#endif
        const bool ok = need == 0 && (!poll_local || (int)(ld_volatile_shared(&wflag[lane]) - t) >= 0);
        if (__all_sync(0xFFFFFFFFu, ok)) break;
        if ((it & 31u) == 31u) {
          bool stop = ld_acquire_u32(A.abort_flag) != 0 || it >= (1u << 28);
          if (start == 0) start = global_ns();
          if (!stop && (long long)(global_ns() - start) > A.wait_ns) {
            stop = true;
            if (lane == 0) {
              atomicExch(A.abort_flag, 1u);
              set_error(P, t, ERR_TIMEOUT);
            }
          }
          if (__any_sync(0xFFFFFFFFu, stop)) {
            aborted = true;
            break;
          }
        }
      }
      if (aborted) break;
      // acquire: the flag loads above, then the neighbours' link stores
      asm volatile("fence.acq_rel.cta;" ::: "memory");
    }
    NOC_PROF_MARK(0);
    // ---- Phase 2 (own tile): the in-rectangle arrivals, route, store outputs
    if (active) {
      const uint4* sp = sl + pin * 4 * nt;
      if ((exists & ~boundary) & (1u << P_N)) in[P_N] = sp[P_S * nt + in_n];
      if ((exists & ~boundary) & (1u << P_S)) in[P_S] = sp[P_N * nt + in_s];
      if ((exists & ~boundary) & (1u << P_E)) in[P_E] = sp[P_W * nt + in_e];
      if ((exists & ~boundary) & (1u << P_W)) in[P_W] = sp[P_E * nt + in_w];
      route_ranked(P, T, t, in, exists, sl + pout * 4 * nt + i, nt, P.gtag + pout * pstride + (size_t)r * 2,
                   2 * N, NOC_POLL_STAGE ? 0u : edge_out, ic);
    }
    NOC_PROF_MARK(1);
    // ---- publish: this warp has routed cycle t (the warp barrier orders every
    // lane's shared link stores before lane 0's flag store, a release at CTA
    // scope that the waiting warps' acquire fence pairs with).  With two polls
    // in flight (the single-simulation kernels) the outputs that leave the
    // rectangle are copied to their tagged global slots after it: they need no
    // ordering, so the flag goes out first (0.7 % faster per cycle at 208 x 208,
    // 0.2 % at 64 x 64).  The batch kernel, whose small rectangles are mostly
    // edge, stores them inside the router (1 % more simulations/s that way).
    __syncwarp();
    if (lane == 0) st_release_cta_shared(&wflag[warp], t + 1);
#if NOC_POLL_STAGE
    store_edges(sl + pout * 4 * nt + i, nt, P.gtag + pout * pstride + (size_t)r * 2, 2 * N, edge_out, t);
#endif
    NOC_PROF_MARK(2);
    // ---- Phase 3 of this cycle and Phase 1 of the next (own tile only)
    if (active) phase3<W1, W2>(P, T, t, sh_hist);
#if NOC_POLL_STAGE && NOC_EARLY_POLL
    // the first copy of the slots the next cycle's wait reads (the outputs of
    // cycle t), into the stage half that wait reads first
    if (t + 1 != tend && t != t0) {
      const uint4* gtn = P.gtag + (t & 1u) * pstride;
#pragma unroll
      for (int d = 0; d < 4; ++d)
        if (boundary & (1u << d)) {
          cp_async16_cg(stg + d * 2, gtn + rin[d]);
          cp_async16_cg(stg + d * 2 + 1, gtn + rin[d] + 1);
        }
      cp_async_commit();
    }
#endif
    NOC_PROF_MARK(3);
    if (active && t + 1 != tend) phase1<W1, W2>(P, T, t + 1, draining, sh_hist);
    NOC_PROF_MARK(4);
  }
#if NOC_PHASE_PROFILE
  if (lane == 0 && A.prof) {
#pragma unroll
    for (int k = 0; k < 5; ++k) atomicAdd(&A.prof[k], prof_[k]);
    atomicAdd(&A.prof[5], (unsigned long long)(t - t0));
  }
#endif

  // ---- end of launch: full link state of the last cycle, tile state, counters
#if NOC_POLL_STAGE
  asm volatile("cp.async.wait_all;" ::: "memory");   // no stage copy outlives the CTA
#endif
  __syncthreads();
  if (active) {
    const uint32_t plast = (t - (t == tend ? 1u : 0u)) & 1u;
#pragma unroll
    for (int d = 0; d < 4; ++d) P.glink[((size_t)plast * 4 + d) * N + r] = sl[(plast * 4 + d) * nt + i];
    store_tile(P, T);
  }
  __syncthreads();
  for (int k = i; k < 2 * HIST_BINS; k += nt)
    if (sh_hist[k]) atomicAdd(&P.hist[k], (unsigned long long)sh_hist[k]);
}

// POLV names the device code's specialisation (-1: every policy, mode and
// option; -2: every policy and mode without the packet, write-back,
// directory-node and age options; p: the L2 policy p in cache mode only), so the
// instantiations of translation units built with different specialisation
// flags are distinct kernels.
// LB is the launch bound: the most threads a CTA of this build may have.
template <bool HASH, bool DRAIN, int W1, int W2, int POLV, int LB>
__global__ void __launch_bounds__(LB, 1)
    run_kernel(const __grid_constant__ Params P, const __grid_constant__ RunArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (!HASH && !DRAIN)
    run_rect_warps<W1, W2>(P, A, blockIdx.x, smem_raw);
  else
    run_rect<HASH, DRAIN, W1, W2>(P, A, blockIdx.x, smem_raw);
}

template <bool H, bool D, int W1, int W2, int POLV, int LB>
static cudaError_t prepare_run() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(run_kernel<H, D, W1, W2, POLV, LB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)run_smem_bytes_impl(LB));
  if (e == cudaSuccess) done = true;
  return e;
}

template <bool H, bool D, int W1, int W2, int POLV, int LB>
static cudaError_t launch_run_t(const Params& P, const RunArgs& A, cudaStream_t s) {
  cudaError_t e = prepare_run<H, D, W1, W2, POLV, LB>();
  if (e != cudaSuccess) return e;
  const int threads = block_threads_impl(P.W, P.H, A.gx, A.gy);
  if (threads > LB) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&P, (void*)&A};
  return cudaLaunchCooperativeKernel((const void*)run_kernel<H, D, W1, W2, POLV, LB>, dim3(A.gx * A.gy),
                                     dim3(threads), args, run_smem_bytes_impl(threads), s);
}

template <int W1, int W2, int POLV, int LB>
static cudaError_t max_coresident_run_t(int threads, int* out) {
  cudaError_t e = prepare_run<false, false, W1, W2, POLV, LB>();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, run_kernel<false, false, W1, W2, POLV, LB>, threads,
                                                    run_smem_bytes_impl(threads));
  if (e != cudaSuccess) return e;
  *out = per * sms;
  return cudaSuccess;
}

}  // namespace noc
