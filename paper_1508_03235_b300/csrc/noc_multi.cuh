// noc_multi.cuh -- the plain cycle loop with K tiles per thread, for meshes
// that do not fit one co-resident launch of one thread per tile.
//
// The one-tile loop keeps each tile's core record, queue heads and counters in
// its thread's registers for a whole launch, so a mesh must fit the GPU's
// co-resident threads: 148 SMs x 448 at the wide builds' 128 registers, which
// covers every mesh the 16-bit tile indices allow whose shape cuts into at
// most 148 rectangles of at most 448 tiles.  Here a thread runs tiles i and
// i + blockDim.x (K = 2) of its CTA rectangle, so a rectangle holds up to
// 2 x 256 tiles, for the shapes that do not cut that way.  A tile's state
// lives in a 66-word record in shared memory for the whole launch (read from
// the arena at the launch's start, written back at its end, as the one-tile
// loop does with registers) and is moved into registers around each cycle of
// its simulated work.  With it a B300 holds every mesh of up to 65,535 tiles,
// the limit of the 16-bit tile indices a flit carries.
//
// Per warp and cycle t: wait until every input of every one of its tiles
// carries cycle t - 1 (shared-memory flags of the warps holding in-rectangle
// neighbours, tagged global slots across the rectangle's edge, one poll in
// flight), then for each of its tiles: take the state from its record, route
// cycle t, Phase 3 of t, Phase 1 of t + 1, put the state back; then publish
// t + 1.  The order of
// the phases per tile is the one-tile loop's; only when the warp publishes
// changes (after all its tiles' Phases 3 and 1 rather than before), which no
// result depends on.  A warp waits for all its tiles' inputs before routing
// any of them, so, as in the one-tile loop, no warp is more than one cycle
// ahead of a warp or tile that reads its outputs.
#pragma once
#include "noc_kernel.cuh"

namespace noc {

constexpr int MULTI_K = 2;            // tiles per thread
constexpr int MULTI_THREADS = 256;    // threads per CTA (all registers for 255 each)
constexpr int MULTI_WARPS = MULTI_THREADS / 32;
constexpr int REC_WORDS = 43 + NSMALL;  // 32-bit words of a tile's state record

// shared memory: tile records [REC_WORDS][K * threads], links
// [2 parity][4 port][K * threads], histograms
__host__ __device__ inline size_t multi_smem_bytes(int threads) {
  return (size_t)MULTI_K * threads * (REC_WORDS * sizeof(uint32_t) + 8 * sizeof(uint4)) +
         (2 * HIST_BINS + 2) * sizeof(uint32_t);
}

// A tile's state to and from its record: word w of the record of rectangle
// slot j at rec[w * cap + j] (consecutive threads, consecutive words: no bank
// conflicts).  Everything a tile carries from one cycle to the next; the
// ejected flit is set by the router and consumed by Phase 3 in one cycle.
__device__ __forceinline__ void rec_u64(uint32_t* rec, int cap, int w, unsigned long long v) {
  rec[w * cap] = (uint32_t)v;
  rec[(w + 1) * cap] = (uint32_t)(v >> 32);
}
__device__ __forceinline__ unsigned long long rec_get_u64(const uint32_t* rec, int cap, int w) {
  return (unsigned long long)rec[w * cap] | ((unsigned long long)rec[(w + 1) * cap] << 32);
}
__device__ __forceinline__ void rec_uint4(uint32_t* rec, int cap, int w, uint4 v) {
  rec[w * cap] = v.x;
  rec[(w + 1) * cap] = v.y;
  rec[(w + 2) * cap] = v.z;
  rec[(w + 3) * cap] = v.w;
}
__device__ __forceinline__ uint4 rec_get_uint4(const uint32_t* rec, int cap, int w) {
  return make_uint4(rec[w * cap], rec[(w + 1) * cap], rec[(w + 2) * cap], rec[(w + 3) * cap]);
}
static __device__ void tile_to_record(const Tile& T, uint32_t* rec, int cap) {
  rec[0] = T.r;
  rec[1 * cap] = T.x | (T.y << 16);
  rec[2 * cap] = T.next_ref;
  rec[3 * cap] = T.fsm | (T.fsm_write << 8) | (T.om_kind << 16) | (T.om_write << 24);
  rec[4 * cap] = T.fsm_line;
  rec[5 * cap] = T.fsm_timer;
  rec[6 * cap] = T.fsm_start;
  rec[7 * cap] = T.om_line;
  rec[8 * cap] = T.om_start;
  rec[9 * cap] = T.om_timer;
  rec[10 * cap] = T.epoch | (T.om_epoch << 16);
  rec[11 * cap] = T.cq_head | (T.cq_len << 16);
  rec[12 * cap] = T.sq_head | (T.sq_len << 16);
  rec[13 * cap] = T.mq_head | (T.mq_len << 16);
  rec[14 * cap] = T.fwd_next | (T.fwd_n << 16);
  rec_uint4(rec, cap, 15, T.cq_front);
  rec_uint4(rec, cap, 19, T.sq_front);
  rec_uint4(rec, cap, 23, T.mq_front);
  rec[27 * cap] = T.pf_raw;
  rec[28 * cap] = T.pf_ok;
  rec[29 * cap] = T.rk0;
  rec[30 * cap] = T.rcnt;
  rec_u64(rec, cap, 31, T.inj);
  rec_u64(rec, cap, 33, T.ejc);
  rec_u64(rec, cap, 35, T.defl);
  rec_u64(rec, cap, 37, T.latsum);
  rec_u64(rec, cap, 39, T.latmax);
  rec_u64(rec, cap, 41, T.l2lsum);
#pragma unroll
  for (int k = 0; k < NSMALL; ++k) rec[(43 + k) * cap] = T.sm[k];
}
static __device__ void tile_from_record(Tile& T, const uint32_t* rec, int cap) {
  T.r = rec[0];
  const uint32_t xy = rec[1 * cap];
  T.x = xy & 0xFFFFu;
  T.y = xy >> 16;
  T.next_ref = rec[2 * cap];
  const uint32_t b = rec[3 * cap];
  T.fsm = b & 0xFFu;
  T.fsm_write = (b >> 8) & 0xFFu;
  T.om_kind = (b >> 16) & 0xFFu;
  T.om_write = b >> 24;
  T.fsm_line = rec[4 * cap];
  T.fsm_timer = rec[5 * cap];
  T.fsm_start = rec[6 * cap];
  T.om_line = rec[7 * cap];
  T.om_start = rec[8 * cap];
  T.om_timer = rec[9 * cap];
  const uint32_t e = rec[10 * cap];
  T.epoch = e & 0xFFFFu;
  T.om_epoch = e >> 16;
  uint32_t q = rec[11 * cap];
  T.cq_head = q & 0xFFFFu;
  T.cq_len = q >> 16;
  q = rec[12 * cap];
  T.sq_head = q & 0xFFFFu;
  T.sq_len = q >> 16;
  q = rec[13 * cap];
  T.mq_head = q & 0xFFFFu;
  T.mq_len = q >> 16;
  q = rec[14 * cap];
  T.fwd_next = q & 0xFFFFu;
  T.fwd_n = q >> 16;
  T.cq_front = rec_get_uint4(rec, cap, 15);
  T.sq_front = rec_get_uint4(rec, cap, 19);
  T.mq_front = rec_get_uint4(rec, cap, 23);
  T.ej = make_uint4(0, 0, 0, 0);
  T.pf_raw = rec[27 * cap];
  T.pf_ok = rec[28 * cap];
  T.rk0 = rec[29 * cap];
  T.rcnt = rec[30 * cap];
  T.inj = rec_get_u64(rec, cap, 31);
  T.ejc = rec_get_u64(rec, cap, 33);
  T.defl = rec_get_u64(rec, cap, 35);
  T.latsum = rec_get_u64(rec, cap, 37);
  T.latmax = rec_get_u64(rec, cap, 39);
  T.l2lsum = rec_get_u64(rec, cap, 41);
#pragma unroll
  for (int k = 0; k < NSMALL; ++k) T.sm[k] = rec[(43 + k) * cap];
}
inline int multi_block_threads(int W, int H, int gx, int gy) {
  const int bw = (W + gx - 1) / gx, bh = (H + gy - 1) / gy;
  const int per = (bw * bh + MULTI_K - 1) / MULTI_K;
  return ((per + 31) / 32) * 32;
}

template <int W1, int W2>
__device__ __forceinline__ void run_rect_multi(const Params& P, const RunArgs& A, const int b,
                                               unsigned char* smem_raw) {
  constexpr int K = MULTI_K;
  const int nt = blockDim.x, cap = K * nt;
  uint32_t* recs = reinterpret_cast<uint32_t*>(smem_raw);  // [REC_WORDS][cap]
  uint4* sl = reinterpret_cast<uint4*>(recs + (size_t)REC_WORDS * cap);  // [2 parity][4 port][cap]
  uint32_t* sh_hist = reinterpret_cast<uint32_t*>(sl + 8 * cap);
  __shared__ unsigned wflag[MULTI_WARPS];

  const int cx = b % A.gx, cy = b / A.gx;
  const int X0 = cx * P.W / A.gx, X1 = (cx + 1) * P.W / A.gx;
  const int Y0 = cy * P.H / A.gy, Y1 = (cy + 1) * P.H / A.gy;
  const int bw = X1 - X0, bh = Y1 - Y0;
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
  const size_t N = (size_t)P.N;
  const bool draining = A.draining != 0;
  const size_t pstride = 2 * 4 * N;  // uint4 per parity of the tagged slots

  // per tile slot k of this thread: rectangle index j = i + k * nt
  bool act[K];
  uint32_t r[K], exists[K], boundary[K], edge_out[K], rin[K][4];
  int nb[K][4];  // shared-memory slot (rectangle index) of each in-rectangle neighbour
  unsigned lm = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = i + k * nt;
    act[k] = j < bw * bh;
    int lx = 0, ly = 0;
    if (act[k]) tile_of(j, bw, bh, A.thread_map, lx, ly);
    nb[k][P_N] = ly > 0 ? tile_index(lx, ly - 1, bw, bh, A.thread_map) : 0;
    nb[k][P_S] = ly < bh - 1 ? tile_index(lx, ly + 1, bw, bh, A.thread_map) : 0;
    nb[k][P_E] = lx < bw - 1 ? tile_index(lx + 1, ly, bw, bh, A.thread_map) : 0;
    nb[k][P_W] = lx > 0 ? tile_index(lx - 1, ly, bw, bh, A.thread_map) : 0;
    const uint32_t x = X0 + lx, y = Y0 + ly;
    r[k] = y * P.W + x;
    exists[k] = !act[k] ? 0u
                : (y > 0 ? 1u << P_N : 0u) | (y + 1 < (uint32_t)P.H ? 1u << P_S : 0u) |
                      (x + 1 < (uint32_t)P.W ? 1u << P_E : 0u) | (x > 0 ? 1u << P_W : 0u);
    boundary[k] = exists[k] & ((ly == 0 ? 1u << P_N : 0u) | (ly == bh - 1 ? 1u << P_S : 0u) |
                               (lx == bw - 1 ? 1u << P_E : 0u) | (lx == 0 ? 1u << P_W : 0u));
    edge_out[k] = b == A.silent_cta ? 0u : boundary[k];
    // the warps of this CTA holding this tile's in-rectangle neighbours
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if ((exists[k] & ~boundary[k]) & (1u << d)) lm |= 1u << ((nb[k][d] % nt) >> 5);
    rin[k][P_N] = (boundary[k] & (1u << P_N)) ? (P_S * (uint32_t)N + r[k] - P.W) * 2 : 0;
    rin[k][P_S] = (boundary[k] & (1u << P_S)) ? (P_N * (uint32_t)N + r[k] + P.W) * 2 : 0;
    rin[k][P_E] = (boundary[k] & (1u << P_E)) ? (P_W * (uint32_t)N + r[k] + 1) * 2 : 0;
    rin[k][P_W] = (boundary[k] & (1u << P_W)) ? (P_E * (uint32_t)N + r[k] - 1) * 2 : 0;
  }
  lm = __reduce_or_sync(0xFFFFFFFFu, lm) & ~(1u << warp);
  const bool poll_local = lane < MULTI_WARPS && ((lm >> lane) & 1u);

  for (int k = i; k < 2 * HIST_BINS; k += nt) sh_hist[k] = 0;
  const uint32_t t0 = A.t0, tend = A.t0 + A.n;
  if (i < MULTI_WARPS) wflag[i] = t0;
  {
    const uint32_t pin = (t0 - 1u) & 1u;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int j = i + k * nt;
#pragma unroll
        for (int d = 0; d < 4; ++d) sl[(pin * 4 + d) * cap + j] = P.glink[((size_t)pin * 4 + d) * N + r[k]];
      }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (act[k]) {
      Tile T;
      load_tile(P, r[k], T);
      phase1<W1, W2>(P, T, t0, draining, sh_hist);
      tile_to_record(T, recs + i + k * nt, cap);
    }

  uint32_t t = t0;
  for (; t < tend; ++t) {
    const uint32_t pin = (t - 1u) & 1u, pout = t & 1u;
    uint4 ein[K][4];  // inputs across the rectangle's edge
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int d = 0; d < 4; ++d) ein[k][d] = make_uint4(0, 0, 0, 0);
    if (t == t0) {
      // the previous launch's last outputs, complete in the global links
      const uint4* gl = P.glink + (size_t)pin * 4 * N;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (boundary[k] & (1u << P_N)) ein[k][P_N] = __ldcg(&gl[P_S * N + r[k] - P.W]);
        if (boundary[k] & (1u << P_S)) ein[k][P_S] = __ldcg(&gl[P_N * N + r[k] + P.W]);
        if (boundary[k] & (1u << P_E)) ein[k][P_E] = __ldcg(&gl[P_W * N + r[k] + 1]);
        if (boundary[k] & (1u << P_W)) ein[k][P_W] = __ldcg(&gl[P_E * N + r[k] - 1]);
      }
    } else {
      const uint32_t tag = link_tag(t - 1);
      const uint4* gt = P.gtag + pin * pstride;
      uint32_t need[K];
#pragma unroll
      for (int k = 0; k < K; ++k) need[k] = boundary[k];
      unsigned long long start = 0;
      bool aborted = false;
      for (unsigned it = 0;; ++it) {
        bool got = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
          for (int d = 0; d < 4; ++d)
            if (need[k] & (1u << d)) {
              const uint4 a = ld_relaxed_v4(gt + rin[k][d]), c = ld_relaxed_v4(gt + rin[k][d] + 1);
              if (tag_decode(a, c, tag, ein[k][d])) need[k] &= ~(1u << d);
            }
          got = got && need[k] == 0;
        }
        const bool ok = got && (!poll_local || (int)(ld_volatile_shared(&wflag[lane]) - t) >= 0);
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
      asm volatile("fence.acq_rel.cta;" ::: "memory");   // acquire
    }
    // ---- each tile: route cycle t, Phase 3 of t, Phase 1 of t + 1
    const uint4* sp = sl + pin * 4 * cap;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int j = i + k * nt;
        Tile T;
        tile_from_record(T, recs + j, cap);
        const InjCand ic = inj_candidate(P, T);
        uint4 in[4];
        const uint32_t local = exists[k] & ~boundary[k];
        in[P_N] = (local & (1u << P_N)) ? sp[P_S * cap + nb[k][P_N]] : ein[k][P_N];
        in[P_S] = (local & (1u << P_S)) ? sp[P_N * cap + nb[k][P_S]] : ein[k][P_S];
        in[P_E] = (local & (1u << P_E)) ? sp[P_W * cap + nb[k][P_E]] : ein[k][P_E];
        in[P_W] = (local & (1u << P_W)) ? sp[P_E * cap + nb[k][P_W]] : ein[k][P_W];
        route_ranked(P, T, t, in, exists[k], sl + pout * 4 * cap + j, cap,
                     P.gtag + pout * pstride + (size_t)r[k] * 2, 2 * N, edge_out[k], ic);
        phase3<W1, W2>(P, T, t, sh_hist);
        if (t + 1 != tend) phase1<W1, W2>(P, T, t + 1, draining, sh_hist);
        tile_to_record(T, recs + j, cap);
      }
    // ---- publish: this warp has routed cycle t for all its tiles
    __syncwarp();
    if (lane == 0) st_release_cta_shared(&wflag[warp], t + 1);
  }

  // ---- end of launch: full link state of the last cycle, tile state, counters
  __syncthreads();
  {
    const uint32_t plast = (t - (t == tend ? 1u : 0u)) & 1u;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (act[k]) {
        const int j = i + k * nt;
#pragma unroll
        for (int d = 0; d < 4; ++d) P.glink[((size_t)plast * 4 + d) * N + r[k]] = sl[(plast * 4 + d) * cap + j];
        Tile T;
        tile_from_record(T, recs + j, cap);
        store_tile(P, T);
      }
  }
  __syncthreads();
  for (int k = i; k < 2 * HIST_BINS; k += nt)
    if (sh_hist[k]) atomicAdd(&P.hist[k], (unsigned long long)sh_hist[k]);
}

template <int W1, int W2, int POLV>
__global__ void __launch_bounds__(MULTI_THREADS, 1)
    run_multi_kernel(const __grid_constant__ Params P, const __grid_constant__ RunArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  run_rect_multi<W1, W2>(P, A, blockIdx.x, smem_raw);
}

template <int W1, int W2, int POLV>
static cudaError_t prepare_multi() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(run_multi_kernel<W1, W2, POLV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)multi_smem_bytes(MULTI_THREADS));
  if (e == cudaSuccess) done = true;
  return e;
}

template <int W1, int W2, int POLV>
static cudaError_t launch_multi_t(const Params& P, const RunArgs& A, cudaStream_t s) {
  cudaError_t e = prepare_multi<W1, W2, POLV>();
  if (e != cudaSuccess) return e;
  const int threads = multi_block_threads(P.W, P.H, A.gx, A.gy);
  void* args[] = {(void*)&P, (void*)&A};
  return cudaLaunchCooperativeKernel((const void*)run_multi_kernel<W1, W2, POLV>, dim3(A.gx * A.gy),
                                     dim3(threads), args, multi_smem_bytes(threads), s);
}

template <int W1, int W2, int POLV>
static cudaError_t max_coresident_multi_t(int threads, int* out) {
  cudaError_t e = prepare_multi<W1, W2, POLV>();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, run_multi_kernel<W1, W2, POLV>, threads,
                                                    multi_smem_bytes(threads));
  if (e != cudaSuccess) return e;
  *out = per * sms;
  return cudaSuccess;
}

}  // namespace noc
