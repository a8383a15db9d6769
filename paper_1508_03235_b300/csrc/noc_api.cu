// noc_api.cu -- host side of the C ABI declared in include/noc.h.
//
// A handle owns the host description of one simulation and one device arena
// (all state arrays, 256-byte aligned).  The arena is either caller memory
// bound with noc_bind_memory (e.g. a torch tensor) or taken with cudaMalloc on
// first use.  All device work is enqueued on the handle's stream.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "noc.h"
#include "noc_host.h"

using namespace noc;

namespace noc {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int configure(int mesh_w, int mesh_h, const noc_cache_cfg* c, int l2_policy, const noc_traffic* tr,
              uint64_t seed, Params& P) {
  if (!c || !tr) return fail(NOC_ERR_ARG, "null argument");
  if (mesh_w < 1 || mesh_h < 1 || (long)mesh_w * mesh_h > 65535)
    return fail(NOC_ERR_ARG, "mesh %dx%d: need 1..65535 tiles", mesh_w, mesh_h);
  if (l2_policy < 0 || l2_policy > 2) return fail(NOC_ERR_ARG, "l2_policy %d", l2_policy);
  if (c->l1_sets < 1 || c->l1_ways < 1 || c->l1_ways > MAX_WAYS || c->l2_sets < 1 || c->l2_ways < 1 ||
      c->l2_ways > MAX_WAYS)
    return fail(NOC_ERR_ARG, "cache geometry: sets >= 1, ways 1..16");
  if (c->l1_miss_cycles < 0 || c->mem_latency < 1) return fail(NOC_ERR_ARG, "latencies");
  if (c->core_q < 1 || c->svc_q < 1 || c->mem_q < 1 || c->core_q > 65535 || c->svc_q > 65535 ||
      c->mem_q > 65535)
    return fail(NOC_ERR_ARG, "queue capacities must be 1..65535");
  if (l2_policy == NOC_L2_LSPD_MIGRATE &&
      (c->mig_window < 1 || c->mig_window > HIST_MAX || c->mig_threshold < 1 ||
       c->fwd_entries < 1 || c->fwd_entries > 65535))
    return fail(NOC_ERR_ARG, "migration: window 1..30, threshold >= 1, forward entries >= 1");
  if (c->packet_mode < 0 || c->packet_mode > 1 ||
      (c->packet_mode && (c->rob_entries < 1 || c->rob_entries > 64 || c->svc_q < 16)))
    return fail(NOC_ERR_ARG, "packets: mode 0/1, reorder entries 1..64, svc_q >= 16");
  if (c->dir_central < 0 || c->dir_central > 1 ||
      (c->dir_central && (c->dir_tile < 0 || (long)c->dir_tile >= (long)mesh_w * mesh_h)))
    return fail(NOC_ERR_ARG, "directory node: dir_central 0/1, dir_tile a tile of the mesh");
  if (c->l1_write_back < 0 || c->l1_write_back > 1) return fail(NOC_ERR_ARG, "l1_write_back 0/1");
  if (c->age_mode < 0 || c->age_mode > 1) return fail(NOC_ERR_ARG, "age_mode 0/1");
  if (tr->mode < 0 || tr->mode > 2 || tr->period < 0) return fail(NOC_ERR_ARG, "traffic mode/period");
  if (tr->write_q16 > 65536 || tr->priv_q16 + (uint64_t)tr->shared_q16 > 65536 || tr->hot_q16 > 65536)
    return fail(NOC_ERR_ARG, "q16 fractions out of range");
  if (tr->mode == NOC_MODE_CACHE) {
    if (tr->priv_q16 > 0 && tr->priv_lines < 1) return fail(NOC_ERR_ARG, "priv_lines");
    if (tr->shared_q16 > 0 && tr->shared_lines < 1) return fail(NOC_ERR_ARG, "shared_lines");
    if (tr->priv_q16 + tr->shared_q16 < 65536 && tr->remote_lines < 1)
      return fail(NOC_ERR_ARG, "remote_lines");
  }
  if (tr->hot_side < 0 || tr->hot_side > mesh_w || tr->hot_side > mesh_h)
    return fail(NOC_ERR_ARG, "hot_side");
  const uint64_t N = (uint64_t)mesh_w * mesh_h;
  const uint64_t total = (uint64_t)tr->remote_lines + tr->shared_lines + (uint64_t)tr->priv_lines * N;
  if (total >= (1ull << 26)) return fail(NOC_ERR_ARG, "address space above 2^26 lines");

  memset(&P, 0, sizeof P);
  P.W = mesh_w;
  P.H = mesh_h;
  P.N = (int)N;
  P.policy = l2_policy;
  P.mode = tr->mode;
  P.period = tr->period;
  P.l1_sets = c->l1_sets;
  P.l1_ways = c->l1_ways;
  P.l2_sets = c->l2_sets;
  P.l2_ways = c->l2_ways;
  P.l1_miss = c->l1_miss_cycles;
  P.mem_lat = c->mem_latency;
  P.mig_window = c->mig_window;
  P.mig_threshold = c->mig_threshold;
  P.core_q = c->core_q;
  P.svc_q = c->svc_q;
  P.mem_q = c->mem_q;
  P.fwd_cap = c->fwd_entries > 0 ? c->fwd_entries : 1;
  P.packet_mode = c->packet_mode;
  P.rob_entries = c->packet_mode ? c->rob_entries : 0;
  P.dir_central = c->dir_central;
  P.dir_tile = c->dir_central ? c->dir_tile : 0;
  P.l1_write_back = c->l1_write_back;
  P.age_mode = c->age_mode;
  P.write_q16 = tr->write_q16;
  P.priv_q16 = tr->priv_q16;
  P.shared_q16 = tr->shared_q16;
  P.hot_q16 = tr->hot_q16;
  P.hot_side = tr->hot_side;
  P.hot_x0 = mesh_w / 2 - tr->hot_side / 2;
  P.hot_y0 = mesh_h / 2 - tr->hot_side / 2;
  P.priv_lines = tr->priv_lines;
  P.shared_lines = tr->shared_lines;
  P.remote_lines = tr->remote_lines;
  P.total_lines = (uint32_t)total;
  set_divisors(P);
  P.seed = seed;
  P.stream = tr->stream;
  return NOC_OK;
}

}  // namespace noc

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  return fail(NOC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr uint32_t kMaxChunk = 1u << 20;  // cycles per launch (32-bit counter deltas)
constexpr int kBatchRefcap = 256;          // references drawn ahead per tile of a batch instance

}  // namespace

struct noc_sim {
  Params P;
  noc_cache_cfg cache;
  noc_traffic traf;
  uint64_t seed;
  // arena layout (byte offsets)
  size_t o_rob, o_glink, o_gtag, o_core, o_cq, o_sq, o_mq, o_l1, o_l1own, o_l2, o_l2ep, o_l2hist, o_dir, o_fwd,
      o_stats, o_hist, o_flags, o_err, o_abort, o_scratch, o_refbuf, o_refk0, o_refcnt, bytes;
  int refcap = 512;              // references drawn ahead per tile (0 = draw in place)
  size_t n_flags;
  unsigned char* base = nullptr;
  bool owned = false;
  bool ready = false;
  cudaStream_t stream = nullptr;
  int gx = 0, gy = 0;          // requested tiling (0 = automatic)
  int run_gx = 0, run_gy = 0;  // tiling in use
  int tpt = 0;                 // requested tiles per thread (0 = automatic, 1, 2)
  int run_tpt = 0;             // tiles per thread in use (0 = not chosen yet)
  uint32_t cycle = 0;
  bool draining = false;       // set by noc_drain, cleared by noc_reset
  // tagged edge slots: all zero, or last written by a plain launch ending at
  // gtag_end (a plain launch starting anywhere else clears them first)
  bool gtag_clean = false;
  uint32_t gtag_end = 0;
  // hash trace
  bool hash_on = false;
  unsigned long long* d_hash = nullptr;
  size_t hash_cap = 0;
  int64_t hash_n = 0;
  // drain
  unsigned int* d_busy = nullptr;
  size_t busy_cap = 0;
  // trace mode
  std::vector<std::vector<uint32_t>> traces;
  bool trace_dirty = true;
  uint32_t* d_trace = nullptr;
  size_t trace_cap = 0;
  uint32_t* d_trace_off = nullptr;
  // debug knobs
  long long wait_ns = 2000000000ll;
  int silent_cta = -1;
  int thread_map = 0;     // tile-to-thread order inside a CTA rectangle
  int64_t launches = 0;
  int last_variant = -1;  // run_variant() of the last cycle-kernel launch
  int last_bound = 0;     // launch bound (most threads per CTA) of that launch's build
  // plain launches on the checked build (noc_set_checks)
  bool checks_on = false;
  // per-phase clock profile of the plain loop (noc_set_phase_profile)
  bool prof_on = false;
  unsigned long long* d_prof = nullptr;  // 6 words, device
  // cycle-kernel timing: event pairs [2k, 2k + 1] around launch k
  bool time_kernels = false;
  std::vector<cudaEvent_t> tev;
  size_t tev_used = 0;
};

namespace {

void layout(noc_sim* s) {
  const size_t N = (size_t)s->P.N;
  const Params& P = s->P;
  size_t cur = 0;
  auto take = [&](size_t b) {
    size_t o = align256(cur);
    cur = o + b;
    return o;
  };
  const size_t w1 = N * P.l1_sets * P.l1_ways, w2 = N * P.l2_sets * P.l2_ways;
  const bool lspd = P.policy != POL_INTERLEAVED, mig = P.policy == POL_MIGRATE;
  s->n_flags = FLAG_SLOTS * std::min<size_t>(N, 4096);
  s->o_glink = take(2 * 4 * N * sizeof(uint4));
  s->o_gtag = take(2 * 4 * N * 2 * sizeof(uint4));
  s->o_core = take(NCORE * N * sizeof(uint32_t));
  s->o_cq = take(N * P.core_q * sizeof(uint4));
  s->o_sq = take(N * P.svc_q * sizeof(uint4));
  s->o_mq = take(N * P.mem_q * sizeof(uint4));
  s->o_l1 = take(w1 * sizeof(uint32_t));
  s->o_l1own = take(w1 * sizeof(uint16_t));
  s->o_l2 = take(w2 * sizeof(uint32_t));
  s->o_l2ep = take(lspd ? w2 * sizeof(uint16_t) : 0);
  s->o_l2hist = take(mig ? w2 * hist_stride(P.mig_window) * sizeof(uint16_t) : 0);
  s->o_dir = take(lspd ? (size_t)P.total_lines * sizeof(uint32_t) : 0);
  s->o_fwd = take(mig ? N * P.fwd_cap * 2 * sizeof(uint32_t) : 0);
  s->o_rob = take(N * P.rob_entries * 2 * sizeof(uint32_t));
  s->o_stats = take((size_t)NSTAT * N * sizeof(unsigned long long));
  s->o_hist = take(2 * HIST_BINS * sizeof(unsigned long long));
  s->o_flags = take(s->n_flags * sizeof(unsigned int));
  s->o_err = take(sizeof(unsigned long long));
  s->o_abort = take(sizeof(unsigned int));
  s->o_scratch = take(64 * sizeof(unsigned long long));
  s->o_refbuf = take(N * (size_t)s->refcap * sizeof(uint32_t));
  s->o_refk0 = take(s->refcap ? N * sizeof(uint32_t) : 0);
  s->o_refcnt = take(s->refcap ? N * sizeof(uint32_t) : 0);
  s->bytes = align256(cur);
}

void set_pointers(noc_sim* s) {
  Params& P = s->P;
  unsigned char* b = s->base;
  const bool lspd = P.policy != POL_INTERLEAVED, mig = P.policy == POL_MIGRATE;
  P.glink = reinterpret_cast<uint4*>(b + s->o_glink);
  P.gtag = reinterpret_cast<uint4*>(b + s->o_gtag);
  P.core = reinterpret_cast<uint32_t*>(b + s->o_core);
  P.cq = reinterpret_cast<uint4*>(b + s->o_cq);
  P.sq = reinterpret_cast<uint4*>(b + s->o_sq);
  P.mq = reinterpret_cast<uint4*>(b + s->o_mq);
  P.l1 = reinterpret_cast<uint32_t*>(b + s->o_l1);
  P.l1own = reinterpret_cast<uint16_t*>(b + s->o_l1own);
  P.l2 = reinterpret_cast<uint32_t*>(b + s->o_l2);
  P.l2ep = lspd ? reinterpret_cast<uint16_t*>(b + s->o_l2ep) : nullptr;
  P.l2hist = mig ? reinterpret_cast<uint16_t*>(b + s->o_l2hist) : nullptr;
  P.dir = lspd ? reinterpret_cast<uint32_t*>(b + s->o_dir) : nullptr;
  P.fwd = mig ? reinterpret_cast<uint32_t*>(b + s->o_fwd) : nullptr;
  P.rob = P.rob_entries ? reinterpret_cast<uint32_t*>(b + s->o_rob) : nullptr;
  P.stats = reinterpret_cast<unsigned long long*>(b + s->o_stats);
  P.hist = reinterpret_cast<unsigned long long*>(b + s->o_hist);
  P.flags = reinterpret_cast<unsigned int*>(b + s->o_flags);
  P.err = reinterpret_cast<unsigned long long*>(b + s->o_err);
  P.refcap = s->refcap;
  P.refbuf = s->refcap ? reinterpret_cast<uint32_t*>(b + s->o_refbuf) : nullptr;
  P.refk0 = s->refcap ? reinterpret_cast<uint32_t*>(b + s->o_refk0) : nullptr;
  P.refcnt = s->refcap ? reinterpret_cast<uint32_t*>(b + s->o_refcnt) : nullptr;
}

unsigned int* abort_ptr(noc_sim* s) { return reinterpret_cast<unsigned int*>(s->base + s->o_abort); }
unsigned long long* scratch_ptr(noc_sim* s) {
  return reinterpret_cast<unsigned long long*>(s->base + s->o_scratch);
}

int do_reset(noc_sim* s) {
  Params& P = s->P;
  cudaStream_t st = s->stream;
  const size_t N = (size_t)P.N;
  const size_t w1 = N * P.l1_sets * P.l1_ways, w2 = N * P.l2_sets * P.l2_ways;
  CU(cudaMemsetAsync(P.glink, 0, 2 * 4 * N * sizeof(uint4), st), "reset links");
  CU(cudaMemsetAsync(P.gtag, 0, 2 * 4 * N * 2 * sizeof(uint4), st), "reset edge slots");
  s->gtag_clean = true;
  CU(cudaMemsetAsync(P.core, 0, NCORE * N * sizeof(uint32_t), st), "reset cores");
  CU(cudaMemsetAsync(P.l1, 0, w1 * sizeof(uint32_t), st), "reset L1");
  CU(cudaMemsetAsync(P.l1own, 0, w1 * sizeof(uint16_t), st), "reset L1 owners");
  CU(cudaMemsetAsync(P.l2, 0, w2 * sizeof(uint32_t), st), "reset L2");
  if (P.l2ep) CU(cudaMemsetAsync(P.l2ep, 0, w2 * sizeof(uint16_t), st), "reset L2 epochs");
  if (P.l2hist)
    CU(cudaMemsetAsync(P.l2hist, 0, w2 * hist_stride(P.mig_window) * sizeof(uint16_t), st), "reset history");
  if (P.dir) CU(cudaMemsetAsync(P.dir, 0xFF, (size_t)P.total_lines * 4, st), "reset directory");
  if (P.fwd) CU(cudaMemsetAsync(P.fwd, 0, N * P.fwd_cap * 8, st), "reset forward tables");
  if (P.rob) CU(cudaMemsetAsync(P.rob, 0, N * P.rob_entries * 8, st), "reset reorder buffers");
  CU(cudaMemsetAsync(P.stats, 0, (size_t)NSTAT * N * 8, st), "reset counters");
  CU(cudaMemsetAsync(P.hist, 0, 2 * HIST_BINS * 8, st), "reset histograms");
  CU(cudaMemsetAsync(P.flags, 0, s->n_flags * 4, st), "reset flags");
  CU(cudaMemsetAsync(P.err, 0xFF, 8, st), "reset error word");
  CU(cudaMemsetAsync(abort_ptr(s), 0, 4, st), "reset abort flag");
  if (P.refcnt) CU(cudaMemsetAsync(P.refcnt, 0, N * 4, st), "reset reference window");
  s->cycle = 0;
  s->hash_n = 0;
  s->draining = false;
  return NOC_OK;
}

int ensure_memory(noc_sim* s) {
  if (s->ready) return NOC_OK;
  if (!s->base) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, s->bytes);
    if (e != cudaSuccess) return fail(NOC_ERR_OOM, "cudaMalloc(%zu): %s", s->bytes, cudaGetErrorString(e));
    s->base = static_cast<unsigned char*>(p);
    s->owned = true;
  }
  set_pointers(s);
  int rc = do_reset(s);
  if (rc) return rc;
  s->ready = true;
  return NOC_OK;
}

// threads per CTA and co-resident CTAs of a launch with `tpt` tiles per thread
int launch_threads(const noc_sim* s, int tpt, int gx, int gy) {
  return tpt == 2 ? multi_threads(s->P.W, s->P.H, gx, gy) : block_threads(s->P.W, s->P.H, gx, gy);
}
int max_launch_threads(int tpt) { return tpt == 2 ? MULTI_MAX_THREADS : RUN_MAX_THREADS; }
cudaError_t coresident(const noc_sim* s, int tpt, int threads, int* cap) {
  return tpt == 2 ? max_coresident_multi(s->P, threads, cap) : max_coresident_ctas(s->P, threads, cap);
}

// choose the CTA rectangle grid for `tpt` tiles per thread: the fewest CTAs
// whose rectangles hold at most 128 tiles, else the smallest rectangles that
// still fit co-resident; NOC_ERR_ARG (without a message) if none does
int choose_tiling_tpt(noc_sim* s, int tpt, int* gx_out, int* gy_out) {
  const int W = s->P.W, H = s->P.H;
  int cap_of[RUN_MAX_THREADS / 32 + 1];
  for (int k = 0; k <= RUN_MAX_THREADS / 32; ++k) cap_of[k] = -1;
  int best_gx = 0, best_gy = 0;
  long best_g = 0, best_a = 0, best_p = 0;
  bool best_small = false;
  for (int gy = 1; gy <= H; ++gy)
    for (int gx = 1; gx <= W; ++gx) {
      const int threads = launch_threads(s, tpt, gx, gy);
      if (threads > max_launch_threads(tpt)) continue;
      const long G = (long)gx * gy;
      if (G * FLAG_SLOTS > (long)s->n_flags) continue;
      int& cap = cap_of[threads / 32];
      if (cap < 0) {
        cudaError_t e = coresident(s, tpt, threads, &cap);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy");
      }
      if (G > cap) continue;
      const long bw = (W + gx - 1) / gx, bh = (H + gy - 1) / gy, a = bw * bh, per = bw + bh;
      const bool small = a <= 128;
      bool better;
      if (!best_gx) better = true;
      else if (small != best_small) better = small;
      else if (small) better = G < best_g || (G == best_g && (a < best_a || (a == best_a && per < best_p)));
      else better = a < best_a || (a == best_a && (G < best_g || (G == best_g && per < best_p)));
      if (better) {
        best_gx = gx;
        best_gy = gy;
        best_g = G;
        best_a = a;
        best_p = per;
        best_small = small;
      }
    }
  if (!best_gx) return NOC_ERR_ARG;
  *gx_out = best_gx;
  *gy_out = best_gy;
  return NOC_OK;
}

// tiles per thread and CTA rectangle grid of the plain loop: the requested
// ones, else one tile per thread if the mesh fits one co-resident launch that
// way, else two
int choose_layout(noc_sim* s) {
  const int W = s->P.W, H = s->P.H;
  const int tries[2] = {s->tpt ? s->tpt : 1, s->tpt ? 0 : 2};
  for (int tpt : tries) {
    if (!tpt) break;
    int gx = s->gx, gy = s->gy;
    if (gx > 0 && gy > 0) {
      // the requested tiling, if it fits one co-resident launch this way
      const int threads = launch_threads(s, tpt, gx, gy);
      int cap = 0;
      if (threads <= max_launch_threads(tpt)) CU(coresident(s, tpt, threads, &cap), "occupancy");
      if (threads > max_launch_threads(tpt) || gx * gy > cap || gx * gy * FLAG_SLOTS > (int)s->n_flags)
        continue;
    } else {
      int rc = choose_tiling_tpt(s, tpt, &gx, &gy);
      if (rc == NOC_ERR_CUDA) return rc;
      if (rc) continue;
    }
    s->run_tpt = tpt;
    s->run_gx = gx;
    s->run_gy = gy;
    return NOC_OK;
  }
  return fail(NOC_ERR_ARG, "mesh %dx%d does not fit one co-resident launch", W, H);
}

int upload_traces(noc_sim* s) {
  if (s->P.mode != MODE_TRACE || !s->trace_dirty) return NOC_OK;
  const size_t N = (size_t)s->P.N;
  std::vector<uint32_t> off(N + 1, 0), all;
  for (size_t r = 0; r < N; ++r) {
    off[r] = (uint32_t)all.size();
    if (r < s->traces.size()) all.insert(all.end(), s->traces[r].begin(), s->traces[r].end());
  }
  off[N] = (uint32_t)all.size();
  if (!s->d_trace_off) CU(cudaMalloc(&s->d_trace_off, (N + 1) * 4), "trace offsets");
  if (all.size() > s->trace_cap || !s->d_trace) {
    if (s->d_trace) cudaFree(s->d_trace);
    s->trace_cap = all.size() ? all.size() : 1;
    CU(cudaMalloc(&s->d_trace, s->trace_cap * 4), "trace buffer");
  }
  CU(cudaMemcpyAsync(s->d_trace_off, off.data(), (N + 1) * 4, cudaMemcpyHostToDevice, s->stream),
     "trace offsets copy");
  if (!all.empty())
    CU(cudaMemcpyAsync(s->d_trace, all.data(), all.size() * 4, cudaMemcpyHostToDevice, s->stream),
       "trace copy");
  CU(cudaStreamSynchronize(s->stream), "trace upload");
  s->P.trace_off = s->d_trace_off;
  s->P.trace = s->d_trace;
  s->trace_dirty = false;
  return NOC_OK;
}

int read_error(noc_sim* s, int64_t* cyc) {
  unsigned long long e = ~0ull;
  CU(cudaMemcpyAsync(&e, s->P.err, 8, cudaMemcpyDeviceToHost, s->stream), "error word");
  CU(cudaStreamSynchronize(s->stream), "sync");
  if (cyc) *cyc = e == ~0ull ? -1 : (int64_t)(e >> 8);
  if (e == ~0ull) return NOC_OK;
  int code = (int)(e & 0xFF);
  return fail(code, "simulation error %d at cycle %lld", code, (long long)(e >> 8));
}

// run n cycles as one or more cooperative launches
int run_cycles(noc_sim* s, uint32_t n, bool draining, unsigned int* busy) {
  int rc = upload_traces(s);
  if (rc) return rc;
  if (!s->run_gx || !s->run_tpt) {
    rc = choose_layout(s);
    if (rc) return rc;
  }
  const int tpt = s->run_tpt;
  if (tpt == 2 && (busy || s->hash_on))
    return fail(NOC_ERR_ARG, "per-cycle hashes and drains need one tile per thread (a mesh of one "
                             "co-resident launch); this one runs two");
  if (s->checks_on && (tpt == 2 || busy || s->hash_on))
    return fail(NOC_ERR_ARG, "the checked build is the plain loop with one tile per thread: no per-cycle "
                             "hashes, drains or two tiles per thread while checks are on");
  const int threads = launch_threads(s, tpt, s->run_gx, s->run_gy);
  int cap = 0;
  CU(coresident(s, tpt, threads, &cap), "occupancy");
  if (s->checks_on) {
    int ccap = 0;
    CU(max_coresident_checked(s->P, threads, &ccap), "occupancy");
    cap = std::min(cap, ccap);
  }
  if (threads > max_launch_threads(tpt) || s->run_gx * s->run_gy > cap ||
      s->run_gx * s->run_gy * FLAG_SLOTS > (int)s->n_flags)
    return fail(NOC_ERR_ARG, "tiling %dx%d does not fit one co-resident launch with %d tile(s) per thread",
                s->run_gx, s->run_gy, tpt);
  // with references drawn ahead, a launch covers at most refcap references of
  // an on-schedule core
  uint32_t chunk_max = kMaxChunk;
  const bool ahead = s->P.refbuf && s->P.period > 0 && s->P.mode != MODE_TRACE;
  if (ahead) chunk_max = std::min<uint64_t>(kMaxChunk, (uint64_t)s->P.refcap * s->P.period);
  uint32_t done = 0;
  while (done < n) {
    uint32_t c = n - done < chunk_max ? n - done : chunk_max;
    if (ahead) {
      CU(launch_gen_refs(s->P, s->cycle, c, s->stream), "reference draw launch");
      s->launches++;
    }
    RunArgs A;
    A.t0 = s->cycle;
    A.n = c;
    A.draining = draining ? 1 : 0;
    A.gx = s->run_gx;
    A.gy = s->run_gy;
    A.hash_trace = (s->hash_on && !busy) ? s->d_hash + done : nullptr;
    A.busy = busy ? busy + done : nullptr;
    A.abort_flag = abort_ptr(s);
    A.wait_ns = s->wait_ns;
    A.silent_cta = s->silent_cta;
    A.thread_map = s->thread_map;
    A.checked = s->checks_on ? 1 : 0;
    A.prof = (s->prof_on && !s->checks_on && !A.hash_trace && !A.busy && tpt == 1) ? s->d_prof : nullptr;
    if (A.prof) {
      // the profiled build keeps its own register count: check it fits too
      if (threads > RUN_PROF_THREADS)
        return fail(NOC_ERR_ARG, "the profiled loop takes CTAs of at most %d threads (tiling %dx%d has %d)",
                    RUN_PROF_THREADS, s->run_gx, s->run_gy, threads);
      int pcap = 0;
      CU(max_coresident_prof(s->P, threads, &pcap), "occupancy");
      if (s->run_gx * s->run_gy > pcap)
        return fail(NOC_ERR_ARG, "tiling %dx%d does not fit one co-resident launch of the profiled loop",
                    s->run_gx, s->run_gy);
    }
    const bool plain = !A.hash_trace && !A.busy;
    if (plain && !s->gtag_clean && s->gtag_end != s->cycle) {
      CU(cudaMemsetAsync(s->P.gtag, 0, 2 * 4 * (size_t)s->P.N * 2 * sizeof(uint4), s->stream),
         "clear edge slots");
      s->gtag_clean = true;
    }
    if (s->time_kernels) {
      while (s->tev.size() < s->tev_used + 2) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e), "event create");
        s->tev.push_back(e);
      }
      CU(cudaEventRecord(s->tev[s->tev_used], s->stream), "event record");
    }
    if (tpt == 2) {
      CU(launch_multi(s->P, A, s->stream), "cycle kernel launch");
      s->last_variant = multi_variant(s->P);
      s->last_bound = MULTI_MAX_THREADS;
    } else {
      CU(launch_run(s->P, A, s->stream), "cycle kernel launch");
      s->last_variant = run_variant(s->P, A);
      s->last_bound = run_launch_bound(s->P, A);
    }
    s->launches++;
    if (s->time_kernels) {
      CU(cudaEventRecord(s->tev[s->tev_used + 1], s->stream), "event record");
      s->tev_used += 2;
    }
    if (plain) {
      s->gtag_clean = false;
      s->gtag_end = s->cycle + c;
    }
    s->cycle += c;
    done += c;
  }
  return NOC_OK;
}

// a host flit of 8 words (type, src, dst, inject, line, a, e, age) in the
// device layout; under age_mode 1 the age goes above the inject cycle
uint4 pack_flit(const Params& P, const uint32_t* f8, uint32_t src) {
  const uint32_t x = P.age_mode ? (f8[3] & (AGE_ONE - 1u)) | (f8[7] << AGE_SHIFT) : f8[3];
  return make_uint4(x, (src & 0xFFFFu) | (f8[2] << 16), (f8[4] & W_LINE) | (f8[0] << 26),
                    (f8[5] & 0xFFFFu) | (f8[6] << 16));
}

}  // namespace

// ============================================================== C ABI
extern "C" {

const char* noc_last_error(void) { return g_last_error.c_str(); }

int noc_create(int mesh_w, int mesh_h, const noc_cache_cfg* c, int l2_policy, const noc_traffic* tr,
               uint64_t seed, noc_sim** out) {
  if (!c || !tr || !out) return fail(NOC_ERR_ARG, "null argument");
  *out = nullptr;
  Params P;
  int rc = configure(mesh_w, mesh_h, c, l2_policy, tr, seed, P);
  if (rc) return rc;
  noc_sim* s = new (std::nothrow) noc_sim();
  if (!s) return fail(NOC_ERR_OOM, "host allocation");
  s->cache = *c;
  s->traf = *tr;
  s->seed = seed;
  s->P = P;
  s->traces.resize((size_t)P.N);
  layout(s);
  *out = s;
  return NOC_OK;
}

void noc_destroy(noc_sim* s) {
  if (!s) return;
  if (s->base && s->owned) cudaFree(s->base);
  if (s->d_hash) cudaFree(s->d_hash);
  if (s->d_busy) cudaFree(s->d_busy);
  if (s->d_trace) cudaFree(s->d_trace);
  if (s->d_trace_off) cudaFree(s->d_trace_off);
  if (s->d_prof) cudaFree(s->d_prof);
  for (cudaEvent_t e : s->tev) cudaEventDestroy(e);
  delete s;
}

size_t noc_required_bytes(const noc_sim* s) { return s ? s->bytes : 0; }

int noc_bind_memory(noc_sim* s, void* p, size_t bytes) {
  if (!s || !p) return fail(NOC_ERR_ARG, "null argument");
  if (s->base) return fail(NOC_ERR_STATE, "memory already bound or allocated");
  if (bytes < s->bytes) return fail(NOC_ERR_ARG, "need %zu bytes, got %zu", s->bytes, bytes);
  if (reinterpret_cast<uintptr_t>(p) & 255) return fail(NOC_ERR_ARG, "memory must be 256-byte aligned");
  s->base = static_cast<unsigned char*>(p);
  s->owned = false;
  return NOC_OK;
}

int noc_set_stream(noc_sim* s, void* stream) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  s->stream = static_cast<cudaStream_t>(stream);
  return NOC_OK;
}

int noc_reset(noc_sim* s) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (!s->ready) return ensure_memory(s);
  return do_reset(s);
}

int noc_step(noc_sim* s, int64_t n) {
  if (!s || n < 0) return fail(NOC_ERR_ARG, "bad argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  if (n == 0) return NOC_OK;
  if ((uint64_t)s->cycle + (uint64_t)n >= (1ull << 32) - 2) return fail(NOC_ERR_ARG, "cycle count above 2^32");
  if (s->P.age_mode && (uint64_t)s->cycle + (uint64_t)n > (1ull << AGE_SHIFT))
    return fail(NOC_ERR_ARG, "age_mode 1 runs end at or before cycle 2^20");
  if (s->hash_on) {
    if ((size_t)n > s->hash_cap) {
      if (s->d_hash) cudaFree(s->d_hash);
      s->d_hash = nullptr;
      CU(cudaMalloc(&s->d_hash, (size_t)n * 8), "hash trace buffer");
      s->hash_cap = (size_t)n;
    }
    CU(cudaMemsetAsync(s->d_hash, 0, (size_t)n * 8, s->stream), "hash trace clear");
    s->hash_n = n;
  }
  return run_cycles(s, (uint32_t)n, s->draining, nullptr);
}

// ---- checkpoint image: header, then the device arena byte for byte
namespace {
constexpr uint64_t kImageMagic = 0x314B504E4F434E42ull;  // "BNCONPK1"
struct ImageHeader {
  uint64_t magic;
  uint64_t arena_bytes;
  uint64_t seed;
  int32_t mesh_w, mesh_h, policy, draining;
  uint32_t cycle, reserved;
  noc_cache_cfg cache;
  noc_traffic traffic;
};
}  // namespace

size_t noc_checkpoint_bytes(const noc_sim* s) { return s ? sizeof(ImageHeader) + s->bytes : 0; }

int noc_save(noc_sim* s, void* buf, size_t bytes) {
  if (!s || !buf) return fail(NOC_ERR_ARG, "null argument");
  if (bytes < noc_checkpoint_bytes(s))
    return fail(NOC_ERR_ARG, "checkpoint needs %zu bytes, got %zu", noc_checkpoint_bytes(s), bytes);
  int rc = ensure_memory(s);
  if (rc) return rc;
  rc = noc_sync(s, nullptr);
  if (rc) return rc;
  ImageHeader h;
  memset(&h, 0, sizeof h);
  h.magic = kImageMagic;
  h.arena_bytes = s->bytes;
  h.seed = s->seed;
  h.mesh_w = s->P.W;
  h.mesh_h = s->P.H;
  h.policy = s->P.policy;
  h.draining = s->draining ? 1 : 0;
  h.cycle = s->cycle;
  h.cache = s->cache;
  h.traffic = s->traf;
  memcpy(buf, &h, sizeof h);
  CU(cudaMemcpy(static_cast<unsigned char*>(buf) + sizeof h, s->base, s->bytes, cudaMemcpyDeviceToHost),
     "checkpoint copy");
  return NOC_OK;
}

int noc_load(noc_sim* s, const void* buf, size_t bytes) {
  if (!s || !buf) return fail(NOC_ERR_ARG, "null argument");
  ImageHeader h;
  if (bytes < sizeof h) return fail(NOC_ERR_ARG, "not a checkpoint image");
  memcpy(&h, buf, sizeof h);
  if (h.magic != kImageMagic) return fail(NOC_ERR_ARG, "not a checkpoint image");
  if (h.arena_bytes != s->bytes || bytes < sizeof h + h.arena_bytes || h.seed != s->seed ||
      h.mesh_w != s->P.W || h.mesh_h != s->P.H || h.policy != s->P.policy ||
      memcmp(&h.cache, &s->cache, sizeof h.cache) != 0 || memcmp(&h.traffic, &s->traf, sizeof h.traffic) != 0)
    return fail(NOC_ERR_ARG, "checkpoint of a different configuration");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  CU(cudaMemcpy(s->base, static_cast<const unsigned char*>(buf) + sizeof h, s->bytes, cudaMemcpyHostToDevice),
     "checkpoint copy");
  s->cycle = h.cycle;
  s->draining = h.draining != 0;
  s->hash_n = 0;
  // the edge slots in the image belong to whatever ran before the save: the
  // next plain launch clears them (its first cycle reads the complete links)
  s->gtag_clean = false;
  s->gtag_end = h.cycle + 1u;
  return NOC_OK;
}

int noc_sync(noc_sim* s, int64_t* err_cycle) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (err_cycle) *err_cycle = -1;
  if (!s->ready) return NOC_OK;
  CU(cudaStreamSynchronize(s->stream), "stream synchronize");
  return read_error(s, err_cycle);
}

int noc_drain(noc_sim* s, int64_t max_cycles, int64_t* taken) {
  if (!s || max_cycles < 0) return fail(NOC_ERR_ARG, "bad argument");
  if (taken) *taken = 0;
  int rc = ensure_memory(s);
  if (rc) return rc;
  rc = noc_sync(s, nullptr);
  if (rc) return rc;
  if (s->P.age_mode && (uint64_t)s->cycle + (uint64_t)max_cycles > (1ull << AGE_SHIFT))
    return fail(NOC_ERR_ARG, "age_mode 1 runs end at or before cycle 2^20");
  if (!s->run_gx || !s->run_tpt) {
    rc = choose_layout(s);
    if (rc) return rc;
  }
  if (s->run_tpt == 2)
    return fail(NOC_ERR_ARG, "a drain needs one tile per thread (a mesh of one co-resident launch)");
  s->draining = true;
  unsigned int busy0 = 0;
  unsigned int* d_b0 = reinterpret_cast<unsigned int*>(scratch_ptr(s));
  CU(cudaMemsetAsync(d_b0, 0, 4, s->stream), "busy clear");
  CU(launch_count_busy(s->P, s->cycle, d_b0, s->stream), "busy count");
  CU(cudaMemcpyAsync(&busy0, d_b0, 4, cudaMemcpyDeviceToHost, s->stream), "busy copy");
  CU(cudaStreamSynchronize(s->stream), "sync");
  if (busy0 == 0) return NOC_OK;
  const uint32_t chunk_max = 4096;
  if (s->busy_cap < chunk_max) {
    if (s->d_busy) cudaFree(s->d_busy);
    s->d_busy = nullptr;
    CU(cudaMalloc(&s->d_busy, chunk_max * 4), "busy buffer");
    s->busy_cap = chunk_max;
  }
  std::vector<unsigned int> hb(chunk_max);
  int64_t left = max_cycles, run = 0;
  uint32_t chunk = 64;
  while (left > 0) {
    uint32_t c = (int64_t)chunk < left ? chunk : (uint32_t)left;
    const uint32_t before = s->cycle;
    CU(cudaMemsetAsync(s->d_busy, 0, c * 4, s->stream), "busy clear");
    rc = run_cycles(s, c, true, s->d_busy);
    if (rc) return rc;
    CU(cudaMemcpyAsync(hb.data(), s->d_busy, c * 4, cudaMemcpyDeviceToHost, s->stream), "busy copy");
    rc = read_error(s, nullptr);
    if (rc) return rc;
    for (uint32_t j = 0; j < c; ++j)
      if (hb[j] == 0) {
        // quiet after cycle before+j: the state is a fixed point from there on,
        // so the extra cycles changed nothing but the cycle number
        s->cycle = before + j + 1;
        CU(cudaMemsetAsync(s->P.glink, 0, 2 * 4 * (size_t)s->P.N * sizeof(uint4), s->stream),
           "links clear");
        CU(launch_fill_u32(s->P.flags, s->cycle, s->n_flags, s->stream), "flags rewind");
        CU(cudaStreamSynchronize(s->stream), "sync");
        if (taken) *taken = run + j + 1;
        return NOC_OK;
      }
    run += c;
    left -= c;
    if (chunk < chunk_max) chunk *= 2;
  }
  if (taken) *taken = run;
  return fail(NOC_ERR_TIMEOUT, "not quiescent after %lld cycles", (long long)max_cycles);
}

int noc_stats(noc_sim* s, int tile, noc_stats_t* out) {
  if (!s || !out || tile >= s->P.N) return fail(NOC_ERR_ARG, "bad argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  unsigned long long h[NSTAT];
  CU(launch_reduce_stats(s->P, tile, scratch_ptr(s), s->stream), "stats reduce");
  CU(cudaMemcpyAsync(h, scratch_ptr(s), sizeof h, cudaMemcpyDeviceToHost, s->stream), "stats copy");
  CU(cudaStreamSynchronize(s->stream), "sync");
  out->cycle = s->cycle;
  out->injected = h[S_INJ];
  out->ejected = h[S_EJ];
  out->in_flight = h[S_INJ] - h[S_EJ];
  out->deflections = h[S_DEFL];
  out->lat_sum = h[S_LATSUM];
  out->lat_max = h[S_LATMAX];
  out->refs = h[S_REFS];
  out->l1_hit = h[S_L1H];
  out->l1_miss = h[S_L1M];
  out->l2_hit = h[S_L2H];
  out->l2_miss = h[S_L2M];
  out->req_made = h[S_REQM];
  out->req_rcvd = h[S_REQR];
  out->reply_sent = h[S_REPS];
  out->reply_rcvd = h[S_REPR];
  out->dir_search = h[S_DIRS];
  out->mem_req = h[S_MEMREQ];
  out->mem_write = h[S_MEMW];
  out->mem_wb = h[S_MEMWB];
  out->wt_sent = h[S_WTS];
  out->wt_hit = h[S_WTH];
  out->trap = h[S_TRAP];
  out->redir = h[S_REDIR];
  out->migrations = h[S_MIGR];
  out->l2lat_sum = h[S_L2LSUM];
  out->l2lat_cnt = h[S_L2LCNT];
  out->cq_stall = h[S_CQST];
  out->mm_stall = h[S_MMST];
  out->mig_sent = h[S_MIGS];
  return NOC_OK;
}

int noc_latency_hist(noc_sim* s, int which, uint64_t* bins, int nbins) {
  if (!s || !bins || which < 0 || which > 1 || nbins < HIST_BINS) return fail(NOC_ERR_ARG, "bad argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaMemcpyAsync(bins, s->P.hist + which * HIST_BINS, HIST_BINS * 8, cudaMemcpyDeviceToHost,
                     s->stream),
     "histogram copy");
  CU(cudaStreamSynchronize(s->stream), "sync");
  return NOC_OK;
}

static int hash_common(noc_sim* s, uint64_t* out, bool full) {
  if (!s || !out) return fail(NOC_ERR_ARG, "null argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  unsigned long long* d = scratch_ptr(s) + 48;
  CU(cudaMemsetAsync(d, 0, 8, s->stream), "hash clear");
  if (full) CU(launch_state_hash(s->P, s->cycle, d, s->stream), "state hash");
  else CU(launch_dyn_hash(s->P, s->cycle, d, s->stream), "dynamic hash");
  s->launches += full ? 2 : 1;
  CU(cudaMemcpyAsync(out, d, 8, cudaMemcpyDeviceToHost, s->stream), "hash copy");
  CU(cudaStreamSynchronize(s->stream), "sync");
  return NOC_OK;
}

int noc_dyn_hash(noc_sim* s, uint64_t* out) { return hash_common(s, out, false); }
int noc_state_hash(noc_sim* s, uint64_t* out) { return hash_common(s, out, true); }

int noc_set_hash_trace(noc_sim* s, int enable) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  s->hash_on = enable != 0;
  return NOC_OK;
}

int noc_hash_trace(noc_sim* s, uint64_t* buf, int64_t n) {
  if (!s || !buf || n < 0) return fail(NOC_ERR_ARG, "bad argument");
  if (n > s->hash_n) return fail(NOC_ERR_ARG, "only %lld cycles recorded", (long long)s->hash_n);
  if (n == 0) return NOC_OK;
  CU(cudaMemcpyAsync(buf, s->d_hash, (size_t)n * 8, cudaMemcpyDeviceToHost, s->stream), "trace copy");
  CU(cudaStreamSynchronize(s->stream), "sync");
  return NOC_OK;
}

int noc_set_thread_map(noc_sim* s, int map) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (map < 0 || map > 2) return fail(NOC_ERR_ARG, "thread map 0 (perimeter first), 1 (rows) or 2 (columns)");
  s->thread_map = map;
  return NOC_OK;
}

int noc_get_thread_map(const noc_sim* s) { return s ? s->thread_map : -1; }

int noc_set_tiling(noc_sim* s, int gx, int gy) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (gx == 0 && gy == 0) {
    s->gx = s->gy = 0;
    s->run_gx = s->run_gy = 0;
    s->run_tpt = 0;
    return NOC_OK;
  }
  if (gx < 1 || gy < 1 || gx > s->P.W || gy > s->P.H || block_threads(s->P.W, s->P.H, gx, gy) > 512 ||
      (long)gx * gy * FLAG_SLOTS > (long)s->n_flags)
    return fail(NOC_ERR_ARG, "tiling %dx%d invalid for mesh %dx%d", gx, gy, s->P.W, s->P.H);
  s->gx = s->run_gx = gx;
  s->gy = s->run_gy = gy;
  s->run_tpt = 0;  // chosen again (with this tiling) at the next launch
  return NOC_OK;
}

int noc_set_tiles_per_thread(noc_sim* s, int k) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (k < 0 || k > 2) return fail(NOC_ERR_ARG, "tiles per thread 0 (automatic), 1 or 2");
  s->tpt = k;
  s->run_tpt = 0;
  return NOC_OK;
}

int noc_get_tiles_per_thread(const noc_sim* s) { return s ? s->run_tpt : -1; }

int noc_get_tiling(const noc_sim* s, int* gx, int* gy) {
  if (!s || !gx || !gy) return fail(NOC_ERR_ARG, "null argument");
  *gx = s->run_gx;
  *gy = s->run_gy;
  return NOC_OK;
}

int noc_set_trace(noc_sim* s, int core, int64_t n, const uint32_t* refs) {
  if (!s || core < 0 || core >= s->P.N || n < 0 || (n > 0 && !refs)) return fail(NOC_ERR_ARG, "bad argument");
  for (int64_t k = 0; k < n; ++k)
    if ((refs[k] & 0x7FFFFFFFu) >= s->P.total_lines) return fail(NOC_ERR_ARG, "trace line out of range");
  s->traces[core].assign(refs, refs + n);
  s->trace_dirty = true;
  return NOC_OK;
}

int noc_debug_enqueue(noc_sim* s, int tile, int queue, const uint32_t* f8) {
  if (!s || !f8 || tile < 0 || tile >= s->P.N || queue < 0 || queue > 1) return fail(NOC_ERR_ARG, "bad argument");
  if (f8[0] == 0 || f8[0] > T_PROBE || f8[2] >= (uint32_t)s->P.N || f8[2] == (uint32_t)tile)
    return fail(NOC_ERR_ARG, "bad flit");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  const size_t N = (size_t)s->P.N;
  uint32_t* fld = s->P.core + (queue == 0 ? C_CQ : C_SQ) * N + tile;
  uint32_t q;
  CU(cudaMemcpy(&q, fld, 4, cudaMemcpyDeviceToHost), "queue read");
  const uint32_t cap = queue == 0 ? s->P.core_q : s->P.svc_q, head = q & 0xFFFFu, len = q >> 16;
  if (len >= cap) return fail(NOC_ERR_QUEUE_OVERFLOW, "queue full");
  uint4 f = pack_flit(s->P, f8, (uint32_t)tile);
  f.x = 0;
  uint4* buf = (queue == 0 ? s->P.cq : s->P.sq) + (size_t)tile * cap + (head + len) % cap;
  CU(cudaMemcpy(buf, &f, sizeof f, cudaMemcpyHostToDevice), "queue write");
  q = head | ((len + 1) << 16);
  CU(cudaMemcpy(fld, &q, 4, cudaMemcpyHostToDevice), "queue update");
  return NOC_OK;
}

int noc_debug_link(noc_sim* s, int tile, int dir, const uint32_t* f8) {
  if (!s || !f8 || tile < 0 || tile >= s->P.N || dir < 0 || dir > 3) return fail(NOC_ERR_ARG, "bad argument");
  const int W = s->P.W, H = s->P.H, x = tile % W, y = tile / W;
  int nb = -1;
  if (dir == P_N && y > 0) nb = tile - W;
  if (dir == P_S && y < H - 1) nb = tile + W;
  if (dir == P_E && x < W - 1) nb = tile + 1;
  if (dir == P_W && x > 0) nb = tile - 1;
  if (nb < 0) return fail(NOC_ERR_ARG, "no neighbour in that direction");
  if (f8[0] == 0 || f8[0] > T_PROBE || f8[2] >= (uint32_t)s->P.N) return fail(NOC_ERR_ARG, "bad flit");
  if (f8[7] && (!s->P.age_mode || f8[7] > AGE_MAX || f8[3] >= AGE_ONE))
    return fail(NOC_ERR_ARG, "a flit's age needs age_mode 1, at most 4095, and an inject cycle below 2^20");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  const size_t N = (size_t)s->P.N;
  const uint32_t par = (s->cycle - 1u) & 1u;
  uint4 f = pack_flit(s->P, f8, f8[1]);
  CU(cudaMemcpy(s->P.glink + ((size_t)par * 4 + (dir ^ 1)) * N + nb, &f, sizeof f, cudaMemcpyHostToDevice),
     "link write");
  // counted as injected at its source so that conservation holds
  const uint32_t src = f8[1] < N ? f8[1] : (uint32_t)nb;
  unsigned long long v;
  CU(cudaMemcpy(&v, s->P.stats + S_INJ * N + src, 8, cudaMemcpyDeviceToHost), "counter read");
  v++;
  CU(cudaMemcpy(s->P.stats + S_INJ * N + src, &v, 8, cudaMemcpyHostToDevice), "counter write");
  return NOC_OK;
}

int noc_get_links(noc_sim* s, uint32_t* out) {
  if (!s || !out) return fail(NOC_ERR_ARG, "null argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  const size_t N = (size_t)s->P.N;
  std::vector<uint4> h(4 * N);
  const uint32_t par = (s->cycle - 1u) & 1u;
  CU(cudaMemcpy(h.data(), s->P.glink + (size_t)par * 4 * N, 4 * N * sizeof(uint4), cudaMemcpyDeviceToHost),
     "links copy");
  for (size_t r = 0; r < N; ++r)
    for (int d = 0; d < 4; ++d) {
      uint4 f = h[d * N + r];
      uint32_t* o = out + (r * 4 + d) * 8;
      uint32_t ty = f.z >> 26;
      o[0] = ty;
      o[1] = ty ? (f.y & 0xFFFFu) : 0;
      o[2] = ty ? (f.y >> 16) : 0;
      o[3] = ty ? (s->P.age_mode ? f.x & (AGE_ONE - 1u) : f.x) : 0;
      o[4] = ty ? (f.z & W_LINE) : 0;
      o[5] = ty ? (f.w & 0xFFFFu) : 0;
      o[6] = ty ? (f.w >> 16) : 0;
      o[7] = ty && s->P.age_mode ? f.x >> AGE_SHIFT : 0;
    }
  return NOC_OK;
}

int noc_get_cache(noc_sim* s, int tile, int which, uint32_t* out) {
  if (!s || !out || tile < 0 || tile >= s->P.N || which < 1 || which > 2) return fail(NOC_ERR_ARG, "bad argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  const Params& P = s->P;
  const size_t sets = which == 1 ? P.l1_sets : P.l2_sets, ways = which == 1 ? P.l1_ways : P.l2_ways;
  const size_t n = sets * ways, base = (size_t)tile * n;
  std::vector<uint32_t> w(n);
  std::vector<uint16_t> aux(n, 0);
  CU(cudaMemcpy(w.data(), (which == 1 ? P.l1 : P.l2) + base, n * 4, cudaMemcpyDeviceToHost), "cache copy");
  if (which == 1) CU(cudaMemcpy(aux.data(), P.l1own + base, n * 2, cudaMemcpyDeviceToHost), "owner copy");
  else if (P.l2ep) CU(cudaMemcpy(aux.data(), P.l2ep + base, n * 2, cudaMemcpyDeviceToHost), "epoch copy");
  for (size_t k = 0; k < n; ++k) {
    uint32_t v = w[k];
    bool valid = (v & W_VALID) != 0;
    uint32_t* o = out + k * 4;
    o[0] = valid;
    o[1] = valid ? (v & W_LINE) : 0;
    o[2] = !valid ? 0 : (which == 1 ? aux[k] : (((v & W_DIRTY) ? 1u : 0u) | ((uint32_t)aux[k] << 16)));
    o[3] = valid ? ((v >> W_RANK_SHIFT) & 15u) : 0;
  }
  return NOC_OK;
}

int noc_dir_get(noc_sim* s, uint32_t line, uint32_t* out) {
  if (!s || !out) return fail(NOC_ERR_ARG, "null argument");
  *out = DIR_NONE;
  if (!s->P.dir || line >= s->P.total_lines) return NOC_OK;
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  CU(cudaMemcpy(out, s->P.dir + line, 4, cudaMemcpyDeviceToHost), "directory copy");
  return NOC_OK;
}

int noc_get_core(noc_sim* s, int tile, uint32_t* o) {
  if (!s || !o || tile < 0 || tile >= s->P.N) return fail(NOC_ERR_ARG, "bad argument");
  int rc = ensure_memory(s);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->stream), "sync");
  const size_t N = (size_t)s->P.N;
  uint32_t c[NCORE];
  for (int k = 0; k < NCORE; ++k)
    CU(cudaMemcpy(&c[k], s->P.core + k * N + tile, 4, cudaMemcpyDeviceToHost), "core copy");
  o[0] = c[C_NEXT];
  o[1] = c[C_FSMB] & 0xFFu;
  o[2] = c[C_FLINE];
  o[3] = (c[C_FSMB] >> 8) & 0xFFu;
  o[4] = c[C_FTIMER];
  o[5] = c[C_FSTART];
  o[6] = (c[C_FSMB] >> 16) & 0xFFu;
  o[7] = c[C_OLINE];
  o[8] = c[C_FSMB] >> 24;
  o[9] = c[C_OSTART];
  o[10] = c[C_OTIMER];
  o[11] = c[C_EPOCH] >> 16;
  o[12] = c[C_EPOCH] & 0xFFFFu;
  o[13] = c[C_CQ] >> 16;
  o[14] = c[C_SQ] >> 16;
  o[15] = c[C_MQ] >> 16;
  o[16] = c[C_FWD] >> 16;
  return NOC_OK;
}

int noc_debug_wait_limit(noc_sim* s, int64_t ns, int silent_cta) {
  if (!s || ns < 1) return fail(NOC_ERR_ARG, "bad argument");
  s->wait_ns = ns;
  s->silent_cta = silent_cta;
  return NOC_OK;
}

int64_t noc_kernel_launches(const noc_sim* s) { return s ? s->launches : -1; }

int noc_last_launch_bound(const noc_sim* s) { return s ? s->last_bound : -1; }

int noc_set_checks(noc_sim* s, int enable) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  s->checks_on = enable != 0;
  return NOC_OK;
}

int noc_set_phase_profile(noc_sim* s, int enable) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (enable && !s->d_prof) {
    CU(cudaMalloc(&s->d_prof, 6 * sizeof(unsigned long long)), "profile buffer");
    CU(cudaMemsetAsync(s->d_prof, 0, 6 * sizeof(unsigned long long), s->stream), "profile clear");
  }
  s->prof_on = enable != 0;
  return NOC_OK;
}

int noc_phase_profile(noc_sim* s, uint64_t* out6) {
  if (!s || !out6) return fail(NOC_ERR_ARG, "null argument");
  for (int k = 0; k < 6; ++k) out6[k] = 0;
  if (!s->d_prof) return NOC_OK;
  CU(cudaMemcpyAsync(out6, s->d_prof, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream),
     "profile copy");
  CU(cudaMemsetAsync(s->d_prof, 0, 6 * sizeof(unsigned long long), s->stream), "profile clear");
  CU(cudaStreamSynchronize(s->stream), "sync");
  return NOC_OK;
}

int noc_last_variant(const noc_sim* s, int* loop, int* kind, int* l1_bound, int* l2_bound) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (s->last_variant < 0) return fail(NOC_ERR_STATE, "no cycle-kernel launch yet");
  static const int bounds[3][2] = {{4, 8}, {4, 16}, {16, 16}};
  const int v = s->last_variant, c = v & 15;
  if (loop) *loop = v >> 8;
  if (kind) *kind = (v >> 4) & 15;
  if (l1_bound) *l1_bound = bounds[c][0];
  if (l2_bound) *l2_bound = bounds[c][1];
  return NOC_OK;
}

int noc_kernel_time(noc_sim* s, int enable, double* ms_out, int64_t* launches_out) {
  if (!s) return fail(NOC_ERR_ARG, "null handle");
  if (ms_out || launches_out) {
    double ms = 0.0;
    if (s->tev_used) CU(cudaEventSynchronize(s->tev[s->tev_used - 1]), "event sync");
    for (size_t k = 0; k + 1 < s->tev_used; k += 2) {
      float m = 0.f;
      CU(cudaEventElapsedTime(&m, s->tev[k], s->tev[k + 1]), "event time");
      ms += m;
    }
    if (ms_out) *ms_out = ms;
    if (launches_out) *launches_out = (int64_t)(s->tev_used / 2);
    s->tev_used = 0;
  }
  s->time_kernels = enable != 0;
  return NOC_OK;
}

}  // extern "C"

// ============================================================== batch engine
struct noc_batch {
  std::vector<noc_sim*> sims;
  std::vector<int64_t> cycles;
  unsigned char* pool = nullptr;
  size_t pool_bytes = 0;
  bool pool_owned = false;
  cudaStream_t stream = nullptr;
  std::vector<int> rect;       // per instance: CTA rectangle side (capacity rect * rect tiles)
  std::vector<char> strips;    // per instance: cut into strips of that capacity, not squares
  std::vector<int> group;      // per instance: kernel-variant group (0..4, see noc_batch_run)
  bool collect_hash = true;
  int waves = 0;
  int64_t launches = 0;
  bool done = false;
  std::vector<noc_stats_t> stats;
  std::vector<uint64_t> hash;
  std::vector<std::vector<uint64_t>> hist;
  std::vector<int> err;
  std::vector<int64_t> err_cycle;
  std::vector<int> variant;  // kind << 4 | way class of the kernel that ran each instance
  // device tables
  void* d_tab = nullptr;
  size_t tab_bytes = 0;
};

extern "C" {

int noc_batch_create(int n, const noc_instance_desc* d, noc_batch** out) {
  if (n < 1 || !d || !out) return fail(NOC_ERR_ARG, "bad argument");
  *out = nullptr;
  noc_batch* b = new (std::nothrow) noc_batch();
  if (!b) return fail(NOC_ERR_OOM, "host allocation");
  for (int i = 0; i < n; ++i) {
    if (d[i].traffic.mode == NOC_MODE_TRACE || d[i].cycles < 0 || d[i].cycles >= (int64_t)kMaxChunk) {
      noc_batch_destroy(b);
      return fail(NOC_ERR_ARG, "instance %d: trace mode or cycles outside [0, 2^20)", i);
    }
    noc_sim* s = nullptr;
    int rc = noc_create(d[i].mesh_w, d[i].mesh_h, &d[i].cache, d[i].l2_policy, &d[i].traffic,
                        d[i].seed, &s);
    if (rc) {
      noc_batch_destroy(b);
      return rc;
    }
    // one window of references per tile, drawn before the wave's launch;
    // past it an instance draws in place
    s->refcap = kBatchRefcap;
    layout(s);
    b->sims.push_back(s);
    b->cycles.push_back(d[i].cycles);
  }
  b->stats.resize(n);
  b->hash.assign(n, 0);
  b->hist.assign(n, std::vector<uint64_t>(2 * HIST_BINS, 0));
  b->err.assign(n, 0);
  b->err_cycle.assign(n, -1);
  b->variant.assign(n, -1);
  b->rect.assign(n, 8);
  b->strips.assign(n, 0);
  // kernel-variant groups: the instances the specialised kernels of way class
  // 0, 1, 2 serve -- interleaved L2 (groups 0-2), LSPD with local placement
  // (5-7), LSPD with migration (8-10), each in cache mode with exact ways --
  // those without the packet, write-back, directory-node and age options on
  // the base kernel (3), then the rest on the general kernel (4); those two
  // with the largest way bounds among their instances
  b->group.assign(n, 0);
  int gw1[NOC_BATCH_GROUPS], gw2[NOC_BATCH_GROUPS];
  for (int g = 0; g < NOC_BATCH_GROUPS; ++g) gw1[g] = gw2[g] = 1;
  for (int i = 0; i < n; ++i) {
    const Params& P = b->sims[i]->P;
    const int kind = variant_kind(P), c = batch_way_class(P.l1_ways, P.l2_ways);
    const int g = kind == KIND_IL        ? c
                  : kind == KIND_LOCAL   ? 5 + c
                  : kind == KIND_MIGRATE ? 8 + c
                  : kind == KIND_BASE    ? 3
                                         : 4;
    b->group[i] = g;
    gw1[g] = std::max(gw1[g], P.l1_ways);
    gw2[g] = std::max(gw2[g], P.l2_ways);
  }
  for (int i = 0; i < n; ++i) {
    const int g = b->group[i];
    const int kind = g < 3 ? KIND_IL : g == 3 ? KIND_BASE : g == 4 ? KIND_GEN : g < 8 ? KIND_LOCAL : KIND_MIGRATE;
    b->variant[i] = (kind << 4) | batch_way_class(gw1[g], gw2[g]);
  }
  *out = b;
  return NOC_OK;
}

void noc_batch_destroy(noc_batch* b) {
  if (!b) return;
  for (noc_sim* s : b->sims) {
    s->base = nullptr;  // pool memory is released below, not per instance
    noc_destroy(s);
  }
  if (b->pool && b->pool_owned) cudaFree(b->pool);
  if (b->d_tab) cudaFree(b->d_tab);
  delete b;
}

size_t noc_batch_min_bytes(const noc_batch* b) {
  size_t m = 0;
  if (b)
    for (const noc_sim* s : b->sims) m = std::max(m, s->bytes);
  return m;
}

size_t noc_batch_total_bytes(const noc_batch* b) {
  size_t t = 0;
  if (b)
    for (const noc_sim* s : b->sims) t += s->bytes;
  return t;
}

int noc_batch_bind_memory(noc_batch* b, void* p, size_t bytes) {
  if (!b || !p) return fail(NOC_ERR_ARG, "null argument");
  if (reinterpret_cast<uintptr_t>(p) & 255) return fail(NOC_ERR_ARG, "pool must be 256-byte aligned");
  if (b->pool && b->pool_owned) cudaFree(b->pool);
  b->pool = static_cast<unsigned char*>(p);
  b->pool_bytes = bytes;
  b->pool_owned = false;
  return NOC_OK;
}

int noc_batch_set_stream(noc_batch* b, void* stream) {
  if (!b) return fail(NOC_ERR_ARG, "null handle");
  b->stream = static_cast<cudaStream_t>(stream);
  for (noc_sim* s : b->sims) s->stream = b->stream;
  return NOC_OK;
}

int noc_batch_set_rect(noc_batch* b, int side) {
  if (!b || side < 1 || side * side > 384) return fail(NOC_ERR_ARG, "rectangle side 1..19");
  for (int& r : b->rect) r = side;
  return NOC_OK;
}

int noc_batch_set_strips(noc_batch* b, int enable) {
  if (!b) return fail(NOC_ERR_ARG, "null handle");
  for (char& v : b->strips) v = enable != 0;
  return NOC_OK;
}

int noc_batch_set_layout(noc_batch* b, int i, int side, int strips, int map) {
  if (!b || i < -1 || i >= (int)b->sims.size()) return fail(NOC_ERR_ARG, "bad instance");
  if (side < 1 || side * side > 384) return fail(NOC_ERR_ARG, "rectangle side 1..19");
  if (map < 0 || map > 2) return fail(NOC_ERR_ARG, "thread map 0, 1 or 2");
  const int lo = i < 0 ? 0 : i, hi = i < 0 ? (int)b->sims.size() : i + 1;
  for (int k = lo; k < hi; ++k) {
    b->rect[k] = side;
    b->strips[k] = strips != 0;
    b->sims[k]->thread_map = map;
  }
  return NOC_OK;
}

int noc_batch_group(const noc_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->sims.size()) return -1;
  return b->group[i];
}

int noc_batch_set_thread_map(noc_batch* b, int map) {
  if (!b || map < 0 || map > 2) return fail(NOC_ERR_ARG, "thread map 0, 1 or 2");
  for (noc_sim* s : b->sims) s->thread_map = map;
  return NOC_OK;
}

int noc_batch_set_collect_hash(noc_batch* b, int enable) {
  if (!b) return fail(NOC_ERR_ARG, "null handle");
  b->collect_hash = enable != 0;
  return NOC_OK;
}

// run one kernel-variant group of a batch: memory waves over the pool, one
// work-queue launch per wave, results read back per instance
static int run_batch_group(noc_batch* b, const std::vector<int>& members, int side, int w1, int w2,
                           int kind, int* first_err) {
  const int threads = ((side * side + 31) / 32) * 32;
  int cap = 0;
  CU(max_coresident_batch(w1, w2, kind, threads, &cap), "occupancy");
  std::vector<int> by_size = members;
  for (int i : by_size) {
    noc_sim* s = b->sims[i];
    // squares of side x side tiles, or strips of the same capacity: as wide as
    // the mesh (or the capacity) and as many rows as then fit
    int bw = side, bh = side;
    if (b->strips[i]) {
      bw = std::min(s->P.W, side * side);
      bh = std::max(1, side * side / bw);
    }
    int gx = (s->P.W + bw - 1) / bw, gy = (s->P.H + bh - 1) / bh;
    if (gx * gy > cap || gx * gy * FLAG_SLOTS > (int)s->n_flags)
      return fail(NOC_ERR_ARG, "instance %d needs %d CTAs, %d fit co-resident", i, gx * gy, cap);
    s->run_gx = gx;
    s->run_gy = gy;
  }
  // Queue order.  An instance runs once all its rectangles are popped, so the
  // CTAs are handed out in rounds of `cap`: instances are packed first-fit
  // decreasing by CTA count (then by work) into rounds that fill the
  // co-resident CTAs, and the rounds are queued one after another.  Instances
  // of equal length then start together each round instead of leaving part
  // of the GPU waiting for a gang that does not fit.
  auto ctas = [&](int i) { return b->sims[i]->run_gx * b->sims[i]->run_gy; };
  std::stable_sort(by_size.begin(), by_size.end(), [&](int a, int c) {
    if (ctas(a) != ctas(c)) return ctas(a) > ctas(c);
    return (double)b->sims[a]->P.N * b->cycles[a] > (double)b->sims[c]->P.N * b->cycles[c];
  });
  std::vector<std::vector<int>> rounds;
  std::vector<int> room;
  for (int i : by_size) {
    size_t k = 0;
    while (k < rounds.size() && room[k] < ctas(i)) ++k;
    if (k == rounds.size()) {
      rounds.emplace_back();
      room.push_back(cap);
    }
    rounds[k].push_back(i);
    room[k] -= ctas(i);
  }
  std::vector<int> order;
  for (const auto& r : rounds) order.insert(order.end(), r.begin(), r.end());
  size_t pos = 0;
  while (pos < order.size()) {
    // admit instances in order while their state fits the pool
    std::vector<int> wave;
    size_t used = 0;
    while (pos < order.size()) {
      noc_sim* s = b->sims[order[pos]];
      size_t need = align256(s->bytes);
      if (used + need > b->pool_bytes) break;
      s->base = b->pool + used;
      s->owned = false;
      s->ready = false;
      s->stream = b->stream;
      used += need;
      wave.push_back(order[pos++]);
    }
    b->waves++;
    // reset every instance of the wave and build the work queue
    std::vector<Params> hp;
    std::vector<RunArgs> ha;
    std::vector<int> item_inst, item_rect, need;
    for (int k = 0; k < (int)wave.size(); ++k) {
      noc_sim* s = b->sims[wave[k]];
      int rc = ensure_memory(s);
      if (rc) return rc;
      if (s->P.refcap && b->cycles[wave[k]] > 0) {
        CU(launch_gen_refs(s->P, 0, (uint32_t)b->cycles[wave[k]], b->stream), "reference draw launch");
        b->launches++;
      }
      RunArgs A;
      memset(&A, 0, sizeof A);
      A.t0 = 0;
      A.n = (uint32_t)b->cycles[wave[k]];
      A.gx = s->run_gx;
      A.gy = s->run_gy;
      A.abort_flag = abort_ptr(s);
      A.wait_ns = s->wait_ns;
      A.silent_cta = -1;
      A.thread_map = s->thread_map;
      hp.push_back(s->P);
      ha.push_back(A);
      const int G = s->run_gx * s->run_gy;
      need.push_back(A.n ? G : 0);
      if (A.n)
        for (int r = 0; r < G; ++r) {
          item_inst.push_back(k);
          item_rect.push_back(r);
        }
    }
    const int m = (int)wave.size(), ni = (int)item_inst.size();
    size_t o_p = 0, o_a = align256(o_p + m * sizeof(Params)), o_ii = align256(o_a + m * sizeof(RunArgs)),
           o_ir = align256(o_ii + ni * 4), o_nd = align256(o_ir + ni * 4), o_cl = align256(o_nd + m * 4),
           o_nx = align256(o_cl + m * 4), bytes = align256(o_nx + 4);
    if (bytes > b->tab_bytes) {
      if (b->d_tab) cudaFree(b->d_tab);
      b->d_tab = nullptr;
      CU(cudaMalloc(&b->d_tab, bytes), "batch tables");
      b->tab_bytes = bytes;
    }
    unsigned char* t = static_cast<unsigned char*>(b->d_tab);
    cudaStream_t st = b->stream;
    CU(cudaMemcpyAsync(t + o_p, hp.data(), m * sizeof(Params), cudaMemcpyHostToDevice, st), "params");
    CU(cudaMemcpyAsync(t + o_a, ha.data(), m * sizeof(RunArgs), cudaMemcpyHostToDevice, st), "args");
    if (ni) {
      CU(cudaMemcpyAsync(t + o_ii, item_inst.data(), ni * 4, cudaMemcpyHostToDevice, st), "items");
      CU(cudaMemcpyAsync(t + o_ir, item_rect.data(), ni * 4, cudaMemcpyHostToDevice, st), "items");
    }
    CU(cudaMemcpyAsync(t + o_nd, need.data(), m * 4, cudaMemcpyHostToDevice, st), "need");
    CU(cudaMemsetAsync(t + o_cl, 0, m * 4, st), "claimed");
    CU(cudaMemsetAsync(t + o_nx, 0, 4, st), "queue head");
    BatchArgs B;
    B.params = reinterpret_cast<const Params*>(t + o_p);
    B.args = reinterpret_cast<const RunArgs*>(t + o_a);
    B.item_inst = reinterpret_cast<const int*>(t + o_ii);
    B.item_rect = reinterpret_cast<const int*>(t + o_ir);
    B.need = reinterpret_cast<const int*>(t + o_nd);
    B.claimed = reinterpret_cast<unsigned int*>(t + o_cl);
    B.next_item = reinterpret_cast<unsigned int*>(t + o_nx);
    B.n_items = ni;
    // A CTA that pops a rectangle waits until its instance's other rectangles
    // are popped, i.e. at most until instances already running end.  Those
    // run at a few microseconds per simulated cycle; the bound allows 500 us
    // per cycle of the wave's longest instance, plus 20 s.
    int64_t max_cycles = 0;
    for (int k = 0; k < m; ++k) max_cycles = std::max<int64_t>(max_cycles, b->cycles[wave[k]]);
    B.gang_ns = 20ll * 1000000000ll + max_cycles * 500000ll;
    if (ni) {
      CU(launch_batch(B, std::min(cap, ni), threads, w1, w2, kind, st), "batch kernel launch");
      b->launches++;
    }
    CU(cudaStreamSynchronize(st), "batch wave");
    // read each instance's results before its memory is reused
    for (int k = 0; k < m; ++k) {
      const int i = wave[k];
      noc_sim* s = b->sims[i];
      s->cycle = (uint32_t)b->cycles[i];
      int64_t ec = -1;
      int rc = read_error(s, &ec);
      b->err[i] = rc;
      b->err_cycle[i] = ec;
      if (rc && !*first_err) *first_err = rc;
      rc = noc_stats(s, -1, &b->stats[i]);
      if (rc) return rc;
      b->launches++;
      rc = noc_latency_hist(s, 0, b->hist[i].data(), HIST_BINS);
      if (!rc) rc = noc_latency_hist(s, 1, b->hist[i].data() + HIST_BINS, HIST_BINS);
      if (rc) return rc;
      if (b->collect_hash) {
        uint64_t h = 0;
        rc = noc_state_hash(s, &h);
        if (rc) return rc;
        b->hash[i] = h;
        b->launches += 2;
      }
      s->ready = false;
      s->base = nullptr;
    }
  }
  return NOC_OK;
}

int noc_batch_run(noc_batch* b) {
  if (!b) return fail(NOC_ERR_ARG, "null handle");
  const int n = (int)b->sims.size();
  if (!b->pool) {
    size_t fr = 0, tot = 0;
    CU(cudaMemGetInfo(&fr, &tot), "memory info");
    size_t want = std::min(noc_batch_total_bytes(b), (size_t)(fr * 0.8));
    want = std::max(want, noc_batch_min_bytes(b));
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) return fail(NOC_ERR_OOM, "batch pool of %zu bytes: %s", want, cudaGetErrorString(e));
    b->pool = static_cast<unsigned char*>(p);
    b->pool_bytes = want;
    b->pool_owned = true;
  }
  if (noc_batch_min_bytes(b) > b->pool_bytes)
    return fail(NOC_ERR_OOM, "pool of %zu bytes is below the largest instance (%zu)", b->pool_bytes,
                noc_batch_min_bytes(b));
  // one run per kernel-variant group (fixed at create) and rectangle side:
  // the CTAs of one launch all have the side's thread count
  b->waves = 0;
  int first_err = NOC_OK;
  static const int bounds[3][2] = {{4, 8}, {4, 16}, {16, 16}};
  for (int g = 0; g < NOC_BATCH_GROUPS; ++g)
    for (int side = 1; side * side <= 384; ++side) {
      std::vector<int> members;
      for (int i = 0; i < n; ++i)
        if (b->group[i] == g && b->rect[i] == side) members.push_back(i);
      if (members.empty()) continue;
      const int v = b->variant[members[0]], kind = v >> 4, c = v & 15;
      int rc = run_batch_group(b, members, side, bounds[c][0], bounds[c][1], kind, &first_err);
      if (rc) return rc;
    }
  b->done = true;
  if (first_err) return fail(first_err, "an instance ended with error %d", first_err);
  return NOC_OK;
}

int noc_batch_waves(const noc_batch* b) { return b ? b->waves : -1; }

int noc_batch_error(const noc_batch* b, int i, int64_t* err_cycle) {
  if (!b || i < 0 || i >= (int)b->sims.size()) return fail(NOC_ERR_ARG, "bad argument");
  if (err_cycle) *err_cycle = b->err_cycle[i];
  return b->err[i];
}

int noc_batch_stats(const noc_batch* b, int i, noc_stats_t* out) {
  if (!b || !out || i < 0 || i >= (int)b->sims.size()) return fail(NOC_ERR_ARG, "bad argument");
  if (!b->done) return fail(NOC_ERR_STATE, "batch has not run");
  *out = b->stats[i];
  return NOC_OK;
}

int noc_batch_state_hash(const noc_batch* b, int i, uint64_t* out) {
  if (!b || !out || i < 0 || i >= (int)b->sims.size()) return fail(NOC_ERR_ARG, "bad argument");
  if (!b->done || !b->collect_hash) return fail(NOC_ERR_STATE, "no hashes collected");
  *out = b->hash[i];
  return NOC_OK;
}

int noc_batch_latency_hist(const noc_batch* b, int i, int which, uint64_t* bins, int nbins) {
  if (!b || !bins || i < 0 || i >= (int)b->sims.size() || which < 0 || which > 1 || nbins < HIST_BINS)
    return fail(NOC_ERR_ARG, "bad argument");
  if (!b->done) return fail(NOC_ERR_STATE, "batch has not run");
  memcpy(bins, b->hist[i].data() + which * HIST_BINS, HIST_BINS * 8);
  return NOC_OK;
}

int64_t noc_batch_kernel_launches(const noc_batch* b) { return b ? b->launches : -1; }

int noc_batch_variant(const noc_batch* b, int i, int* kind, int* l1_bound, int* l2_bound) {
  if (!b || i < 0 || i >= (int)b->sims.size()) return fail(NOC_ERR_ARG, "bad argument");
  if (b->variant[i] < 0) return fail(NOC_ERR_STATE, "batch has not run");
  static const int bounds[3][2] = {{4, 8}, {4, 16}, {16, 16}};
  const int v = b->variant[i], c = v & 15;
  if (kind) *kind = v >> 4;
  if (l1_bound) *l1_bound = bounds[c][0];
  if (l2_bound) *l2_bound = bounds[c][1];
  return NOC_OK;
}

}  // extern "C"
