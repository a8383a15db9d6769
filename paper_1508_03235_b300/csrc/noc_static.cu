// noc_static.cu -- a simulation entry point that allocates no device memory.
//
// Who needs it: code that runs where the process's device memory is already
// owned by someone else -- a framework whose caching allocator has reserved
// the HBM, so a stray cudaMalloc would fail or fragment it, or a host loop
// that must never allocate (nor take cudaMalloc/cudaFree's implicit device
// synchronisation) once it is running.  noc_run_static runs a whole
// simulation from cycle 0 with every piece of simulator state and scratch
// (links, tile records, queues, caches, per-CTA cycle flags, error word) in
// one fixed, file-scope device array, and writes only the caller's output.
//
// The array is NOC_STATIC_SCRATCH_BYTES (16 MiB) and every GPU that loads the
// library holds it until the process exits.  All calls share it and it keeps
// the previous call's contents, so each call clears what must start at zero.
// Within one process the calls cannot overlap: an internal lock is held from
// the first clear until the call's stream has finished.  Each process has its
// own copy of the array.
#include <cstring>
#include <mutex>

#include "noc.h"
#include "noc_host.h"

using namespace noc;

static __device__ __align__(256) unsigned char g_static_scratch[NOC_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_mu;
unsigned char* g_dev_ptr[256];  // device address of g_static_scratch, per device
bool g_dev_ready[256];

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// noc_stats_t from the per-counter totals (device order of the model's list)
__global__ void pack_stats_kernel(const unsigned long long* h, unsigned long long cycle,
                                  unsigned long long* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int order[] = {S_INJ, S_EJ, -1, S_DEFL, S_LATSUM, S_LATMAX, S_REFS, S_L1H, S_L1M,
                       S_L2H, S_L2M, S_REQM, S_REQR, S_REPS, S_REPR, S_DIRS, S_MEMREQ, S_MEMW,
                       S_MEMWB, S_WTS, S_WTH, S_TRAP, S_REDIR, S_MIGR, S_L2LSUM, S_L2LCNT,
                       S_CQST, S_MMST, S_MIGS};
  out[0] = cycle;
  for (int k = 0; k < 29; ++k) out[1 + k] = order[k] < 0 ? h[S_INJ] - h[S_EJ] : h[order[k]];
}

}  // namespace

extern "C" int noc_run_static(int mesh_w, int mesh_h, const noc_cache_cfg* c, int l2_policy,
                              const noc_traffic* tr, uint64_t seed, int64_t n_cycles,
                              void* dev_stats_out, void* cuda_stream) {
  if (!c || !tr || !dev_stats_out) return fail(NOC_ERR_ARG, "null argument");
  if (n_cycles < 0 || n_cycles >= (1ll << 31)) return fail(NOC_ERR_ARG, "n_cycles outside [0, 2^31)");
  // the same configurations noc_create accepts, with the same messages
  Params P;
  int rc = configure(mesh_w, mesh_h, c, l2_policy, tr, seed, P);
  if (rc) return rc;
  // trace mode needs per-core reference lists, which live outside the array
  if (tr->mode == NOC_MODE_TRACE)
    return fail(NOC_ERR_ARG, "trace mode is not available without allocation");
  if (c->age_mode && n_cycles > (1ll << AGE_SHIFT))
    return fail(NOC_ERR_ARG, "age_mode 1 runs end at or before cycle 2^%d", AGE_SHIFT);
  const size_t N = (size_t)P.N;
  const uint64_t total = P.total_lines;

  // carve the state out of the static array
  const size_t w1 = N * P.l1_sets * P.l1_ways, w2 = N * P.l2_sets * P.l2_ways;
  const bool lspd = l2_policy != NOC_L2_INTERLEAVED, mig = l2_policy == NOC_L2_LSPD_MIGRATE;
  const size_t n_flags = 1024 * FLAG_SLOTS;
  size_t off[20], cur = 0;
  const size_t sz[20] = {2 * 4 * N * 16, NCORE * N * 4, N * P.core_q * 16, N * P.svc_q * 16,
                         N * P.mem_q * 16, w1 * 4, w1 * 2, w2 * 4, lspd ? w2 * 2 : 0,
                         mig ? w2 * hist_stride(P.mig_window) * 2 : 0, lspd ? (size_t)total * 4 : 0,
                         mig ? N * P.fwd_cap * 8 : 0, (size_t)NSTAT * N * 8,
                         2 * HIST_BINS * 8, n_flags * 4, 8, 4, 64 * 8, 2 * 4 * N * 32,
                         N * (size_t)P.rob_entries * 8};
  for (int k = 0; k < 20; ++k) {
    off[k] = a256(cur);
    cur = off[k] + sz[k];
  }
  if (cur > NOC_STATIC_SCRATCH_BYTES)
    return fail(NOC_ERR_ARG, "state needs %zu bytes > NOC_STATIC_SCRATCH_BYTES (%u)", cur,
                (unsigned)NOC_STATIC_SCRATCH_BYTES);

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
  if (dev < 0 || dev >= 256) return fail(NOC_ERR_CUDA, "device %d out of range", dev);
  if (!g_dev_ready[dev]) {
    // first call on this device: the array's device address, with it current
    void* p = nullptr;
    ce = cudaGetSymbolAddress(&p, g_static_scratch);
    if (ce != cudaSuccess || !p)
      return fail(NOC_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(ce));
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    g_dev_ready[dev] = true;
  }
  unsigned char* b = g_dev_ptr[dev];
  P.glink = reinterpret_cast<uint4*>(b + off[0]);
  P.core = reinterpret_cast<uint32_t*>(b + off[1]);
  P.cq = reinterpret_cast<uint4*>(b + off[2]);
  P.sq = reinterpret_cast<uint4*>(b + off[3]);
  P.mq = reinterpret_cast<uint4*>(b + off[4]);
  P.l1 = reinterpret_cast<uint32_t*>(b + off[5]);
  P.l1own = reinterpret_cast<uint16_t*>(b + off[6]);
  P.l2 = reinterpret_cast<uint32_t*>(b + off[7]);
  P.l2ep = lspd ? reinterpret_cast<uint16_t*>(b + off[8]) : nullptr;
  P.l2hist = mig ? reinterpret_cast<uint16_t*>(b + off[9]) : nullptr;
  P.dir = lspd ? reinterpret_cast<uint32_t*>(b + off[10]) : nullptr;
  P.fwd = mig ? reinterpret_cast<uint32_t*>(b + off[11]) : nullptr;
  P.stats = reinterpret_cast<unsigned long long*>(b + off[12]);
  P.hist = reinterpret_cast<unsigned long long*>(b + off[13]);
  P.flags = reinterpret_cast<unsigned int*>(b + off[14]);
  P.err = reinterpret_cast<unsigned long long*>(b + off[15]);
  unsigned int* abort_flag = reinterpret_cast<unsigned int*>(b + off[16]);
  unsigned long long* totals = reinterpret_cast<unsigned long long*>(b + off[17]);
  P.gtag = reinterpret_cast<uint4*>(b + off[18]);
  P.rob = P.rob_entries ? reinterpret_cast<uint32_t*>(b + off[19]) : nullptr;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // everything the simulation reads before writing starts from its reset value
  for (int k = 0; k < 20; ++k) {
    if (!sz[k] || k == 2 || k == 3 || k == 4) continue;  // queue slots are written before read
    int v = (k == 10 || k == 15) ? 0xFF : 0;              // directory NONE, no error
    ce = cudaMemsetAsync(b + off[k], v, sz[k], st);
    if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(ce));
  }

  // CTA rectangles: the fewest that hold at most 256 tiles each and fit co-resident
  int gx = 0, gy = 0;
  for (int side = 16; side >= 1 && !gx; side /= 2) {
    int tx = (mesh_w + side - 1) / side, ty = (mesh_h + side - 1) / side;
    int threads = block_threads(mesh_w, mesh_h, tx, ty), cap = 0;
    if (threads > RUN_MAX_THREADS || (size_t)tx * ty * FLAG_SLOTS > n_flags) continue;
    ce = max_coresident_ctas(P, threads, &cap);
    if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "occupancy: %s", cudaGetErrorString(ce));
    if (tx * ty <= cap) {
      gx = tx;
      gy = ty;
    }
  }
  if (!gx) return fail(NOC_ERR_ARG, "mesh %dx%d does not fit one co-resident launch", mesh_w, mesh_h);

  uint32_t done = 0;
  while (done < (uint32_t)n_cycles) {
    uint32_t left = (uint32_t)n_cycles - done, n = left < (1u << 20) ? left : (1u << 20);
    RunArgs A;
    A.t0 = done;
    A.n = n;
    A.draining = 0;
    A.gx = gx;
    A.gy = gy;
    A.hash_trace = nullptr;
    A.busy = nullptr;
    A.abort_flag = abort_flag;
    A.wait_ns = 2000000000ll;
    A.silent_cta = -1;
    A.thread_map = 0;
    A.prof = nullptr;
    A.checked = 0;
    ce = launch_run(P, A, st);
    if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "cycle kernel launch: %s", cudaGetErrorString(ce));
    done += n;
  }
  ce = launch_reduce_stats(P, -1, totals, st);
  if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "counter reduction: %s", cudaGetErrorString(ce));
  pack_stats_kernel<<<1, 32, 0, st>>>(totals, (unsigned long long)n_cycles,
                                      static_cast<unsigned long long*>(dev_stats_out));
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "counter packing: %s", cudaGetErrorString(ce));
  unsigned long long e = ~0ull;
  ce = cudaMemcpyAsync(&e, P.err, 8, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(NOC_ERR_CUDA, "error word: %s", cudaGetErrorString(ce));
  if (e == ~0ull) return NOC_OK;
  const int code = (int)(e & 0xFF);
  return fail(code, "simulation error %d at cycle %lld", code, (long long)(e >> 8));
}
