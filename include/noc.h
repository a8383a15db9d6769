/*
 * noc.h -- C ABI of libnoc.so, the B300 (sm_103a) simulator of a W x H mesh
 * chip multicore joined by a bufferless, deflection-routed NoC with a
 * logically-shared, physically-distributed (LSPD) L2 (Kumar & Sahu,
 * "Bufferless NOC Simulation of Large Multicore System on GPU Hardware",
 * arXiv 1508.03235).
 *
 * Every simulated cycle: each tile advances its core / L1 / L2-slice /
 * directory state (Sec. 7.1 "Work in phase one"), each router ejects one flit,
 * may inject one, sorts its flits oldest-first and gives each a productive or
 * a deflected output port (Sec. 4.2, Sec. 4.3, Sec. 7.1 "phase two"), and the
 * ejected flit is handled at its tile (Sec. 7.1 "phase three").
 *
 * Conventions for every entry point:
 *   - Status: an int, NOC_OK (0) or one of the NOC_ERR_* codes below;
 *     noc_last_error() returns a thread-local message for the last failure.
 *   - Pointers named `out`/`bins`/`buf` are HOST memory owned by the caller,
 *     large enough for the stated element count; the library only writes them.
 *   - Handles are owned by the caller and released with noc_destroy().
 *   - Device work is enqueued on the stream set by noc_set_stream (default:
 *     the legacy default stream).  noc_step returns after enqueueing; the
 *     query functions (noc_stats, noc_state_hash, ...) synchronise that stream
 *     first.  A handle must not be used from two host threads at once.
 *   - Results depend only on the arguments: never on the stream, the CTA tile
 *     shape, or on what else runs on the GPU.
 */
#ifndef NOC_H
#define NOC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NOC_OK 0
#define NOC_ERR_ARG 1            /* invalid argument or configuration            */
#define NOC_ERR_OOM 2            /* device or host allocation failed             */
#define NOC_ERR_QUEUE_OVERFLOW 3 /* a service queue or memory FIFO overflowed    */
#define NOC_ERR_TIMEOUT 4        /* a device-side wait ran past its limit        */
#define NOC_ERR_CUDA 5           /* a CUDA runtime call failed                   */
#define NOC_ERR_PROTOCOL 6       /* a reply arrived that matches no request      */
#define NOC_ERR_STATE 7          /* call not valid in the handle's current state */
#define NOC_ERR_RANGE 8          /* age_mode 1: a flit deflected with age 4095   */
#define NOC_ERR_OWNER 9          /* checked build: a directory entry touched away
                                    from its line's directory tile (noc_set_checks) */

/* L2 placement (Sec. 3): interleaved homes; LSPD with local placement and a
 * home-tile directory (Sec. 3.2, Sec. 6.2.2); LSPD plus migration and
 * redirection (Sec. 3.3). */
#define NOC_L2_INTERLEAVED 0
#define NOC_L2_LSPD_LOCAL 1
#define NOC_L2_LSPD_MIGRATE 2

/* reference streams: Philox cache traffic (the synthetic stand-in for the
 * paper's trace-driven input, Sec. 6.2.3), network-only probes, or
 * caller-supplied per-core traces */
#define NOC_MODE_CACHE 0
#define NOC_MODE_NETWORK 1
#define NOC_MODE_TRACE 2

/* Cache geometry and latencies (64 B lines).  Paper Sec. 3.1 (private L1,
 * equal L2 slices), Table 4 (set/way/line configurations). */
typedef struct {
  int32_t l1_sets, l1_ways;   /* ways 1..16 */
  int32_t l2_sets, l2_ways;   /* ways 1..16 */
  int32_t l1_miss_cycles;     /* L1 miss wait before the L2 step (Sec. 7.1) */
  int32_t mem_latency;        /* cycles of an off-chip access, >= 1         */
  int32_t mig_window;         /* accessors remembered per L2 block (Sec. 3.1), 1..30 */
  int32_t mig_threshold;      /* occurrences of one requester that migrate the block */
  int32_t core_q;             /* core send-queue capacity (back-pressure)    */
  int32_t svc_q;              /* service-queue capacity (overflow = error)   */
  int32_t mem_q;              /* memory-return FIFO capacity (overflow = error) */
  int32_t fwd_entries;        /* redirection forward-table entries per tile  */
  /* Packets (Table 1, Sec. 2.3).  0: every message is one flit.  1: a data
   * reply (remote L2 access) is 4 flits and a block migration 16, queued
   * together, routed independently and reassembled at the receiver in a
   * reorder buffer of rob_entries packets (1..64; a full buffer is
   * NOC_ERR_QUEUE_OVERFLOW); the message's handler runs in the cycle its last
   * flit is ejected.  Needs svc_q >= 16. */
  int32_t packet_mode, rob_entries;
  /* Directory placement (LSPD policies, Sec. 3.2): dir_central 0 keeps each
   * line's entry at its home tile (line mod N); 1 keeps every entry at one
   * directory node, tile dir_tile (0..N-1) -- the centralized organisation
   * whose node becomes a hot spot.  Ignored by the interleaved policy. */
  int32_t dir_central, dir_tile;
  /* L1 write policy: 0 = write-through (Sec. 3.1, 3.2: every write goes to
   * the L2 that supplied the line); 1 = write-back (Sec. 3.4, 7.1: a write
   * dirties the L1 copy; a dirty victim is written to that L2, or to memory
   * if none holds it, when it is evicted). */
  int32_t l1_write_back;
  /* Router priority (Sec. 4.2, 4.3).  0: oldest first -- smaller inject
   * cycle, then smaller source tile.  1: the paper's age field, a flit's
   * count of deflections (Sec. 6.2.1, 7.1): more deflections first, ties by
   * the age_mode 0 order; a new flit has age 0.  Under age_mode 1 a flit
   * counts at most 4095 deflections (one more ends the step with
   * NOC_ERR_RANGE) and a run ends at or before cycle 2^20 (a step, drain or
   * batch that would pass it is NOC_ERR_ARG). */
  int32_t age_mode;
} noc_cache_cfg;

/* Reference stream.  Fractions are q16 fixed point (65536 = 1).  Reference k
 * of core c is eligible at cycle k*period and is drawn from
 * Philox4x64-10(counter=(k, c, stream, 0), key=(seed, 0x4E4F43)). */
typedef struct {
  int32_t mode;               /* NOC_MODE_*; period 0 = no references        */
  int32_t period;
  uint32_t write_q16, priv_q16, shared_q16; /* remote = the rest            */
  uint32_t hot_q16;           /* share of shared refs sent to the hot block  */
  int32_t hot_side;           /* side of the hot block of tiles at the centre (0 = none) */
  uint32_t priv_lines, shared_lines, remote_lines;
  uint32_t stream;            /* Philox counter word 2                       */
} noc_traffic;

/* Totals over all tiles (lat_max is a maximum).  Counter definitions follow
 * the paper's statistics list (Sec. 6.2.2, Table 3 columns). */
typedef struct {
  uint64_t cycle;
  uint64_t injected, ejected, in_flight, deflections, lat_sum, lat_max, refs;
  uint64_t l1_hit, l1_miss, l2_hit, l2_miss;
  uint64_t req_made, req_rcvd, reply_sent, reply_rcvd, dir_search, mem_req;
  uint64_t mem_write, mem_wb, wt_sent, wt_hit, trap, redir, migrations;
  uint64_t l2lat_sum, l2lat_cnt, cq_stall, mm_stall, mig_sent;
} noc_stats_t;

#define NOC_HIST_BINS 1025 /* 1-cycle bins 0..1023 plus one overflow bin */

typedef struct noc_sim noc_sim;

/* Create a simulation handle (host-side only; device memory is taken at the
 * first call that needs it, from noc_bind_memory or else cudaMalloc on the
 * current device).  Returns NOC_ERR_ARG for an invalid configuration
 * (mesh_w * mesh_h above 65,535 tiles, bad geometry). */
int noc_create(int mesh_w, int mesh_h, const noc_cache_cfg* cache, int l2_policy,
               const noc_traffic* traffic, uint64_t seed, noc_sim** out);
void noc_destroy(noc_sim* sim);

/* Device bytes the handle needs; give the library caller-owned device memory
 * (at least that many bytes, 256-byte aligned) that it will never free. */
size_t noc_required_bytes(const noc_sim* sim);
int noc_bind_memory(noc_sim* sim, void* dev_ptr, size_t bytes);

/* cudaStream_t to enqueue on (NULL = default stream). */
int noc_set_stream(noc_sim* sim, void* cuda_stream);

/* Return to cycle 0: empty caches, links, queues, counters (enqueued). */
int noc_reset(noc_sim* sim);

/* Enqueue n_cycles simulated cycles (Sec. 7.2 main loop) as persistent
 * cooperative launches.  Returns the first error of earlier work if one is
 * already known, else NOC_OK. */
int noc_step(noc_sim* sim, int64_t n_cycles);

/* Stop issuing references and run until nothing is in flight, queued or
 * outstanding, or max_cycles pass.  *taken = cycles run.  Synchronous.
 * NOC_ERR_TIMEOUT if not quiescent after max_cycles.  References stay stopped
 * for later noc_step calls until noc_reset. */
int noc_drain(noc_sim* sim, int64_t max_cycles, int64_t* taken);

/* Wait for enqueued work; return the first device error (NOC_OK if none) and,
 * if err_cycle != NULL, the simulated cycle it happened in (-1 if none). */
int noc_sync(noc_sim* sim, int64_t* err_cycle);

/* Checkpoint and resume.  noc_save writes the whole simulation state -- the
 * device arena byte for byte plus the cycle and a drain's reference stop --
 * into host memory the caller owns (noc_checkpoint_bytes(sim) bytes; waits for
 * the handle's stream).  noc_load restores it into a handle created with the
 * same arguments (mesh, cache configuration, L2 policy, traffic, seed): every
 * later step then gives exactly the results of the run that was saved.  A
 * trace-mode handle must be given the same per-core reference lists again.
 * noc_load returns NOC_ERR_ARG, before touching the device, for an image that
 * is not a checkpoint or was saved from another configuration.  Not in the
 * paper (an operational facility). */
size_t noc_checkpoint_bytes(const noc_sim* sim);
int noc_save(noc_sim* sim, void* host_buf, size_t bytes);
int noc_load(noc_sim* sim, const void* host_buf, size_t bytes);

/* Totals (tile < 0) or one tile's counters, copied to host memory. */
int noc_stats(noc_sim* sim, int tile, noc_stats_t* out);
/* which: 0 = flit latency, 1 = L2 access latency; bins: nbins >= NOC_HIST_BINS */
int noc_latency_hist(noc_sim* sim, int which, uint64_t* bins, int nbins);

/* Order-free hashes of the simulation state, with mix64 the splitmix64
 * finaliser and fold(w0, w1, ...) = h <- mix64(w0 + 0x9E3779B97F4A7C15), then
 * h <- mix64(h ^ wi) per further word:
 *   dynamic hash = sum over tiles r (mod 2^64) of fold(r, the four output
 *     flits of the last cycle, the core record words, injected, ejected,
 *     deflections) -- the state a cycle carries to the next;
 *   full hash = dynamic hash + fold(0x18, cycle) + sums of folds over every
 *     valid L1 and L2 way, queue and memory-FIFO entry, directory and forward
 *     entry (each tagged 0x11..0x17).
 * Both are independent of how the state is laid out or ordered in memory. */
int noc_dyn_hash(noc_sim* sim, uint64_t* out);
int noc_state_hash(noc_sim* sim, uint64_t* out);
/* Record the dynamic hash after every cycle of the following noc_step calls
 * (enable != 0), and read the records of the last step: buf has n slots. */
int noc_set_hash_trace(noc_sim* sim, int enable);
int noc_hash_trace(noc_sim* sim, uint64_t* buf, int64_t n);

/* CTA rectangle grid (gx x gy rectangles of the mesh, one CTA each).
 * 0,0 = the library's choice.  Results never depend on it. */
int noc_set_tiling(noc_sim* sim, int gx, int gy);
int noc_get_tiling(const noc_sim* sim, int* gx, int* gy);

/* Tiles per thread of the plain loop: 1 keeps each tile's state in its
 * thread's registers for a whole launch (the fast loop; a mesh must then fit
 * one co-resident launch: at most 148 rectangles of at most 448 tiles on a
 * B300, which every mesh up to the 65,535 tiles that 16-bit tile indices allow
 * meets when its shape cuts that way, e.g. 255 x 257 as 4 x 37 rectangles of
 * 64 x 7); 2 runs two tiles per thread and moves each tile's state through its
 * device records around every cycle (slower per tile, for the shapes that do
 * not cut that way); 0 = automatic (1 if the mesh fits that way, else 2, the
 * default).  With two, per-cycle hash
 * traces and noc_drain are NOC_ERR_ARG (they need the one-tile loop); results
 * never depend on it.  noc_get_tiles_per_thread returns the value in use
 * (0 before the first launch, -1 for a null handle). */
int noc_set_tiles_per_thread(noc_sim* sim, int k);
int noc_get_tiles_per_thread(const noc_sim* sim);

/* Tile-to-thread order inside each CTA rectangle: 0 = perimeter tiles first
 * (the default), 1 = row-major, 2 = column-major.  Results never depend on
 * it; the autotuner picks it with the tiling.  noc_get_thread_map returns the
 * current order, or -1 for a null handle. */
int noc_set_thread_map(noc_sim* sim, int map);
int noc_get_thread_map(const noc_sim* sim);

/* Trace mode: reference list of one core (line | write << 31), copied. */
int noc_set_trace(noc_sim* sim, int core, int64_t n, const uint32_t* refs);

/* Test and inspection entry points (synchronous, between steps).
 * Flits are 8 host words: type, src, dst, inject_cycle, line, a, e, age (the
 * deflection count of age_mode 1; ignored when enqueued, and a non-zero age
 * on a link needs age_mode 1 and at most 4095). */
int noc_debug_enqueue(noc_sim* sim, int tile, int queue /*0 core,1 service*/,
                      const uint32_t* flit8);
int noc_debug_link(noc_sim* sim, int tile, int dir /*0 N,1 S,2 E,3 W*/,
                   const uint32_t* flit8);
int noc_get_links(noc_sim* sim, uint32_t* out /* N*4*8 */);
int noc_get_cache(noc_sim* sim, int tile, int which /*1 L1, 2 L2*/,
                  uint32_t* out /* sets*ways*4: valid, line, aux, rank */);
int noc_dir_get(noc_sim* sim, uint32_t line, uint32_t* out);
int noc_get_core(noc_sim* sim, int tile, uint32_t* out17);
/* Device-wait limit in nanoseconds (default 2e9) and a test fault: CTA
 * `silent_cta` stops publishing its cycle (-1 = none), so its neighbours'
 * bounded waits run out and the step ends with NOC_ERR_TIMEOUT. */
int noc_debug_wait_limit(noc_sim* sim, int64_t ns, int silent_cta);

/* ------------------------------------------------------------------------
 * Batch engine: many independent simulations of uneven size, seed and L2
 * policy in one persistent cooperative launch per memory wave.  CTAs pop
 * (instance, rectangle) items from a device work queue; each instance's
 * rectangles run together with the neighbour waits of noc_step.  Instances
 * are first grouped by the kernel variant that serves them (the interleaved
 * L2 in cache mode with the exact way counts of a variant's class runs on
 * that specialised kernel; all other instances share the general one), and
 * each group runs in its own waves.  Each instance's results are
 * bit-identical to running it alone through noc_create / noc_step (trace
 * mode is not supported in a batch).
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t mesh_w, mesh_h, l2_policy, reserved;
  noc_cache_cfg cache;
  noc_traffic traffic;
  uint64_t seed;
  int64_t cycles;             /* cycles to simulate from cycle 0, < 2^20 */
} noc_instance_desc;

typedef struct noc_batch noc_batch;

int noc_batch_create(int n, const noc_instance_desc* descs, noc_batch** out);
void noc_batch_destroy(noc_batch* batch);
/* Device bytes of the largest instance (the least memory a run can use) and
 * of all instances at once (what one wave needs). */
size_t noc_batch_min_bytes(const noc_batch* batch);
size_t noc_batch_total_bytes(const noc_batch* batch);
/* Caller-owned device pool the instances' state is placed in, wave by wave
 * (never freed by the library); without it the run takes a pool with
 * cudaMalloc sized to the smaller of the total and 80% of free memory. */
int noc_batch_bind_memory(noc_batch* batch, void* dev_ptr, size_t bytes);
int noc_batch_set_stream(noc_batch* batch, void* cuda_stream);
/* CTA rectangle side in tiles (1..19; default 8): a tuning knob only. */
int noc_batch_set_rect(noc_batch* batch, int side);
/* Tile-to-thread order of every instance (as noc_set_thread_map; default 0):
 * a tuning knob only. */
int noc_batch_set_thread_map(noc_batch* batch, int map);
/* enable != 0: cut each instance into strips of at most side * side tiles --
 * as wide as the mesh (or side * side) with as many rows as then fit --
 * instead of side x side squares, so that east-west links stay inside a CTA.
 * A tuning knob only (default 0). */
int noc_batch_set_strips(noc_batch* batch, int enable);
/* Layout of instance i (i = -1: every instance): CTA rectangle side 1..19,
 * strips on or off and tile-to-thread order, as the three setters above.
 * Tuning knobs only; instances of one kernel-variant group with different
 * sides run in separate launches. */
int noc_batch_set_layout(noc_batch* batch, int i, int side, int strips, int thread_map);
/* Collect each instance's full state hash after its wave (default on). */
int noc_batch_set_collect_hash(noc_batch* batch, int enable);
/* Run every instance to its cycle count.  Synchronous.  Returns the first
 * instance error (see noc_batch_error for each). */
int noc_batch_run(noc_batch* batch);
/* Work-queue launches of the last run: at least one per kernel-variant group
 * present, more when a group's state exceeds the pool. */
int noc_batch_waves(const noc_batch* batch);
int noc_batch_error(const noc_batch* batch, int i, int64_t* err_cycle);
int noc_batch_stats(const noc_batch* batch, int i, noc_stats_t* out);
int noc_batch_state_hash(const noc_batch* batch, int i, uint64_t* out);
int noc_batch_latency_hist(const noc_batch* batch, int i, int which, uint64_t* bins, int nbins);
int64_t noc_batch_kernel_launches(const noc_batch* batch);
/* The build of the batch kernel that runs instance i (kind and way bounds as
 * in noc_last_variant); fixed by the descriptors when the batch is created. */
int noc_batch_variant(const noc_batch* batch, int i, int* kind, int* l1_bound, int* l2_bound);
/* Kernel-variant group of instance i, 0..10 (-1 for a bad argument): 0, 1, 2 =
 * the interleaved build of way class (4, 8), (4, 16), (16, 16); 3 = the base
 * build; 4 = the general build; 5, 6, 7 = the LSPD local-placement build and
 * 8, 9, 10 = the LSPD migration build of those way classes.  Instances of one
 * group and one rectangle side share work-queue launches; the autotuner picks
 * a layout per group. */
int noc_batch_group(const noc_batch* batch, int i);

/* Allocation-free run.  No counterpart in the paper: this entry point serves
 * callers that must not allocate device memory -- a process whose HBM is
 * already reserved by another allocator (a framework's caching allocator), or
 * a host loop that may not allocate, nor take the implicit device
 * synchronisation of cudaMalloc/cudaFree, once running.  It simulates
 * n_cycles from cycle 0 (same arguments and results as noc_create + noc_step
 * + noc_stats) with all simulator state and scratch inside one fixed device
 * array of NOC_STATIC_SCRATCH_BYTES that the library holds on every GPU it is
 * loaded on until the process exits; it calls no allocator.
 *   dev_stats_out: DEVICE memory, one noc_stats_t, written by the run.
 *   cuda_stream:   stream to run on (NULL = default); the call waits for it.
 * Returns NOC_ERR_ARG for any configuration noc_create rejects, for trace
 * mode, or when the state would exceed NOC_STATIC_SCRATCH_BYTES; a simulation
 * error code (e.g. NOC_ERR_QUEUE_OVERFLOW) if the run hit one; NOC_ERR_CUDA
 * when a CUDA call fails.  Every failure sets noc_last_error().
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call reuses the same array and clears it first.  Calls in one process are
 * serialised by an internal lock, and each call returns only after its
 * stream has finished, so they never overlap on the GPU; each process has its
 * own copy of the array.  cuda_stream must belong to the current device. */
#define NOC_STATIC_SCRATCH_BYTES (16u << 20)
int noc_run_static(int mesh_w, int mesh_h, const noc_cache_cfg* cache, int l2_policy,
                   const noc_traffic* traffic, uint64_t seed, int64_t n_cycles,
                   void* dev_stats_out, void* cuda_stream);

/* Number of this library's kernels launched through this handle. */
int64_t noc_kernel_launches(const noc_sim* sim);

/* Which build of the cycle kernel served the handle's last launch.  Results
 * never depend on it; it lets a caller (and the tests) see that a
 * configuration ran on the specialised code it qualifies for.
 *   *loop:  0 = the plain loop (per-warp neighbour waits; noc_step),
 *           1 = the traced / draining loop (hash trace on, or noc_drain),
 *           2 = the plain loop with two tiles per thread (always general);
 *   *kind:  0 = general (every policy, mode and option compiled in),
 *           1 = base (every policy and mode; the packet, write-back,
 *               directory-node and deflection-count-age options compiled out),
 *           2 = interleaved L2 in cache mode only, with exactly the way counts
 *               of its bounds,
 *           3 = the same for the LSPD L2 with local placement (Sec. 3.2),
 *           4 = the same for the LSPD L2 with migration (Sec. 3.3), both
 *               without the directory node (the per-phase profiled build of
 *               these two is the base one);
 *   *l1_bound, *l2_bound: the compile-time way bounds, (4, 8), (4, 16) or
 *           (16, 16).
 * Any output pointer may be NULL.  NOC_ERR_STATE before the first launch. */
int noc_last_variant(const noc_sim* sim, int* loop, int* kind, int* l1_bound, int* l2_bound);
/* The launch bound of that build: the most threads a CTA of it may have.
 * The plain loop is built three times, for CTAs of up to 320, 384 and 448
 * threads; a launch takes the smallest that fits, since more registers per
 * thread run faster (the 448 build keeps 128: a CTA of more than 12 warps puts
 * four warps on some of an SM's four register files of 16,384).  The traced
 * loop and the checked build (noc_set_checks) are built for 448, the per-phase
 * profiled loop for 384 and the two-tile loop for 256.  0 before the first
 * launch, -1 for a null handle. */
int noc_last_launch_bound(const noc_sim* sim);

/* Checked build of the plain loop (one tile per thread).  No counterpart in
 * the paper: a single-writer check.  Every per-tile structure is indexed by
 * the tile's own id; the LSPD directory, indexed by the line a message
 * carries, is the one structure a second writer could reach, and the model
 * lets only a line's directory tile (its home, or the directory node) touch
 * its entry (Sec. 3.2, 3.3).  With enable != 0, later noc_step calls run the
 * general plain loop built with that check in the handlers of the messages
 * that touch the directory (DA, DINV, DIRUPD): a message that reaches another
 * tile, or carries a line outside the address space, ends the step with
 * NOC_ERR_OWNER or NOC_ERR_RANGE at its cycle instead of touching the entry.
 * Results are otherwise those of the production builds.  While checks are on,
 * per-cycle hashes, noc_drain and two tiles per thread are NOC_ERR_ARG and the
 * phase profile is off. */
int noc_set_checks(noc_sim* sim, int enable);

/* Per-phase clock profile of the plain loop (one tile per thread).  With
 * enable != 0 (the first call takes a 48-byte device buffer), later plain
 * launches through this handle run a build of the loop that reads the SM
 * clock at each phase boundary of every warp and cycle; that build keeps its
 * own registers (the 384-thread bound; a tiling with larger CTAs is
 * NOC_ERR_ARG while the profile is on), so it runs somewhat slower than the
 * production build.  noc_phase_profile waits for the handle's stream, writes
 * six sums over warps and cycles -- SM clocks spent waiting for the
 * neighbours' outputs, routing, publishing, in Phase 3, in Phase 1, and the
 * number of warp-cycles -- and clears them.  Results never depend on it; the
 * traced loop and the two-tile loop are not profiled.  Not in the paper (an
 * observability facility). */
int noc_set_phase_profile(noc_sim* sim, int enable);
int noc_phase_profile(noc_sim* sim, uint64_t* out6);

/* Device time of the cycle kernel alone.  With enable != 0, every later
 * cycle-kernel launch through this handle is bracketed by a pair of CUDA
 * events on the handle's stream (reference draws and other helper kernels
 * are left out).  If ms_out or launches_out is non-NULL the call first waits
 * for the recorded launches, writes their summed duration in milliseconds
 * and their number, and forgets them.  Returns NOC_ERR_CUDA if an event call
 * fails. */
int noc_kernel_time(noc_sim* sim, int enable, double* ms_out, int64_t* launches_out);

const char* noc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
