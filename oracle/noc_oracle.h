/*
 * noc_oracle.h -- serial reference simulator (the oracle).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it.  It shares no code, header, table or
 * constant generator with the CUDA path; the two meet only through the seeded
 * input parameters (paper_1508_03235_b300/inputs.py) and the written model.
 *
 * The oracle is the paper's serial "golden model" (Sec. 6.1, Sec. 7.1): every
 * cycle it runs Phase 1 (core / L1 / L2 slice / directory work, Sec. 7.1 "Work
 * in phase one") for every tile, then Phase 2 (bufferless deflection routing,
 * "Work in phase two", Sec. 4.3) for every router, then Phase 3 (link transfer,
 * ejection handling, "Work in phase three") for every tile, in that order.
 */
#ifndef NOC_ORACLE_H
#define NOC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (numerically identical to the product library's by spec) */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_QUEUE_OVERFLOW 3
#define ORC_ERR_TIMEOUT 4
#define ORC_ERR_CUDA 5
#define ORC_ERR_PROTOCOL 6
#define ORC_ERR_STATE 7
#define ORC_ERR_RANGE 8 /* age_mode 1: a flit deflected with age ORC_AGE_MAX */

/* age_mode 1 limits: a flit's age counts at most ORC_AGE_MAX deflections, and
 * a run (steps and drains) ends at or before cycle ORC_AGE_CYCLES */
#define ORC_AGE_MAX 4095u
#define ORC_AGE_CYCLES (1ll << 20)

/* L2 placement policies (Sec. 3) */
#define ORC_L2_INTERLEAVED 0   /* home = line mod N holds the only L2 copy      */
#define ORC_L2_LSPD_LOCAL 1    /* LSPD: local placement + home-tile directory   */
#define ORC_L2_LSPD_MIGRATE 2  /* LSPD + migration and redirection (Sec. 3.3)   */

/* traffic modes */
#define ORC_MODE_CACHE 0   /* Philox reference stream through L1/L2/directory */
#define ORC_MODE_NETWORK 1 /* network only: uniform random dst != src probes  */
#define ORC_MODE_TRACE 2   /* explicit per-core reference lists               */

typedef struct {
  int32_t mesh_w, mesh_h, policy;
  int32_t l1_sets, l1_ways, l2_sets, l2_ways;
  int32_t l1_miss_cycles, mem_latency, mig_window, mig_threshold;
  int32_t core_q, svc_q, mem_q, fwd_entries;
  int32_t mode, period;
  uint32_t write_q16, priv_q16, shared_q16, hot_q16;
  int32_t hot_side;
  uint32_t priv_lines, shared_lines, remote_lines;
  uint64_t seed;
  uint32_t stream;
  /* packets (Table 1, Sec. 2.3): 0 = every message is one flit; 1 = a DATA
   * reply (remote L2 access, RA) is 4 flits and a migration (B2) 16 flits,
   * reassembled in a per-tile reorder buffer of rob_entries packets */
  int32_t packet_mode, rob_entries;
  /* directory placement (LSPD policies, Sec. 3.2): 0 = each line's entry at
   * its home tile; 1 = every entry at one directory node, tile dir_tile */
  int32_t dir_central, dir_tile;
  /* L1 write policy: 0 = write-through (Sec. 3.1, 3.2); 1 = write-back, a dirty
   * victim written back to the L2 that supplied it (Sec. 3.4, 7.1) */
  int32_t l1_write_back;
  /* router priority: 0 = oldest first (inject cycle, then source tile);
   * 1 = most deflections first (the paper's age field), then the same order */
  int32_t age_mode;
} orc_params;

/* statistic indices (order fixed by the written model) */
enum {
  ORC_ST_INJECTED = 0, ORC_ST_EJECTED, ORC_ST_DEFLECTIONS, ORC_ST_LAT_SUM,
  ORC_ST_LAT_MAX, ORC_ST_REFS, ORC_ST_L1_HIT, ORC_ST_L1_MISS, ORC_ST_L2_HIT,
  ORC_ST_L2_MISS, ORC_ST_REQ_MADE, ORC_ST_REQ_RCVD, ORC_ST_REPLY_SENT,
  ORC_ST_REPLY_RCVD, ORC_ST_DIR_SEARCH, ORC_ST_MEM_REQ, ORC_ST_MEM_WRITE,
  ORC_ST_MEM_WB, ORC_ST_WT_SENT, ORC_ST_WT_HIT, ORC_ST_TRAP, ORC_ST_REDIR,
  ORC_ST_MIGRATIONS, ORC_ST_L2LAT_SUM, ORC_ST_L2LAT_CNT, ORC_ST_CQ_STALL,
  ORC_ST_MM_STALL, ORC_ST_MIG_SENT,
  ORC_NSTAT
};
#define ORC_HIST_BINS 1025

typedef struct orc_sim orc_sim;

int orc_create(const orc_params* p, orc_sim** out);
void orc_destroy(orc_sim* s);
/* run n cycles; if trace != NULL, trace[i] = dynamic-state hash after cycle i */
int orc_step(orc_sim* s, int64_t n, uint64_t* trace);
/* stop issuing references; run until quiescent or max_cycles; *taken = cycles run */
int orc_drain(orc_sim* s, int64_t max_cycles, int64_t* taken);
int64_t orc_cycle(const orc_sim* s);
int orc_error(const orc_sim* s, int64_t* err_cycle);
/* totals over tiles (tile < 0) or one tile's counters; out has ORC_NSTAT slots */
int orc_stats(const orc_sim* s, int tile, uint64_t* out);
/* which: 0 = flit latency, 1 = L2 access latency; bins has ORC_HIST_BINS slots */
int orc_hist(const orc_sim* s, int which, uint64_t* bins);
uint64_t orc_dyn_hash(const orc_sim* s);
uint64_t orc_state_hash(const orc_sim* s);

/* trace mode: per-core reference lists, ref = line | write << 31 */
int orc_set_trace(orc_sim* s, int core, int64_t n, const uint32_t* refs);

/* flits as 8 words: type, src, dst, inject_cycle, line, a, e, age (the
 * deflection count of age_mode 1; an enqueued flit's age is ignored) */
int orc_debug_enqueue(orc_sim* s, int tile, int queue /*0 core, 1 service*/,
                      const uint32_t* flit8);
/* place a flit so that it arrives at `tile` from direction dir (0 N,1 S,2 E,3 W)
 * in the next cycle; a non-zero age needs age_mode 1 */
int orc_debug_link(orc_sim* s, int tile, int dir, const uint32_t* flit8);
/* out-links written in the last cycle: N*4 flits of 8 words */
int orc_get_links(const orc_sim* s, uint32_t* out);
/* cache contents of one tile: per (set, way) 4 words: valid, line, aux, rank;
 * aux = owner for L1, dirty | epoch << 16 for L2 */
int orc_get_cache(const orc_sim* s, int tile, int which /*1 = L1, 2 = L2*/,
                  uint32_t* out);
/* directory entry of a line: 0xFFFFFFFF = none, else tile | epoch << 16 */
uint32_t orc_dir_get(const orc_sim* s, uint32_t line);
/* core words: next_ref, fsm, fsm_line, fsm_write, fsm_timer, fsm_start,
 * om_kind, om_line, om_write, om_start, om_timer, om_epoch, epoch,
 * cq_len, sq_len, mq_len, fwd_n */
int orc_get_core(const orc_sim* s, int tile, uint32_t* out17);
/* reference generator exposed for tests: (line, write) of ref k of core c */
int orc_draw_ref(const orc_sim* s, int core, uint32_t k, uint32_t* line,
                 int* write);
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                       uint64_t out[4]);
uint64_t orc_mix64(uint64_t z);

#ifdef __cplusplus
}
#endif
#endif
