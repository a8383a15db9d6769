/*
 * noc_oracle.c -- the oracle: a plain, serial C simulator of the model.
 *
 * TEST INFRASTRUCTURE ONLY (see noc_oracle.h).  Written for obviousness, not
 * speed: arrays of plain structs, one tile at a time, the paper's three phases
 * in the paper's order (Sec. 7.1 serial listing: Phase1 over all routers, then
 * Phase2 over all routers, then Phase3 over all routers, then SimCycle++).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include "noc_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* message types (Table 1 names where the paper has one)                     */
enum {
  T_NONE = 0,
  T_REQ = 1,    /* RA: remote L2 access, requester -> L2 location         */
  T_DATA = 2,   /* reply carrying the L1 block                            */
  T_WT = 3,     /* L1 write-through (Sec. 3.1: L1s are write-through)     */
  T_DA = 4,     /* directory access (Table 1 DA)                          */
  T_DRPOS = 5,  /* directory reply: owner found (Table 1 DR)              */
  T_DRNEG = 6,  /* directory reply: not on chip (Table 1 DR)              */
  T_NACK = 7,   /* trap reply (Sec. 6.2.1 "Trap")                         */
  T_DINV = 8,   /* victim's directory entry delete (Sec. 3.4)             */
  T_MIG = 9,    /* L2 block migration (Table 1 B2)                        */
  T_DIRUPD = 10,/* directory update on migration arrival (Sec. 3.3)       */
  T_INV = 11,   /* invalidate the source copy after migration (Sec. 3.3)  */
  T_PROBE = 12  /* network-only traffic                                    */
};

enum { FSM_IDLE = 0, FSM_L2WAIT = 1, FSM_STALL = 2 };
enum { OM_NONE = 0, OM_WAIT_DR = 1, OM_WAIT_DATA = 2, OM_MEM_L2 = 3, OM_MEM_L1 = 4 };

#define NO_TILE 0xFFFFu
#define DIR_NONE 0xFFFFFFFFu

enum { PN = 0, PS = 1, PE = 2, PW = 3 };

typedef struct {
  uint32_t type, src, dst, inject, line, a, e;
  uint32_t age; /* deflections so far (age_mode 1; always 0 under age_mode 0) */
} Flit;

typedef struct {
  uint64_t last_use; /* LRU: larger = more recent */
  uint32_t line;
  uint32_t owner;    /* L1: tile whose L2 holds the block (WT target)    */
  uint32_t epoch;    /* L2 (LSPD): epoch of this copy's directory entry  */
  uint8_t valid, dirty;
  uint8_t migrating; /* L2 (migration): a MIG for this copy is in flight  */
  uint8_t hist_n;    /* L2 (migration): accessors recorded in hist       */
  uint32_t* hist;    /* L2 (migration): last mig_window accessors        */
} Way;

typedef struct {
  int sets, ways;
  Way* w;
  uint32_t* hist_store; /* sets*ways*mig_window, migration policy only */
  uint64_t tick;
} Cache;

typedef struct {
  Flit* buf;
  int cap, head, len;
} FlitQ;

typedef struct {
  uint32_t ready, line, req;
} MemEnt;

typedef struct {
  Cache l1, l2;
  FlitQ cq, sq;
  MemEnt* mq;
  int mq_head, mq_len;
  /* core */
  uint32_t next_ref;
  int fsm;
  uint32_t fsm_line, fsm_timer, fsm_start;
  int fsm_write;
  int om_kind;
  uint32_t om_line, om_start, om_timer, om_epoch;
  int om_write;
  uint32_t epoch;
  /* forward table (redirection): newest at index (fwd_next-1) mod cap */
  uint32_t* fwd_line;
  uint32_t* fwd_tile;
  int fwd_n, fwd_next;
  /* trace mode */
  uint32_t* trace;
  int64_t trace_n;
  /* ejected flit handed from Phase 2 to Phase 3 */
  Flit ejected;
  /* reorder buffer (packet mode): packets with some but not all flits here */
  struct {
    uint32_t src, type, line, count;
    int valid;
  } * rob;
  uint64_t st[ORC_NSTAT];
} Tile;

struct orc_sim {
  orc_params p;
  int N;
  uint32_t total_lines;
  Tile* tiles;
  Flit* out_cur;  /* out-links written by the current cycle's Phase 2 */
  Flit* out_prev; /* out-links of the previous cycle (this cycle's arrivals) */
  uint32_t* dir;  /* directory, one entry per line (LSPD policies)        */
  uint64_t hist[2][ORC_HIST_BINS];
  uint32_t cycle;
  int draining;
  int err;
  int64_t err_cycle;
};

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from its published definition (Salmon, Moraes, Dror and    */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds */
/* of two 64x64->128 multiplies; the key is bumped by the Weyl constants     */
/* between rounds.                                                           */
static void mul128(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                       uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul128(M0, x0, &hi0, &lo0);
    mul128(M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* floor(w * n / 2^64): maps a uniform 64-bit word onto [0, n) */
static uint64_t mulhi(uint64_t w, uint64_t n) {
  uint64_t hi, lo;
  mul128(w, n, &hi, &lo);
  return hi;
}

/* splitmix64 finaliser (Steele, Lea, Flood 2014; constants of Vigna's
 * published variant) */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* fold a word list into one 64-bit value */
static uint64_t fold_start(uint64_t w0) { return orc_mix64(w0 + 0x9E3779B97F4A7C15ull); }
static uint64_t fold(uint64_t h, uint64_t w) { return orc_mix64(h ^ w); }

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
static int tile_x(const orc_sim* s, int r) { return r % s->p.mesh_w; }
static int tile_y(const orc_sim* s, int r) { return r / s->p.mesh_w; }

/* neighbour of r through port d, or -1 at the mesh edge */
static int neighbour(const orc_sim* s, int r, int d) {
  int x = tile_x(s, r), y = tile_y(s, r);
  switch (d) {
    case PN: return y > 0 ? r - s->p.mesh_w : -1;
    case PS: return y < s->p.mesh_h - 1 ? r + s->p.mesh_w : -1;
    case PE: return x < s->p.mesh_w - 1 ? r + 1 : -1;
    default: return x > 0 ? r - 1 : -1;
  }
}
static int opposite(int d) { return d ^ 1; }

static uint32_t home_of(const orc_sim* s, uint32_t line) { return line % (uint32_t)s->N; }
/* the tile holding a line's directory entry (LSPD): its home, or the one
 * directory node of the centralized variant */
static uint32_t dir_home(const orc_sim* s, uint32_t line) {
  return s->p.dir_central ? (uint32_t)s->p.dir_tile : home_of(s, line);
}

/* ------------------------------------------------------------------------ */
/* errors: the first cycle with an error wins, smaller code on ties          */
static void set_error(orc_sim* s, int code) {
  int64_t c = (int64_t)s->cycle;
  if (!s->err || c < s->err_cycle || (c == s->err_cycle && code < s->err)) {
    s->err = code;
    s->err_cycle = c;
  }
}

/* ------------------------------------------------------------------------ */
/* caches: set-associative, LRU, victim = lowest-index invalid way, else the */
/* least recently used way                                                   */
static Way* way_at(Cache* c, int set, int way) { return &c->w[(size_t)set * c->ways + way]; }

/* empty a way (keeps its history storage) */
static void way_clear(Way* x) {
  uint32_t* h = x->hist;
  memset(x, 0, sizeof *x);
  x->hist = h;
}

static int cache_find(Cache* c, int set, uint32_t line) {
  for (int w = 0; w < c->ways; w++) {
    Way* x = way_at(c, set, w);
    if (x->valid && x->line == line) return w;
  }
  return -1;
}
static void cache_touch(Cache* c, int set, int way) { way_at(c, set, way)->last_use = ++c->tick; }
static int cache_victim(Cache* c, int set) {
  for (int w = 0; w < c->ways; w++)
    if (!way_at(c, set, w)->valid) return w;
  int best = 0;
  for (int w = 1; w < c->ways; w++)
    if (way_at(c, set, w)->last_use < way_at(c, set, best)->last_use) best = w;
  return best;
}
/* rank 0 = most recently used among the valid ways of the set */
static int cache_rank(Cache* c, int set, int way) {
  int rank = 0;
  uint64_t mine = way_at(c, set, way)->last_use;
  for (int w = 0; w < c->ways; w++) {
    Way* x = way_at(c, set, w);
    if (w != way && x->valid && x->last_use > mine) rank++;
  }
  return rank;
}

static int l1_set(const orc_sim* s, uint32_t line) { return (int)(line % (uint32_t)s->p.l1_sets); }
/* with address interleaving the home consumes the line bits below N, so the
 * set index uses the bits above them */
static int l2_set(const orc_sim* s, uint32_t line) {
  if (s->p.policy == ORC_L2_INTERLEAVED) return (int)((line / (uint32_t)s->N) % (uint32_t)s->p.l2_sets);
  return (int)(line % (uint32_t)s->p.l2_sets);
}

/* ------------------------------------------------------------------------ */
/* queues                                                                    */
static Flit make_flit(uint32_t type, uint32_t src, uint32_t dst, uint32_t line, uint32_t a,
                      uint32_t e) {
  Flit f;
  f.type = type;
  f.src = src;
  f.dst = dst;
  f.inject = 0;
  f.line = line;
  f.a = a;
  f.e = e;
  f.age = 0;
  return f;
}
static int q_full(const FlitQ* q) { return q->len >= q->cap; }
static void q_push(FlitQ* q, Flit f) {
  q->buf[(q->head + q->len) % q->cap] = f;
  q->len++;
}
static Flit q_pop(FlitQ* q) {
  Flit f = q->buf[q->head];
  q->head = (q->head + 1) % q->cap;
  q->len--;
  return f;
}

/* flits of a message: 1, or in packet mode the Table 1 sizes of a data reply
 * (remote L2 access, 4) and of a block migration (16) */
static uint32_t packet_flits(const orc_sim* s, uint32_t type) {
  if (!s->p.packet_mode) return 1;
  if (type == T_DATA) return 4;
  if (type == T_MIG) return 16;
  return 1;
}

/* service-queue messages are never refused: exceeding the capacity is an error */
static void send_svc(orc_sim* s, int r, Flit f) {
  Tile* T = &s->tiles[r];
  if (q_full(&T->sq)) {
    set_error(s, ORC_ERR_QUEUE_OVERFLOW);
    return;
  }
  if (f.type == T_WT) T->st[ORC_ST_WT_SENT]++;
  if (f.type == T_REQ) T->st[ORC_ST_REQ_MADE]++;
  if (f.type == T_DATA || f.type == T_DRPOS || f.type == T_DRNEG || f.type == T_NACK)
    T->st[ORC_ST_REPLY_SENT]++;
  uint32_t n = packet_flits(s, f.type);
  if (n == 1) {
    q_push(&T->sq, f);
    return;
  }
  /* a multi-flit packet: n flits queued together, flit i carries a = i, e = n */
  if (T->sq.cap - T->sq.len < (int)n) {
    set_error(s, ORC_ERR_QUEUE_OVERFLOW);
    return;
  }
  for (uint32_t i = 0; i < n; i++) {
    Flit g = f;
    g.a = i;
    g.e = n;
    q_push(&T->sq, g);
  }
}
/* core-queue messages: caller has checked for space */
static void send_core(orc_sim* s, int r, Flit f) {
  Tile* T = &s->tiles[r];
  if (f.type == T_WT) T->st[ORC_ST_WT_SENT]++;
  if (f.type == T_REQ) T->st[ORC_ST_REQ_MADE]++;
  q_push(&T->cq, f);
}

/* ------------------------------------------------------------------------ */
/* statistics                                                                */
static void hist_add(orc_sim* s, int which, uint64_t v) {
  s->hist[which][v < ORC_HIST_BINS - 1 ? v : ORC_HIST_BINS - 1]++;
}
static void l2lat_sample(orc_sim* s, int r, uint32_t t, uint32_t start) {
  uint64_t lat = (uint64_t)(t - start);
  s->tiles[r].st[ORC_ST_L2LAT_SUM] += lat;
  s->tiles[r].st[ORC_ST_L2LAT_CNT]++;
  hist_add(s, 1, lat);
}

/* ------------------------------------------------------------------------ */
/* directory (LSPD policies): one entry per line, kept at the line's home    */
static uint32_t dir_entry(uint32_t tile, uint32_t epoch) { return tile | (epoch << 16); }

/* victim's directory entry delete (Sec. 3.4): at the home, the entry is
 * cleared only if it still names this copy */
static void send_dinv(orc_sim* s, int r, uint32_t vline, uint32_t vepoch) {
  uint32_t h = dir_home(s, vline);
  if ((int)h == r) {
    if (s->dir[vline] == dir_entry((uint32_t)r, vepoch)) s->dir[vline] = DIR_NONE;
  } else {
    send_svc(s, r, make_flit(T_DINV, (uint32_t)r, h, vline, 0, vepoch));
  }
}

/* ------------------------------------------------------------------------ */
/* cache operations                                                          */

/* install a block in r's L2 slice: insert if absent, else touch (Sec. 3.4) */
static void l2_install(orc_sim* s, int r, uint32_t line, uint32_t epoch) {
  Cache* c = &s->tiles[r].l2;
  int set = l2_set(s, line);
  int w = cache_find(c, set, line);
  if (w < 0) {
    w = cache_victim(c, set);
    Way* x = way_at(c, set, w);
    if (x->valid) {
      if (x->dirty) s->tiles[r].st[ORC_ST_MEM_WB]++;
      if (s->p.policy != ORC_L2_INTERLEAVED) send_dinv(s, r, x->line, x->epoch);
    }
    way_clear(x);
    x->valid = 1;
    x->line = line;
  }
  way_at(c, set, w)->epoch = epoch;
  cache_touch(c, set, w);
}

/* record an access in the block's statistics counter of the last mig_window
 * accessors (Sec. 3.1, Sec. 3.3) */
static void hist_push(orc_sim* s, Way* x, uint32_t who) {
  int cap = s->p.mig_window;
  if (x->hist_n < cap) {
    x->hist[x->hist_n++] = who;
  } else {
    for (int i = 0; i + 1 < cap; i++) x->hist[i] = x->hist[i + 1];
    x->hist[cap - 1] = who;
  }
}

/* write-through performed at r's own L2 slice */
static void local_wt(orc_sim* s, int r, uint32_t line) {
  Cache* c = &s->tiles[r].l2;
  int set = l2_set(s, line);
  int w = cache_find(c, set, line);
  if (w >= 0) {
    way_at(c, set, w)->dirty = 1;
    cache_touch(c, set, w);
    s->tiles[r].st[ORC_ST_WT_HIT]++;
  } else {
    s->tiles[r].st[ORC_ST_MEM_WRITE]++;
  }
}

/* a write of `line` reaching the L2 that holds it: the owner recorded with
 * the L1 copy (this tile's own slice, another tile through a WT message, or
 * memory when no slice holds it) */
static void write_to_owner(orc_sim* s, int r, uint32_t line, uint32_t owner) {
  if (owner == (uint32_t)r)
    local_wt(s, r, line);
  else if (owner == NO_TILE)
    s->tiles[r].st[ORC_ST_MEM_WRITE]++;
  else
    send_svc(s, r, make_flit(T_WT, (uint32_t)r, owner, line, 0, 0));
}

/* fill r's L1 with `line` (insert if absent, else touch); `owner` is the tile
 * whose L2 supplied it.  Write-through: a write is passed on to the owner
 * after the fill and victims are clean.  Write-back: a write dirties the L1
 * copy, and a dirty victim is written to its owner first. */
static void l1_fill(orc_sim* s, int r, uint32_t line, uint32_t owner, int write) {
  Cache* c = &s->tiles[r].l1;
  int set = l1_set(s, line);
  int w = cache_find(c, set, line);
  if (w < 0) {
    w = cache_victim(c, set);
    Way* x = way_at(c, set, w);
    if (s->p.l1_write_back && x->valid && x->dirty) write_to_owner(s, r, x->line, x->owner);
    way_clear(x);
    x->valid = 1;
    x->line = line;
  }
  Way* x = way_at(c, set, w);
  x->owner = owner;
  cache_touch(c, set, w);
  if (write) {
    if (s->p.l1_write_back)
      x->dirty = 1;
    else
      write_to_owner(s, r, line, owner);
  }
}

/* ------------------------------------------------------------------------ */
/* reference stream                                                          */
static void draw_words(const orc_sim* s, uint32_t core, uint32_t k, uint64_t w[4]) {
  uint64_t ctr[4] = {k, core, s->p.stream, 0};
  uint64_t key[2] = {s->p.seed, 0x4E4F43ull};
  orc_philox4x64_10(ctr, key, w);
}

static uint32_t draw_line(const orc_sim* s, uint32_t core, uint32_t k, int* write) {
  uint64_t w[4];
  draw_words(s, core, k, w);
  const orc_params* p = &s->p;
  *write = (uint32_t)(w[0] >> 48) < p->write_q16;
  uint32_t r16 = (uint32_t)(w[1] >> 48);
  uint32_t shared_base = p->remote_lines;
  if (r16 < p->priv_q16) {
    uint32_t base = p->remote_lines + p->shared_lines + core * p->priv_lines;
    return base + (uint32_t)mulhi(w[2], p->priv_lines);
  }
  if (r16 < p->priv_q16 + p->shared_q16) {
    if (p->hot_side > 0 && (uint32_t)(w[3] >> 48) < p->hot_q16) {
      int hs = p->hot_side;
      int x0 = p->mesh_w / 2 - hs / 2, y0 = p->mesh_h / 2 - hs / 2;
      uint32_t j = (uint32_t)mulhi(w[2], (uint64_t)hs * hs);
      uint32_t hj = (uint32_t)((y0 + (int)(j / hs)) * p->mesh_w + x0 + (int)(j % hs));
      uint32_t N = (uint32_t)s->N;
      uint32_t i0 = (hj + N - shared_base % N) % N;
      uint32_t cnt = p->shared_lines > i0 ? (p->shared_lines - i0 + N - 1) / N : 0;
      if (cnt > 0) return shared_base + i0 + (uint32_t)mulhi(w[3] << 16, cnt) * N;
    }
    return shared_base + (uint32_t)mulhi(w[2], p->shared_lines);
  }
  return (uint32_t)mulhi(w[2], p->remote_lines);
}

/* ------------------------------------------------------------------------ */
/* Phase 1 (Sec. 7.1 "Work in phase one"): core side of the memory access    */

/* the L1 lookup of a reference; returns 1 if the action was taken */
static int l1_step(orc_sim* s, int r, uint32_t t, uint32_t line, int write) {
  Tile* T = &s->tiles[r];
  Cache* c = &T->l1;
  int set = l1_set(s, line);
  int w = cache_find(c, set, line);
  if (w >= 0) {
    if (write && s->p.l1_write_back) {
      way_at(c, set, w)->dirty = 1;
    } else if (write) {
      uint32_t owner = way_at(c, set, w)->owner;
      if (owner == (uint32_t)r) {
        local_wt(s, r, line);
      } else if (owner == NO_TILE) {
        T->st[ORC_ST_MEM_WRITE]++;
      } else {
        if (q_full(&T->cq)) {
          T->st[ORC_ST_CQ_STALL]++;
          return 0;
        }
        send_core(s, r, make_flit(T_WT, (uint32_t)r, owner, line, 0, 0));
      }
    }
    cache_touch(c, set, w);
    T->st[ORC_ST_L1_HIT]++;
    T->fsm = FSM_IDLE;
    return 1;
  }
  T->st[ORC_ST_L1_MISS]++;
  T->fsm = FSM_L2WAIT;
  T->fsm_line = line;
  T->fsm_write = write;
  T->fsm_start = t;
  T->fsm_timer = t + (uint32_t)s->p.l1_miss_cycles;
  return 1;
}

static void set_om(Tile* T, int kind, uint32_t line, int write, uint32_t start) {
  T->om_kind = kind;
  T->om_line = line;
  T->om_write = write;
  T->om_start = start;
  T->om_timer = 0;
  T->om_epoch = 0;
}

/* the step taken when the L1 miss wait expires */
static void l2_step(orc_sim* s, int r, uint32_t t) {
  Tile* T = &s->tiles[r];
  uint32_t line = T->fsm_line, start = T->fsm_start;
  int write = T->fsm_write;
  int busy = T->om_kind != OM_NONE;
  Cache* c2 = &T->l2;
  int set2 = l2_set(s, line);

  if (s->p.policy == ORC_L2_INTERLEAVED) {
    uint32_t h = home_of(s, line);
    if (h == (uint32_t)r) {
      int w = cache_find(c2, set2, line);
      if (w >= 0) {
        T->st[ORC_ST_L2_HIT]++;
        cache_touch(c2, set2, w);
        l1_fill(s, r, line, (uint32_t)r, write);
        l2lat_sample(s, r, t, start);
        T->fsm = FSM_IDLE;
        return;
      }
      if (busy) {
        T->st[ORC_ST_MM_STALL]++;
        T->fsm = FSM_STALL;
        return;
      }
      T->st[ORC_ST_L2_MISS]++;
      T->st[ORC_ST_MEM_REQ]++;
      set_om(T, OM_MEM_L2, line, write, start);
      T->om_timer = t + (uint32_t)s->p.mem_latency;
      T->fsm = FSM_IDLE;
      return;
    }
    if (busy) {
      T->st[ORC_ST_MM_STALL]++;
      T->fsm = FSM_STALL;
      return;
    }
    if (q_full(&T->cq)) {
      T->st[ORC_ST_CQ_STALL]++;
      return;
    }
    send_core(s, r, make_flit(T_REQ, (uint32_t)r, h, line, (uint32_t)r, 0));
    set_om(T, OM_WAIT_DATA, line, write, start);
    T->fsm = FSM_IDLE;
    return;
  }

  /* LSPD: the requester's own slice first (local placement, Sec. 3.3) */
  int w = cache_find(c2, set2, line);
  if (w >= 0) {
    T->st[ORC_ST_L2_HIT]++;
    cache_touch(c2, set2, w);
    if (s->p.policy == ORC_L2_LSPD_MIGRATE) hist_push(s, way_at(c2, set2, w), (uint32_t)r);
    l1_fill(s, r, line, (uint32_t)r, write);
    l2lat_sample(s, r, t, start);
    T->fsm = FSM_IDLE;
    return;
  }
  if (busy) {
    T->st[ORC_ST_MM_STALL]++;
    T->fsm = FSM_STALL;
    return;
  }
  uint32_t h = dir_home(s, line);
  if (h == (uint32_t)r) {
    /* the directory entry is at this tile: no flit for the lookup */
    uint32_t D = s->dir[line];
    if (D == DIR_NONE || (D & 0xFFFFu) == (uint32_t)r) {
      T->st[ORC_ST_L2_MISS]++;
      T->st[ORC_ST_DIR_SEARCH]++;
      T->epoch = (T->epoch + 1) & 0xFFFFu;
      s->dir[line] = dir_entry((uint32_t)r, T->epoch);
      set_om(T, OM_MEM_L2, line, write, start);
      T->om_timer = t + (uint32_t)s->p.mem_latency;
      T->om_epoch = T->epoch;
      T->st[ORC_ST_MEM_REQ]++;
      T->fsm = FSM_IDLE;
      return;
    }
    if (q_full(&T->cq)) {
      T->st[ORC_ST_CQ_STALL]++;
      return;
    }
    T->st[ORC_ST_L2_MISS]++;
    T->st[ORC_ST_DIR_SEARCH]++;
    send_core(s, r, make_flit(T_REQ, (uint32_t)r, D & 0xFFFFu, line, (uint32_t)r, 0));
    set_om(T, OM_WAIT_DATA, line, write, start);
    T->fsm = FSM_IDLE;
    return;
  }
  if (q_full(&T->cq)) {
    T->st[ORC_ST_CQ_STALL]++;
    return;
  }
  T->st[ORC_ST_L2_MISS]++;
  T->epoch = (T->epoch + 1) & 0xFFFFu;
  send_core(s, r, make_flit(T_DA, (uint32_t)r, h, line, 0, T->epoch));
  set_om(T, OM_WAIT_DR, line, write, start);
  T->fsm = FSM_IDLE;
}

static void phase1(orc_sim* s, int r, uint32_t t) {
  Tile* T = &s->tiles[r];

  /* (i) memory returns at an interleaved home: install, then reply */
  while (T->mq_len > 0 && T->mq[T->mq_head].ready <= t) {
    MemEnt m = T->mq[T->mq_head];
    T->mq_head = (T->mq_head + 1) % s->p.mem_q;
    T->mq_len--;
    l2_install(s, r, m.line, 0);
    send_svc(s, r, make_flit(T_DATA, (uint32_t)r, m.req, m.line, 0, 0));
  }

  /* (ii) the outstanding memory fetch of this core completes */
  if ((T->om_kind == OM_MEM_L2 || T->om_kind == OM_MEM_L1) && T->om_timer <= t) {
    if (T->om_kind == OM_MEM_L2) {
      l2_install(s, r, T->om_line, T->om_epoch);
      l1_fill(s, r, T->om_line, (uint32_t)r, T->om_write);
    } else {
      l1_fill(s, r, T->om_line, NO_TILE, T->om_write);
    }
    l2lat_sample(s, r, t, T->om_start);
    set_om(T, OM_NONE, 0, 0, 0);
  }

  /* (iii) at most one core action */
  if (T->fsm == FSM_L2WAIT) {
    if (t >= T->fsm_timer) l2_step(s, r, t);
    return;
  }
  if (T->fsm == FSM_STALL) {
    if (T->om_kind == OM_NONE) l1_step(s, r, t, T->fsm_line, T->fsm_write);
    return;
  }
  if (s->draining || s->p.period <= 0) return;
  uint64_t k = T->next_ref;
  if ((uint64_t)t < k * (uint64_t)s->p.period) return;

  if (s->p.mode == ORC_MODE_NETWORK) {
    if (s->N < 2) return;
    if (q_full(&T->cq)) {
      T->st[ORC_ST_CQ_STALL]++;
      return;
    }
    uint64_t w[4];
    draw_words(s, (uint32_t)r, (uint32_t)k, w);
    uint32_t dst = (uint32_t)mulhi(w[1], (uint64_t)(s->N - 1));
    if (dst >= (uint32_t)r) dst++;
    send_core(s, r, make_flit(T_PROBE, (uint32_t)r, dst, 0, 0, 0));
    T->next_ref++;
    T->st[ORC_ST_REFS]++;
    return;
  }

  uint32_t line;
  int write;
  if (s->p.mode == ORC_MODE_TRACE) {
    if ((int64_t)k >= T->trace_n) return;
    line = T->trace[k] & 0x7FFFFFFFu;
    write = (int)(T->trace[k] >> 31);
  } else {
    line = draw_line(s, (uint32_t)r, (uint32_t)k, &write);
  }
  if (l1_step(s, r, t, line, write)) {
    T->next_ref++;
    T->st[ORC_ST_REFS]++;
  }
}

/* ------------------------------------------------------------------------ */
/* Phase 2 (Sec. 4.3, Sec. 7.1 "Work in phase two"): one bufferless router   */

/* priority (Sec. 4.2, 4.3).  age_mode 0: older (smaller inject cycle) first,
 * then smaller source tile.  age_mode 1: the age the paper's flit carries --
 * its count of deflections (Sec. 4.2, 6.2.1, 7.1) -- highest first, ties by
 * the same (inject cycle, source tile) order. */
static int older(const orc_sim* s, const Flit* a, const Flit* b) {
  if (s->p.age_mode && a->age != b->age) return a->age > b->age;
  if (a->inject != b->inject) return a->inject < b->inject;
  return a->src < b->src;
}

static void phase2(orc_sim* s, int r, uint32_t t) {
  Tile* T = &s->tiles[r];
  int x = tile_x(s, r), y = tile_y(s, r);
  Flit arr[5];
  int n = 0, degree = 0, exists[4];
  for (int d = 0; d < 4; d++) {
    int nb = neighbour(s, r, d);
    exists[d] = nb >= 0;
    if (nb < 0) continue;
    degree++;
    Flit f = s->out_prev[(size_t)nb * 4 + opposite(d)];
    if (f.type != T_NONE) arr[n++] = f;
  }
  int n_arrived = n;

  /* eject: the highest-priority arrival addressed to this tile */
  int ej = -1;
  for (int i = 0; i < n; i++)
    if (arr[i].dst == (uint32_t)r && (ej < 0 || older(s, &arr[i], &arr[ej]))) ej = i;
  T->ejected.type = T_NONE;
  if (ej >= 0) {
    T->ejected = arr[ej];
    for (int i = ej; i + 1 < n; i++) arr[i] = arr[i + 1];
    n--;
  }

  /* sort the remaining arrivals oldest first (insertion sort) */
  for (int i = 1; i < n; i++) {
    Flit k = arr[i];
    int j = i - 1;
    while (j >= 0 && older(s, &k, &arr[j])) {
      arr[j + 1] = arr[j];
      j--;
    }
    arr[j + 1] = k;
  }

  /* inject when an input port is free: service queue first, then core queue.
   * The new flit is the youngest, so it is considered last. */
  if (n_arrived < degree) {
    FlitQ* q = T->sq.len > 0 ? &T->sq : (T->cq.len > 0 ? &T->cq : NULL);
    if (q) {
      Flit f = q_pop(q);
      f.inject = t;
      f.src = (uint32_t)r;
      f.age = 0; /* a new flit has age zero (Sec. 7.1) */
      arr[n++] = f;
      T->st[ORC_ST_INJECTED]++;
    }
  }

  /* port selection: each flit in priority order takes the first free port of
   * [X-productive, Y-productive, N, S, E, W] */
  int taken[4] = {0, 0, 0, 0};
  Flit* out = &s->out_cur[(size_t)r * 4];
  memset(out, 0, 4 * sizeof(Flit));
  for (int i = 0; i < n; i++) {
    int dx = (int)(arr[i].dst % (uint32_t)s->p.mesh_w) - x;
    int dy = (int)(arr[i].dst / (uint32_t)s->p.mesh_w) - y;
    int xp = dx > 0 ? PE : (dx < 0 ? PW : -1);
    int yp = dy > 0 ? PS : (dy < 0 ? PN : -1);
    int pref[6] = {xp, yp, PN, PS, PE, PW};
    int port = -1;
    for (int k = 0; k < 6 && port < 0; k++) {
      int p = pref[k];
      if (p >= 0 && exists[p] && !taken[p]) port = p;
    }
    /* a free existing port always remains: arrivals + injected <= degree */
    taken[port] = 1;
    out[port] = arr[i];
    if (port != xp && port != yp) {
      T->st[ORC_ST_DEFLECTIONS]++;
      if (s->p.age_mode) { /* a deflection ages the flit (Sec. 4.2) */
        if (out[port].age == ORC_AGE_MAX) set_error(s, ORC_ERR_RANGE);
        else out[port].age++;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Phase 3 (Sec. 7.1 "Work in phase three"): the ejected flit's handler      */
static void protocol_error(orc_sim* s) { set_error(s, ORC_ERR_PROTOCOL); }

static void phase3(orc_sim* s, int r, uint32_t t) {
  Tile* T = &s->tiles[r];
  Flit f = T->ejected;
  if (f.type == T_NONE) return;
  T->ejected.type = T_NONE;

  uint64_t lat = (uint64_t)(t - f.inject);
  T->st[ORC_ST_EJECTED]++;
  T->st[ORC_ST_LAT_SUM] += lat;
  if (lat > T->st[ORC_ST_LAT_MAX]) T->st[ORC_ST_LAT_MAX] = lat;
  hist_add(s, 0, lat);

  /* packet mode: the handler runs once, when the last flit of a packet is in */
  if (f.e > 1 && packet_flits(s, f.type) > 1) {
    int hit = -1, free_slot = -1;
    for (int i = 0; i < s->p.rob_entries; i++) {
      if (T->rob[i].valid && T->rob[i].src == f.src && T->rob[i].type == f.type &&
          T->rob[i].line == f.line)
        hit = i;
      else if (!T->rob[i].valid && free_slot < 0)
        free_slot = i;
    }
    if (hit < 0) {
      if (free_slot < 0) {
        set_error(s, ORC_ERR_QUEUE_OVERFLOW);
        return;
      }
      hit = free_slot;
      T->rob[hit].valid = 1;
      T->rob[hit].src = f.src;
      T->rob[hit].type = f.type;
      T->rob[hit].line = f.line;
      T->rob[hit].count = 0;
    }
    if (++T->rob[hit].count < f.e) return;
    T->rob[hit].valid = 0;
  }

  Cache* c2 = &T->l2;
  int set2 = l2_set(s, f.line);
  int policy = s->p.policy;
  switch (f.type) {
    case T_PROBE:
      break;

    case T_REQ: {
      uint32_t q = f.a;
      T->st[ORC_ST_REQ_RCVD]++;
      int w = cache_find(c2, set2, f.line);
      if (w >= 0) {
        T->st[ORC_ST_L2_HIT]++;
        cache_touch(c2, set2, w);
        send_svc(s, r, make_flit(T_DATA, (uint32_t)r, q, f.line, 0, 0));
        if (policy == ORC_L2_LSPD_MIGRATE) {
          Way* x = way_at(c2, set2, w);
          hist_push(s, x, q);
          int cnt = 0;
          for (int i = 0; i < x->hist_n; i++) cnt += x->hist[i] == q;
          if (x->hist_n == s->p.mig_window && cnt >= s->p.mig_threshold && !x->migrating) {
            x->migrating = 1;
            T->st[ORC_ST_MIG_SENT]++;
            send_svc(s, r, make_flit(T_MIG, (uint32_t)r, q, f.line, 0, 0));
          }
        }
        break;
      }
      T->st[ORC_ST_L2_MISS]++;
      if (policy == ORC_L2_INTERLEAVED) {
        if (T->mq_len >= s->p.mem_q) {
          set_error(s, ORC_ERR_QUEUE_OVERFLOW);
          break;
        }
        MemEnt* m = &T->mq[(T->mq_head + T->mq_len) % s->p.mem_q];
        m->ready = t + (uint32_t)s->p.mem_latency;
        m->line = f.line;
        m->req = q;
        T->mq_len++;
        T->st[ORC_ST_MEM_REQ]++;
        break;
      }
      if (policy == ORC_L2_LSPD_MIGRATE) {
        /* redirection (Sec. 3.3): newest forward entry for the line */
        int cap = s->p.fwd_entries;
        for (int i = 0; i < T->fwd_n; i++) {
          int slot = ((T->fwd_next - 1 - i) % cap + cap) % cap;
          if (T->fwd_line[slot] == f.line) {
            uint32_t m = T->fwd_tile[slot];
            if (m != q) {
              T->st[ORC_ST_REDIR]++;
              send_svc(s, r, make_flit(T_REQ, (uint32_t)r, m, f.line, q, 0));
              goto req_done;
            }
            break;
          }
        }
      }
      T->st[ORC_ST_TRAP]++;
      send_svc(s, r, make_flit(T_NACK, (uint32_t)r, q, f.line, 0, 0));
    req_done:
      break;
    }

    case T_DATA:
      T->st[ORC_ST_REPLY_RCVD]++;
      if (T->om_kind != OM_WAIT_DATA || T->om_line != f.line) {
        protocol_error(s);
        break;
      }
      l1_fill(s, r, f.line, f.src, T->om_write);
      l2lat_sample(s, r, t, T->om_start);
      set_om(T, OM_NONE, 0, 0, 0);
      break;

    case T_WT: {
      int w = cache_find(c2, set2, f.line);
      if (w >= 0) {
        way_at(c2, set2, w)->dirty = 1;
        cache_touch(c2, set2, w);
        T->st[ORC_ST_WT_HIT]++;
      } else {
        T->st[ORC_ST_MEM_WRITE]++;
      }
      break;
    }

    case T_DA: {
      uint32_t q = f.src;
      uint32_t D = s->dir[f.line];
      T->st[ORC_ST_DIR_SEARCH]++;
      if (D == DIR_NONE || (D & 0xFFFFu) == q) {
        s->dir[f.line] = dir_entry(q, f.e);
        send_svc(s, r, make_flit(T_DRNEG, (uint32_t)r, q, f.line, 0, f.e));
      } else {
        send_svc(s, r, make_flit(T_DRPOS, (uint32_t)r, q, f.line, D & 0xFFFFu, 0));
      }
      break;
    }

    case T_DRNEG:
      T->st[ORC_ST_REPLY_RCVD]++;
      if (T->om_kind != OM_WAIT_DR || T->om_line != f.line) {
        protocol_error(s);
        break;
      }
      T->om_kind = OM_MEM_L2;
      T->om_timer = t + (uint32_t)s->p.mem_latency;
      T->om_epoch = f.e;
      T->st[ORC_ST_MEM_REQ]++;
      break;

    case T_DRPOS:
      T->st[ORC_ST_REPLY_RCVD]++;
      if (T->om_kind != OM_WAIT_DR || T->om_line != f.line) {
        protocol_error(s);
        break;
      }
      send_svc(s, r, make_flit(T_REQ, (uint32_t)r, f.a, f.line, (uint32_t)r, 0));
      T->om_kind = OM_WAIT_DATA;
      break;

    case T_NACK:
      T->st[ORC_ST_REPLY_RCVD]++;
      if (T->om_kind != OM_WAIT_DATA || T->om_line != f.line) {
        protocol_error(s);
        break;
      }
      T->om_kind = OM_MEM_L1;
      T->om_timer = t + (uint32_t)s->p.mem_latency;
      T->st[ORC_ST_MEM_REQ]++;
      break;

    case T_DINV:
      if (s->dir[f.line] == dir_entry(f.src, f.e)) s->dir[f.line] = DIR_NONE;
      break;

    case T_MIG: {
      uint32_t o = f.src;
      T->epoch = (T->epoch + 1) & 0xFFFFu;
      l2_install(s, r, f.line, T->epoch);
      int w = cache_find(c2, set2, f.line);
      Way* x = way_at(c2, set2, w);
      x->hist_n = 0;
      x->migrating = 0;
      uint32_t h = dir_home(s, f.line);
      if (h == (uint32_t)r) {
        /* the directory update happens here: same as a DIRUPD handler */
        s->dir[f.line] = dir_entry((uint32_t)r, T->epoch);
        T->st[ORC_ST_MIGRATIONS]++;
        send_svc(s, r, make_flit(T_INV, (uint32_t)r, o, f.line, (uint32_t)r, 0));
      } else {
        send_svc(s, r, make_flit(T_DIRUPD, (uint32_t)r, h, f.line, o, T->epoch));
      }
      break;
    }

    case T_DIRUPD: {
      uint32_t m = f.src, o = f.a;
      s->dir[f.line] = dir_entry(m, f.e);
      T->st[ORC_ST_MIGRATIONS]++;
      if (o == (uint32_t)r) {
        int w = cache_find(c2, set2, f.line);
        if (w >= 0) {
          Way* x = way_at(c2, set2, w);
          if (x->dirty) T->st[ORC_ST_MEM_WB]++;
          way_clear(x);
        }
        int cap = s->p.fwd_entries;
        T->fwd_line[T->fwd_next] = f.line;
        T->fwd_tile[T->fwd_next] = m;
        T->fwd_next = (T->fwd_next + 1) % cap;
        if (T->fwd_n < cap) T->fwd_n++;
      } else {
        send_svc(s, r, make_flit(T_INV, (uint32_t)r, o, f.line, m, 0));
      }
      break;
    }

    case T_INV: {
      int w = cache_find(c2, set2, f.line);
      if (w >= 0) {
        Way* x = way_at(c2, set2, w);
        if (x->dirty) T->st[ORC_ST_MEM_WB]++;
        way_clear(x);
      }
      int cap = s->p.fwd_entries;
      T->fwd_line[T->fwd_next] = f.line;
      T->fwd_tile[T->fwd_next] = f.a;
      T->fwd_next = (T->fwd_next + 1) % cap;
      if (T->fwd_n < cap) T->fwd_n++;
      break;
    }

    default:
      protocol_error(s);
  }
}

/* ------------------------------------------------------------------------ */
/* hashes                                                                    */
static void flit_words(const Flit* f, uint64_t w[3]) {
  if (f->type == T_NONE) {
    w[0] = w[1] = w[2] = 0;
    return;
  }
  w[0] = (uint64_t)f->type | ((uint64_t)f->src << 16) | ((uint64_t)f->dst << 32) |
         ((uint64_t)f->a << 48);
  w[1] = (uint64_t)f->line | ((uint64_t)f->inject << 32);
  w[2] = (uint64_t)f->e | ((uint64_t)f->age << 32);
}

static uint64_t tile_hash(const orc_sim* s, int r) {
  const Tile* T = &s->tiles[r];
  uint64_t h = fold_start((uint64_t)r);
  for (int d = 0; d < 4; d++) {
    uint64_t w[3];
    flit_words(&s->out_prev[(size_t)r * 4 + d], w);
    h = fold(h, w[0]);
    h = fold(h, w[1]);
    h = fold(h, w[2]);
  }
  int wait = T->fsm == FSM_L2WAIT, busy = T->fsm != FSM_IDLE, om = T->om_kind != OM_NONE;
  int mem = T->om_kind == OM_MEM_L2 || T->om_kind == OM_MEM_L1;
  uint64_t c[10];
  c[0] = T->next_ref;
  c[1] = (uint64_t)T->fsm | ((uint64_t)(busy ? T->fsm_write : 0) << 8) |
         ((uint64_t)T->om_kind << 16) | ((uint64_t)(om ? T->om_write : 0) << 24) |
         ((uint64_t)T->epoch << 32);
  c[2] = (uint64_t)(busy ? T->fsm_line : 0) | ((uint64_t)(wait ? T->fsm_timer : 0) << 32);
  c[3] = (uint64_t)(wait ? T->fsm_start : 0) |
         ((uint64_t)(T->om_kind == OM_MEM_L2 ? T->om_epoch : 0) << 32);
  c[4] = (uint64_t)(om ? T->om_line : 0) | ((uint64_t)(mem ? T->om_timer : 0) << 32);
  c[5] = om ? T->om_start : 0;
  c[6] = (uint64_t)T->cq.len | ((uint64_t)T->sq.len << 16) | ((uint64_t)T->mq_len << 32) |
         ((uint64_t)T->fwd_n << 48);
  c[7] = T->st[ORC_ST_INJECTED];
  c[8] = T->st[ORC_ST_EJECTED];
  c[9] = T->st[ORC_ST_DEFLECTIONS];
  for (int i = 0; i < 10; i++) h = fold(h, c[i]);
  return h;
}

uint64_t orc_dyn_hash(const orc_sim* s) {
  uint64_t H = 0;
  for (int r = 0; r < s->N; r++) {
    H += tile_hash(s, r);
    /* packet mode: one term per partly received packet (none otherwise) */
    const Tile* T = &s->tiles[r];
    for (int i = 0; i < s->p.rob_entries && s->p.packet_mode; i++)
      if (T->rob[i].valid)
        H += fold(fold(fold(fold_start(0x1A), (uint64_t)r),
                       (uint64_t)T->rob[i].line | ((uint64_t)T->rob[i].type << 26)),
                  (uint64_t)T->rob[i].src | ((uint64_t)T->rob[i].count << 16));
  }
  return H;
}

uint64_t orc_state_hash(const orc_sim* s) {
  uint64_t H = orc_dyn_hash(s);
  H += fold(fold_start(0x18), s->cycle);
  for (int r = 0; r < s->N; r++) {
    const Tile* T = &s->tiles[r];
    Cache* c1 = (Cache*)&T->l1;
    for (int set = 0; set < c1->sets; set++)
      for (int w = 0; w < c1->ways; w++) {
        Way* x = way_at(c1, set, w);
        if (!x->valid) continue;
        uint64_t h = fold_start(0x11);
        h = fold(h, (uint64_t)r);
        h = fold(h, (uint64_t)set);
        h = fold(h, (uint64_t)w);
        h = fold(h, (uint64_t)x->line | ((uint64_t)x->dirty << 31));
        h = fold(h, x->owner);
        h = fold(h, (uint64_t)cache_rank(c1, set, w));
        H += h;
      }
    Cache* c2 = (Cache*)&T->l2;
    for (int set = 0; set < c2->sets; set++)
      for (int w = 0; w < c2->ways; w++) {
        Way* x = way_at(c2, set, w);
        if (!x->valid) continue;
        uint64_t h = fold_start(0x12);
        h = fold(h, (uint64_t)r);
        h = fold(h, (uint64_t)set);
        h = fold(h, (uint64_t)w);
        h = fold(h, x->line);
        h = fold(h, (uint64_t)x->dirty);
        h = fold(h, (uint64_t)cache_rank(c2, set, w));
        h = fold(h, x->epoch);
        h = fold(h, (uint64_t)x->migrating);
        h = fold(h, (uint64_t)x->hist_n);
        for (int i = 0; i < x->hist_n; i++) h = fold(h, x->hist[i]);
        H += h;
      }
    const FlitQ* qs[2] = {&T->cq, &T->sq};
    for (int qi = 0; qi < 2; qi++)
      for (int i = 0; i < qs[qi]->len; i++) {
        uint64_t w[3];
        flit_words(&qs[qi]->buf[(qs[qi]->head + i) % qs[qi]->cap], w);
        uint64_t h = fold_start(0x13 + (uint64_t)qi);
        h = fold(h, (uint64_t)r);
        h = fold(h, (uint64_t)i);
        h = fold(h, w[0]);
        h = fold(h, w[1]);
        h = fold(h, w[2]);
        H += h;
      }
    for (int i = 0; i < T->mq_len; i++) {
      const MemEnt* m = &T->mq[(T->mq_head + i) % s->p.mem_q];
      uint64_t h = fold_start(0x15);
      h = fold(h, (uint64_t)r);
      h = fold(h, (uint64_t)i);
      h = fold(h, m->ready);
      h = fold(h, m->line);
      h = fold(h, m->req);
      H += h;
    }
    int cap = s->p.fwd_entries;
    for (int i = 0; i < T->fwd_n; i++) {
      int slot = ((T->fwd_next - 1 - i) % cap + cap) % cap;
      uint64_t h = fold_start(0x17);
      h = fold(h, (uint64_t)r);
      h = fold(h, (uint64_t)i);
      h = fold(h, T->fwd_line[slot]);
      h = fold(h, T->fwd_tile[slot]);
      H += h;
    }
  }
  if (s->dir)
    for (uint32_t line = 0; line < s->total_lines; line++) {
      uint32_t D = s->dir[line];
      if (D == DIR_NONE) continue;
      uint64_t h = fold_start(0x16);
      h = fold(h, line);
      h = fold(h, D & 0xFFFFu);
      h = fold(h, D >> 16);
      H += h;
    }
  return H;
}

/* ------------------------------------------------------------------------ */
/* lifecycle                                                                 */
static int check_params(const orc_params* p) {
  if (p->mesh_w < 1 || p->mesh_h < 1 || (int64_t)p->mesh_w * p->mesh_h > 65535) return 0;
  if (p->policy < 0 || p->policy > 2) return 0;
  if (p->l1_sets < 1 || p->l1_ways < 1 || p->l1_ways > 16) return 0;
  if (p->l2_sets < 1 || p->l2_ways < 1 || p->l2_ways > 16) return 0;
  if (p->l1_miss_cycles < 0 || p->mem_latency < 1) return 0;
  if (p->core_q < 1 || p->svc_q < 1 || p->mem_q < 1) return 0;
  if (p->policy == ORC_L2_LSPD_MIGRATE &&
      (p->mig_window < 1 || p->mig_window > 30 || p->mig_threshold < 1 || p->fwd_entries < 1))
    return 0;
  if (p->mode < 0 || p->mode > 2 || p->period < 0) return 0;
  if (p->write_q16 > 65536 || p->priv_q16 + p->shared_q16 > 65536 || p->hot_q16 > 65536) return 0;
  if (p->mode == ORC_MODE_CACHE) {
    if (p->priv_q16 > 0 && p->priv_lines < 1) return 0;
    if (p->shared_q16 > 0 && p->shared_lines < 1) return 0;
    if (p->priv_q16 + p->shared_q16 < 65536 && p->remote_lines < 1) return 0;
  }
  if (p->hot_side < 0 || p->hot_side > p->mesh_w || p->hot_side > p->mesh_h) return 0;
  uint64_t total = (uint64_t)p->remote_lines + p->shared_lines +
                   (uint64_t)p->priv_lines * (uint64_t)p->mesh_w * p->mesh_h;
  if (total >= (1ull << 26)) return 0;
  if (p->packet_mode < 0 || p->packet_mode > 1) return 0;
  if (p->packet_mode && (p->rob_entries < 1 || p->rob_entries > 64 || p->svc_q < 16)) return 0;
  if (p->dir_central < 0 || p->dir_central > 1) return 0;
  if (p->l1_write_back < 0 || p->l1_write_back > 1) return 0;
  if (p->age_mode < 0 || p->age_mode > 1) return 0;
  if (p->dir_central && (p->dir_tile < 0 || p->dir_tile >= p->mesh_w * p->mesh_h)) return 0;
  return 1;
}

int orc_create(const orc_params* p, orc_sim** out) {
  if (!p || !out || !check_params(p)) return ORC_ERR_ARG;
  orc_sim* s = (orc_sim*)calloc(1, sizeof *s);
  if (!s) return ORC_ERR_OOM;
  s->p = *p;
  if (s->p.fwd_entries < 1) s->p.fwd_entries = 1;
  s->N = p->mesh_w * p->mesh_h;
  s->total_lines = p->remote_lines + p->shared_lines + p->priv_lines * (uint32_t)s->N;
  s->tiles = (Tile*)calloc((size_t)s->N, sizeof(Tile));
  s->out_cur = (Flit*)calloc((size_t)s->N * 4, sizeof(Flit));
  s->out_prev = (Flit*)calloc((size_t)s->N * 4, sizeof(Flit));
  if (!s->tiles || !s->out_cur || !s->out_prev) goto oom;
  if (p->policy != ORC_L2_INTERLEAVED) {
    s->dir = (uint32_t*)malloc((size_t)s->total_lines * sizeof(uint32_t));
    if (!s->dir) goto oom;
    for (uint32_t i = 0; i < s->total_lines; i++) s->dir[i] = DIR_NONE;
  }
  for (int r = 0; r < s->N; r++) {
    Tile* T = &s->tiles[r];
    T->l1.sets = p->l1_sets;
    T->l1.ways = p->l1_ways;
    T->l1.w = (Way*)calloc((size_t)p->l1_sets * p->l1_ways, sizeof(Way));
    T->l2.sets = p->l2_sets;
    T->l2.ways = p->l2_ways;
    T->l2.w = (Way*)calloc((size_t)p->l2_sets * p->l2_ways, sizeof(Way));
    if (T->l2.w && p->policy == ORC_L2_LSPD_MIGRATE) {
      size_t nw = (size_t)p->l2_sets * p->l2_ways;
      T->l2.hist_store = (uint32_t*)calloc(nw * (size_t)p->mig_window, sizeof(uint32_t));
      if (!T->l2.hist_store) goto oom;
      for (size_t i = 0; i < nw; i++) T->l2.w[i].hist = T->l2.hist_store + i * (size_t)p->mig_window;
    }
    T->cq.cap = p->core_q;
    T->cq.buf = (Flit*)calloc((size_t)p->core_q, sizeof(Flit));
    T->sq.cap = p->svc_q;
    T->sq.buf = (Flit*)calloc((size_t)p->svc_q, sizeof(Flit));
    T->mq = (MemEnt*)calloc((size_t)p->mem_q, sizeof(MemEnt));
    T->fwd_line = (uint32_t*)calloc((size_t)s->p.fwd_entries, sizeof(uint32_t));
    T->fwd_tile = (uint32_t*)calloc((size_t)s->p.fwd_entries, sizeof(uint32_t));
    if (!T->l1.w || !T->l2.w || !T->cq.buf || !T->sq.buf || !T->mq || !T->fwd_line ||
        !T->fwd_tile)
      goto oom;
    if (p->packet_mode) {
      T->rob = calloc((size_t)p->rob_entries, sizeof *T->rob);
      if (!T->rob) goto oom;
    }
  }
  *out = s;
  return ORC_OK;
oom:
  orc_destroy(s);
  return ORC_ERR_OOM;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  if (s->tiles)
    for (int r = 0; r < s->N; r++) {
      Tile* T = &s->tiles[r];
      free(T->l1.w);
      free(T->l2.w);
      free(T->l2.hist_store);
      free(T->cq.buf);
      free(T->sq.buf);
      free(T->mq);
      free(T->fwd_line);
      free(T->fwd_tile);
      free(T->rob);
      free(T->trace);
    }
  free(s->tiles);
  free(s->out_cur);
  free(s->out_prev);
  free(s->dir);
  free(s);
}

/* one simulated cycle: the three phases over all tiles, in order */
static void one_cycle(orc_sim* s) {
  uint32_t t = s->cycle;
  for (int r = 0; r < s->N; r++) phase1(s, r, t);
  for (int r = 0; r < s->N; r++) phase2(s, r, t);
  for (int r = 0; r < s->N; r++) phase3(s, r, t);
  Flit* tmp = s->out_prev;
  s->out_prev = s->out_cur;
  s->out_cur = tmp;
  s->cycle++;
}

int orc_step(orc_sim* s, int64_t n, uint64_t* trace) {
  if (!s || n < 0) return ORC_ERR_ARG;
  if (s->err) return s->err;
  if (s->p.age_mode && (int64_t)s->cycle + n > ORC_AGE_CYCLES) return ORC_ERR_ARG;
  for (int64_t i = 0; i < n; i++) {
    one_cycle(s);
    if (trace) trace[i] = orc_dyn_hash(s);
    if (s->err) return s->err;
  }
  return ORC_OK;
}

static int quiescent(const orc_sim* s) {
  for (int r = 0; r < s->N; r++) {
    const Tile* T = &s->tiles[r];
    if (T->cq.len || T->sq.len || T->mq_len || T->fsm != FSM_IDLE || T->om_kind != OM_NONE)
      return 0;
    for (int i = 0; i < s->p.rob_entries && s->p.packet_mode; i++)
      if (T->rob[i].valid) return 0;
  }
  /* flits are counted at the injecting and at the ejecting tile */
  uint64_t inj = 0, ej = 0;
  for (int r = 0; r < s->N; r++) {
    inj += s->tiles[r].st[ORC_ST_INJECTED];
    ej += s->tiles[r].st[ORC_ST_EJECTED];
  }
  return inj == ej;
}

int orc_drain(orc_sim* s, int64_t max_cycles, int64_t* taken) {
  if (!s || max_cycles < 0) return ORC_ERR_ARG;
  if (s->err) return s->err;
  if (s->p.age_mode && (int64_t)s->cycle + max_cycles > ORC_AGE_CYCLES) return ORC_ERR_ARG;
  s->draining = 1;
  int64_t i = 0;
  while (!quiescent(s) && i < max_cycles) {
    one_cycle(s);
    i++;
    if (s->err) break;
  }
  if (taken) *taken = i;
  if (s->err) return s->err;
  return quiescent(s) ? ORC_OK : ORC_ERR_TIMEOUT;
}

int64_t orc_cycle(const orc_sim* s) { return s ? (int64_t)s->cycle : -1; }

int orc_error(const orc_sim* s, int64_t* err_cycle) {
  if (!s) return ORC_ERR_ARG;
  if (err_cycle) *err_cycle = s->err ? s->err_cycle : -1;
  return s->err;
}

int orc_stats(const orc_sim* s, int tile, uint64_t* out) {
  if (!s || !out || tile >= s->N) return ORC_ERR_ARG;
  for (int i = 0; i < ORC_NSTAT; i++) out[i] = 0;
  for (int r = 0; r < s->N; r++) {
    if (tile >= 0 && r != tile) continue;
    for (int i = 0; i < ORC_NSTAT; i++) {
      if (i == ORC_ST_LAT_MAX) {
        if (s->tiles[r].st[i] > out[i]) out[i] = s->tiles[r].st[i];
      } else {
        out[i] += s->tiles[r].st[i];
      }
    }
  }
  return ORC_OK;
}

int orc_hist(const orc_sim* s, int which, uint64_t* bins) {
  if (!s || !bins || which < 0 || which > 1) return ORC_ERR_ARG;
  memcpy(bins, s->hist[which], sizeof s->hist[which]);
  return ORC_OK;
}

int orc_set_trace(orc_sim* s, int core, int64_t n, const uint32_t* refs) {
  if (!s || core < 0 || core >= s->N || n < 0 || (n > 0 && !refs)) return ORC_ERR_ARG;
  Tile* T = &s->tiles[core];
  free(T->trace);
  T->trace = NULL;
  T->trace_n = 0;
  if (n == 0) return ORC_OK;
  T->trace = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  if (!T->trace) return ORC_ERR_OOM;
  for (int64_t i = 0; i < n; i++) {
    if ((refs[i] & 0x7FFFFFFFu) >= s->total_lines) return ORC_ERR_ARG;
    T->trace[i] = refs[i];
  }
  T->trace_n = n;
  return ORC_OK;
}

static Flit flit_from8(const uint32_t* w) {
  Flit f;
  f.type = w[0];
  f.src = w[1];
  f.dst = w[2];
  f.inject = w[3];
  f.line = w[4];
  f.a = w[5];
  f.e = w[6];
  f.age = w[7];
  return f;
}

int orc_debug_enqueue(orc_sim* s, int tile, int queue, const uint32_t* flit8) {
  if (!s || !flit8 || tile < 0 || tile >= s->N || queue < 0 || queue > 1) return ORC_ERR_ARG;
  Flit f = flit_from8(flit8);
  f.age = 0;
  if (f.type == T_NONE || f.type > T_PROBE || f.dst >= (uint32_t)s->N || f.dst == (uint32_t)tile)
    return ORC_ERR_ARG;
  f.src = (uint32_t)tile;
  FlitQ* q = queue == 0 ? &s->tiles[tile].cq : &s->tiles[tile].sq;
  if (q_full(q)) return ORC_ERR_QUEUE_OVERFLOW;
  q_push(q, f);
  return ORC_OK;
}

int orc_debug_link(orc_sim* s, int tile, int dir, const uint32_t* flit8) {
  if (!s || !flit8 || tile < 0 || tile >= s->N || dir < 0 || dir > 3) return ORC_ERR_ARG;
  int nb = neighbour(s, tile, dir);
  if (nb < 0) return ORC_ERR_ARG;
  Flit f = flit_from8(flit8);
  if (f.type == T_NONE || f.type > T_PROBE || f.dst >= (uint32_t)s->N) return ORC_ERR_ARG;
  if (f.age && !s->p.age_mode) return ORC_ERR_ARG;
  /* counted as injected so that conservation holds */
  s->tiles[f.src < (uint32_t)s->N ? f.src : (uint32_t)nb].st[ORC_ST_INJECTED]++;
  s->out_prev[(size_t)nb * 4 + opposite(dir)] = f;
  return ORC_OK;
}

int orc_get_links(const orc_sim* s, uint32_t* out) {
  if (!s || !out) return ORC_ERR_ARG;
  for (int i = 0; i < s->N * 4; i++) {
    const Flit* f = &s->out_prev[i];
    uint32_t* o = &out[(size_t)i * 8];
    o[0] = f->type;
    o[1] = f->type ? f->src : 0;
    o[2] = f->type ? f->dst : 0;
    o[3] = f->type ? f->inject : 0;
    o[4] = f->type ? f->line : 0;
    o[5] = f->type ? f->a : 0;
    o[6] = f->type ? f->e : 0;
    o[7] = f->type ? f->age : 0;
  }
  return ORC_OK;
}

int orc_get_cache(const orc_sim* s, int tile, int which, uint32_t* out) {
  if (!s || !out || tile < 0 || tile >= s->N || which < 1 || which > 2) return ORC_ERR_ARG;
  Cache* c = which == 1 ? (Cache*)&s->tiles[tile].l1 : (Cache*)&s->tiles[tile].l2;
  for (int set = 0; set < c->sets; set++)
    for (int w = 0; w < c->ways; w++) {
      Way* x = way_at(c, set, w);
      uint32_t* o = &out[((size_t)set * c->ways + w) * 4];
      o[0] = (uint32_t)x->valid;
      o[1] = x->valid ? x->line : 0;
      o[2] = !x->valid ? 0 : (which == 1 ? x->owner : ((uint32_t)x->dirty | (x->epoch << 16)));
      o[3] = x->valid ? (uint32_t)cache_rank(c, set, w) : 0;
    }
  return ORC_OK;
}

uint32_t orc_dir_get(const orc_sim* s, uint32_t line) {
  if (!s || !s->dir || line >= s->total_lines) return DIR_NONE;
  return s->dir[line];
}

int orc_get_core(const orc_sim* s, int tile, uint32_t* o) {
  if (!s || !o || tile < 0 || tile >= s->N) return ORC_ERR_ARG;
  const Tile* T = &s->tiles[tile];
  o[0] = T->next_ref;
  o[1] = (uint32_t)T->fsm;
  o[2] = T->fsm_line;
  o[3] = (uint32_t)T->fsm_write;
  o[4] = T->fsm_timer;
  o[5] = T->fsm_start;
  o[6] = (uint32_t)T->om_kind;
  o[7] = T->om_line;
  o[8] = (uint32_t)T->om_write;
  o[9] = T->om_start;
  o[10] = T->om_timer;
  o[11] = T->om_epoch;
  o[12] = T->epoch;
  o[13] = (uint32_t)T->cq.len;
  o[14] = (uint32_t)T->sq.len;
  o[15] = (uint32_t)T->mq_len;
  o[16] = (uint32_t)T->fwd_n;
  return ORC_OK;
}

int orc_draw_ref(const orc_sim* s, int core, uint32_t k, uint32_t* line, int* write) {
  if (!s || !line || !write || core < 0 || core >= s->N) return ORC_ERR_ARG;
  *line = draw_line(s, (uint32_t)core, k, write);
  return ORC_OK;
}
