// noc_model.cuh -- device-side model of one tile of the simulated multicore.
//
// One CUDA thread owns one tile for a whole launch and keeps its core state,
// queue heads and counters in registers; caches, queues and the directory stay
// in HBM.  The three phases of the paper's cycle (Sec. 7.1) are the functions
// phase1 / route / phase3 below; the persistent kernel in noc_kernel.cu calls
// them in the order P2(t) -> P3(t) -> P1(t+1) so that the cache work of a tile
// overlaps the wait for its neighbours' outputs.
#pragma once
#include <cstdint>

namespace noc {

// A translation unit compiled with -DNOC_FIXED_POLICY=<p> -DNOC_FIXED_MODE=<m>
// builds the device code for that L2 policy and traffic mode alone (the other
// paths are compiled out); otherwise both are read from the parameters.
// With -DNOC_BASE every policy and mode stays, but the options beyond the
// paper's workloads (multi-flit packets, L1 write-back, the centralized
// directory node, the deflection-count age) are compiled out.  With -DNOC_EXACT_WAYS the cache-set code
// takes the way counts to be exactly the translation unit's compile-time
// bounds NOC_W1 and NOC_W2.
#if defined(NOC_EXACT_WAYS)
#define L1WAYS(P) (NOC_W1)
#define L2WAYS(P) (NOC_W2)
#else
#define L1WAYS(P) ((P).l1_ways)
#define L2WAYS(P) ((P).l2_ways)
#endif
#if defined(NOC_FIXED_POLICY) && defined(NOC_FIXED_MODE)
#define POLICY(P) (NOC_FIXED_POLICY)
#define MODE(P) (NOC_FIXED_MODE)
#define NOC_WITH_LSPD (NOC_FIXED_POLICY != 0)
#define NOC_EXTENSIONS 0
#else
#define POLICY(P) ((P).policy)
#define MODE(P) ((P).mode)
#define NOC_WITH_LSPD 1
#if defined(NOC_BASE)
#define NOC_EXTENSIONS 0
#else
#define NOC_EXTENSIONS 1
#endif
#endif
#if NOC_EXTENSIONS
#define PACKETS(P) ((P).packet_mode)
#define L1WB(P) ((P).l1_write_back)
#define DIRC(P) ((P).dir_central)
#define AGE1(P) ((P).age_mode)
#else
#define PACKETS(P) 0
#define L1WB(P) 0
#define DIRC(P) 0
#define AGE1(P) 0
#endif

// ---------------------------------------------------------------- constants
enum : uint32_t {
  T_NONE = 0, T_REQ = 1, T_DATA = 2, T_WT = 3, T_DA = 4, T_DRPOS = 5, T_DRNEG = 6,
  T_NACK = 7, T_DINV = 8, T_MIG = 9, T_DIRUPD = 10, T_INV = 11, T_PROBE = 12
};
enum : uint32_t { FSM_IDLE = 0, FSM_L2WAIT = 1, FSM_STALL = 2 };
enum : uint32_t { OM_NONE = 0, OM_WAIT_DR = 1, OM_WAIT_DATA = 2, OM_MEM_L2 = 3, OM_MEM_L1 = 4 };
enum : int { P_N = 0, P_S = 1, P_E = 2, P_W = 3 };
enum : int { POL_INTERLEAVED = 0, POL_LOCAL = 1, POL_MIGRATE = 2 };
enum : int { MODE_CACHE = 0, MODE_NETWORK = 1, MODE_TRACE = 2 };
enum : int { ERR_OVERFLOW = 3, ERR_TIMEOUT = 4, ERR_PROTOCOL = 6, ERR_RANGE = 8, ERR_OWNER = 9 };

constexpr uint32_t NO_TILE = 0xFFFFu;
constexpr uint32_t DIR_NONE = 0xFFFFFFFFu;
constexpr int HIST_BINS = 1025;
constexpr int MAX_WAYS = 16;  // most ways a cache may have
constexpr int HIST_MAX = 30;  // longest access history kept per L2 way
// u16 words per L2 way in the history array: [n, migrating, who x mig_window]
inline int hist_stride(int mig_window) { return (mig_window + 3) & ~1; }

// cache way word: bit31 valid | bits27-30 LRU rank | bit26 dirty | bits0-25 line
constexpr uint32_t W_VALID = 1u << 31;
constexpr uint32_t W_DIRTY = 1u << 26;
constexpr uint32_t W_LINE = (1u << 26) - 1;
constexpr int W_RANK_SHIFT = 27;

// counters kept per tile (order = the model's statistics list)
enum : int {
  S_INJ = 0, S_EJ, S_DEFL, S_LATSUM, S_LATMAX, S_REFS, S_L1H, S_L1M, S_L2H, S_L2M,
  S_REQM, S_REQR, S_REPS, S_REPR, S_DIRS, S_MEMREQ, S_MEMW, S_MEMWB, S_WTS, S_WTH,
  S_TRAP, S_REDIR, S_MIGR, S_L2LSUM, S_L2LCNT, S_CQST, S_MMST, S_MIGS, NSTAT
};
// counters from S_REFS on are 32-bit per-launch deltas in registers (the
// L2-latency sum is kept separately as 64 bits)
constexpr int NSMALL = NSTAT - S_REFS;

// core-state SoA fields ([field][tile] u32), saved between launches
enum : int {
  C_NEXT = 0, C_FSMB, C_FLINE, C_FTIMER, C_FSTART, C_OLINE, C_OSTART, C_OTIMER, C_EPOCH,
  C_CQ, C_SQ, C_MQ, C_FWD, NCORE
};

// ---------------------------------------------------------------- parameters
struct Params {
  int W, H, N, policy, mode, period;
  int l1_sets, l1_ways, l2_sets, l2_ways;
  int l1_miss, mem_lat, mig_window, mig_threshold, hist_stride;
  int core_q, svc_q, mem_q, fwd_cap;
  int packet_mode, rob_entries;  // Table 1 packets; reorder-buffer entries per tile
  int dir_central, dir_tile;     // directory entries at each line's home, or all at dir_tile
  int l1_write_back;             // 0: write-through L1; 1: write-back L1
  int age_mode;                  // 0: oldest first; 1: most deflections first
  uint32_t write_q16, priv_q16, shared_q16, hot_q16;
  int hot_side, hot_x0, hot_y0;
  uint32_t priv_lines, shared_lines, remote_lines, total_lines;
  unsigned long long seed;
  uint32_t stream;
  // multiply-high reciprocals: n / d == umul64hi(n, m) for d >= 2 (m = 2^64 / d
  // rounded up), exact for every n < 2^32; see set_divisors()
  unsigned long long mW, mN, mL1, mL2;
  // n / W == umulhi(n, mW32) for W >= 2 (mW32 = 2^32 / W rounded up; 0 for
  // W == 1), exact for n < 2^16: tile indices
  uint32_t mW32;
  // device arrays
  uint4* glink;          // [2][4][N] out-links by parity, port, tile
  // out-links that cross a CTA rectangle's edge, as written during a launch of
  // the plain cycle loop: [2][4][N] slots of two uint4, each 32-bit word half
  // a flit (low 16 bits) and the cycle tag (high 16 bits); see link_tag()
  uint4* gtag;
  uint32_t* core;        // [NCORE][N]
  uint4* cq;             // [N][core_q]
  uint4* sq;             // [N][svc_q]
  uint4* mq;             // [N][mem_q]  (ready, line, requester, 0)
  uint32_t* l1;          // [N][l1_sets][l1_ways] way words
  uint16_t* l1own;       // [N][l1_sets][l1_ways]
  uint32_t* l2;          // [N][l2_sets][l2_ways] way words
  uint16_t* l2ep;        // [N][l2_sets][l2_ways]    (LSPD)
  uint16_t* l2hist;      // [N][l2_sets][l2_ways][hist_stride] (migrate)
  uint32_t* dir;         // [total_lines]            (LSPD)
  uint32_t* fwd;         // [N][fwd_cap][2]          (migrate)
  // packet mode: per tile, rob_entries partly received packets, two words
  // each: line | type << 26 | valid << 31, and src | flits received << 16
  uint32_t* rob;         // [N][rob_entries][2]
  uint32_t* trace_off;   // [N+1]                    (trace mode)
  uint32_t* trace;       // refs                     (trace mode)
  // references drawn ahead by gen_refs_kernel: refbuf[tile][j] is reference
  // refk0[tile] + j (line | write << 31, or the probe destination), for
  // j < refcnt[tile]; refbuf == nullptr or j >= refcnt: drawn in place
  uint32_t* refbuf;      // [N][refcap]
  uint32_t* refk0;       // [N]
  uint32_t* refcnt;      // [N]
  int refcap;
  unsigned long long* stats;  // [NSTAT][N]
  unsigned long long* hist;   // [2][HIST_BINS]
  unsigned int* flags;        // [CTAs] last completed cycle + 1
  unsigned long long* err;    // min over (cycle << 8 | code); ~0 = none
};

// n / d with the reciprocal m of d (m = 0 encodes d == 1)
__device__ __forceinline__ uint32_t qdiv(uint32_t n, unsigned long long m) {
  return m ? (uint32_t)__umul64hi((unsigned long long)n, m) : n;
}
// host: reciprocals of the divisors used on the hot path
inline unsigned long long recip64(uint32_t d) { return d <= 1 ? 0ull : (~0ull) / d + 1; }
inline void set_divisors(Params& P) {
  P.hist_stride = hist_stride(P.mig_window);
  P.mW = recip64((uint32_t)P.W);
  P.mW32 = P.W <= 1 ? 0u : (uint32_t)((0x100000000ull + (uint32_t)P.W - 1) / (uint32_t)P.W);
  P.mN = recip64((uint32_t)P.N);
  P.mL1 = recip64((uint32_t)P.l1_sets);
  P.mL2 = recip64((uint32_t)P.l2_sets);
}

// ---------------------------------------------------------------- flits
// uint4 flit: x = inject cycle, y = src | dst << 16, z = line | type << 26,
// w = a | e << 16.  All-zero = empty link.  Under age_mode 1, x holds the
// inject cycle in its low AGE_SHIFT bits (runs end before cycle 2^AGE_SHIFT)
// and the flit's deflection count (its age, at most AGE_MAX) above them.
constexpr uint32_t AGE_SHIFT = 20;
constexpr uint32_t AGE_MAX = 4095;
constexpr uint32_t AGE_ONE = 1u << AGE_SHIFT;
__device__ __forceinline__ uint4 mkflit(uint32_t type, uint32_t src, uint32_t dst, uint32_t line,
                                        uint32_t a, uint32_t e) {
  return make_uint4(0u, src | (dst << 16), line | (type << 26), a | (e << 16));
}
__device__ __forceinline__ uint32_t ftype(uint4 f) { return f.z >> 26; }
__device__ __forceinline__ uint32_t fline(uint4 f) { return f.z & W_LINE; }
__device__ __forceinline__ uint32_t fsrc(uint4 f) { return f.y & 0xFFFFu; }
__device__ __forceinline__ uint32_t fdst(uint4 f) { return f.y >> 16; }
__device__ __forceinline__ uint32_t fa(uint4 f) { return f.w & 0xFFFFu; }
__device__ __forceinline__ uint32_t fe(uint4 f) { return f.w >> 16; }
// inject cycle and age of a flit (the age is 0 under age_mode 0)
__device__ __forceinline__ uint32_t finject(const Params& P, uint4 f) {
  return AGE1(P) ? f.x & (AGE_ONE - 1u) : f.x;
}
__device__ __forceinline__ uint32_t fage(const Params& P, uint4 f) {
  return AGE1(P) ? f.x >> AGE_SHIFT : 0u;
}
// priority key, smaller first: older (smaller inject cycle), then smaller
// source; under age_mode 1 more deflections before both (the age bits of x
// inverted, so that a larger age gives a smaller key).  The word x is the
// key's high half as it is, the source its low half.
__device__ __forceinline__ unsigned long long fkey(const Params& P, uint4 f) {
  const uint32_t flip = AGE1(P) ? (AGE_MAX << AGE_SHIFT) : 0u;
  return ((unsigned long long)(f.x ^ flip) << 32) | (f.y & 0xFFFFu);
}

// Tagged link slots (cross-rectangle links of the plain cycle loop).  Every
// 32-bit word carries 16 bits of the flit and the tag of the cycle that wrote
// it, so a reader that sees all eight words carry the tag it expects has the
// whole flit of that cycle: the data is its own ready flag, with no fence on
// the writer's side.  Tags have the top bit set, so zeroed slots never match;
// slot (t & 1) is rewritten every cycle, so within a launch a stale slot holds
// cycle t - 2 and never matches the tag of t.
__device__ __forceinline__ uint32_t link_tag(uint32_t t) { return 0x8000u | (t & 0x7FFFu); }
__device__ __forceinline__ void tag_encode(uint4 f, uint32_t tag, uint4& a, uint4& b) {
  a = make_uint4(__byte_perm(f.x, tag, 0x5410), __byte_perm(f.x, tag, 0x5432),
                 __byte_perm(f.y, tag, 0x5410), __byte_perm(f.y, tag, 0x5432));
  b = make_uint4(__byte_perm(f.z, tag, 0x5410), __byte_perm(f.z, tag, 0x5432),
                 __byte_perm(f.w, tag, 0x5410), __byte_perm(f.w, tag, 0x5432));
}
// true (and the flit in f) when all eight words carry `tag`
__device__ __forceinline__ bool tag_decode(uint4 a, uint4 b, uint32_t tag, uint4& f) {
  const uint32_t T = tag << 16;
  const uint32_t d = (a.x ^ T) | (a.y ^ T) | (a.z ^ T) | (a.w ^ T) | (b.x ^ T) | (b.y ^ T) |
                     (b.z ^ T) | (b.w ^ T);
  f = make_uint4(__byte_perm(a.x, a.y, 0x5410), __byte_perm(a.z, a.w, 0x5410),
                 __byte_perm(b.x, b.y, 0x5410), __byte_perm(b.z, b.w, 0x5410));
  return (d >> 16) == 0;
}
__device__ __forceinline__ void st_relaxed_v4(uint4* p, uint4 v) {
  asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint4 ld_relaxed_v4(const uint4* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
// store flit f to a tagged slot (two uint4)
__device__ __forceinline__ void tag_store(uint4* slot, uint4 f, uint32_t tag) {
  uint4 a, b;
  tag_encode(f, tag, a, b);
  st_relaxed_v4(slot, a);
  st_relaxed_v4(slot + 1, b);
}

// ---------------------------------------------------------------- hashing
// splitmix64 finaliser and the fold used by every state hash
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long hstart(unsigned long long w) {
  return mix64(w + 0x9E3779B97F4A7C15ull);
}
__device__ __forceinline__ unsigned long long hfold(unsigned long long h, unsigned long long w) {
  return mix64(h ^ w);
}
__device__ __forceinline__ unsigned long long hflit(const Params& P, unsigned long long h, uint4 f) {
  uint32_t ty = ftype(f);
  unsigned long long w0 = 0, w1 = 0, w2 = 0;
  if (ty) {
    w0 = (unsigned long long)ty | ((unsigned long long)fsrc(f) << 16) |
         ((unsigned long long)fdst(f) << 32) | ((unsigned long long)fa(f) << 48);
    w1 = (unsigned long long)fline(f) | ((unsigned long long)finject(P, f) << 32);
    w2 = (unsigned long long)fe(f) | ((unsigned long long)fage(P, f) << 32);
  }
  h = hfold(h, w0);
  h = hfold(h, w1);
  return hfold(h, w2);
}

// ---------------------------------------------------------------- Philox
// Philox4x64-10 from its published definition (Salmon, Moraes, Dror, Shaw,
// SC'11): ten rounds; each multiplies words 0 and 2 by the round constants,
// swaps the halves in and xors in the key; the key is bumped between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long c0, unsigned long long c1,
                                              unsigned long long c2, unsigned long long c3,
                                              unsigned long long k0, unsigned long long k1,
                                              unsigned long long out[4]) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B97F4A7C15ull;
      k1 += 0xBB67AE8584CAA73Bull;
    }
    unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// ---------------------------------------------------------------- tile state
struct Tile {
  uint32_t r, x, y;
  uint32_t next_ref, fsm, fsm_write, fsm_line, fsm_timer, fsm_start;
  uint32_t om_kind, om_write, om_line, om_start, om_timer, om_epoch, epoch;
  uint32_t cq_head, cq_len, sq_head, sq_len, mq_head, mq_len, fwd_next, fwd_n;
  uint4 cq_front, sq_front, mq_front;  // cached queue heads (valid when len > 0)
  uint4 ej;                            // flit ejected this cycle (or empty)
  uint32_t pf_raw, pf_ok;              // reference next_ref (encoded), if pf_ok
  uint32_t rk0, rcnt;                  // this tile's window of drawn-ahead references
  unsigned long long inj, ejc, defl, latsum, latmax, l2lsum;
  uint32_t sm[NSMALL];                 // small per-launch counter deltas
};
#define SMALL(i) T.sm[(i)-S_REFS]

__device__ __forceinline__ void set_error(const Params& P, uint32_t t, int code) {
  atomicMin(P.err, ((unsigned long long)t << 8) | (unsigned long long)code);
}
// one more deflection of flit f under age_mode 1 (Sec. 4.2: a deflection ages
// the flit); a flit already at AGE_MAX is left as it is and the cycle's error
// is raised
__device__ __forceinline__ void age_deflected(const Params& P, uint4& f, uint32_t t) {
  if ((f.x >> AGE_SHIFT) == AGE_MAX) set_error(P, t, ERR_RANGE);
  else f.x += AGE_ONE;
}

__device__ __forceinline__ uint32_t home_of(const Params& P, uint32_t line) {
  return line - qdiv(line, P.mN) * (uint32_t)P.N;
}
// the tile holding a line's directory entry (LSPD): its home, or the one
// directory node of the centralized variant
__device__ __forceinline__ uint32_t dir_home(const Params& P, uint32_t line) {
  return DIRC(P) ? (uint32_t)P.dir_tile : home_of(P, line);
}
__device__ __forceinline__ uint32_t l1_set(const Params& P, uint32_t line) {
  return line - qdiv(line, P.mL1) * (uint32_t)P.l1_sets;
}
__device__ __forceinline__ uint32_t l2_set(const Params& P, uint32_t line) {
  uint32_t v = POLICY(P) == POL_INTERLEAVED ? qdiv(line, P.mN) : line;
  return v - qdiv(v, P.mL2) * (uint32_t)P.l2_sets;
}

// ---------------------------------------------------------------- queues
__device__ __forceinline__ void count_sent(Tile& T, uint32_t ty) {
  if (ty == T_WT) SMALL(S_WTS)++;
  if (ty == T_REQ) SMALL(S_REQM)++;
  if (ty == T_DATA || ty == T_DRPOS || ty == T_DRNEG || ty == T_NACK) SMALL(S_REPS)++;
}
// flits of a message: 1, or in packet mode the Table 1 sizes of a data reply
// (remote L2 access, 4) and of a block migration (16)
__device__ __forceinline__ uint32_t packet_flits(const Params& P, uint32_t ty) {
  if (!PACKETS(P)) return 1;
  return ty == T_DATA ? 4u : (ty == T_MIG ? 16u : 1u);
}
// service-queue messages are never refused: exceeding the capacity is an
// error.  A multi-flit packet is queued whole, flit i carrying a = i, e = n.
__device__ __forceinline__ void send_svc(const Params& P, Tile& T, uint4 f, uint32_t t) {
  if (T.sq_len >= (uint32_t)P.svc_q) {
    set_error(P, t, ERR_OVERFLOW);
    return;
  }
  count_sent(T, ftype(f));
  const uint32_t n = packet_flits(P, ftype(f));
  if (n > 1 && T.sq_len + n > (uint32_t)P.svc_q) {
    set_error(P, t, ERR_OVERFLOW);
    return;
  }
  for (uint32_t i = 0; i < n; ++i) {
    uint4 g = f;
    if (n > 1) g.w = i | (n << 16);
    uint32_t slot = T.sq_head + T.sq_len;
    if (slot >= (uint32_t)P.svc_q) slot -= P.svc_q;
    P.sq[(size_t)T.r * P.svc_q + slot] = g;
    if (T.sq_len == 0) T.sq_front = g;
    T.sq_len++;
  }
}
__device__ __forceinline__ void send_core(const Params& P, Tile& T, uint4 f) {
  count_sent(T, ftype(f));
  uint32_t slot = T.cq_head + T.cq_len;
  if (slot >= (uint32_t)P.core_q) slot -= P.core_q;
  P.cq[(size_t)T.r * P.core_q + slot] = f;
  if (T.cq_len == 0) T.cq_front = f;
  T.cq_len++;
}
__device__ __forceinline__ bool cq_full(const Params& P, const Tile& T) {
  return T.cq_len >= (uint32_t)P.core_q;
}

// ---------------------------------------------------------------- cache sets
// A set's way words live in registers while it is worked on; the loops are
// fully unrolled over MW (a compile-time bound >= the configured ways, chosen
// at launch) so the array never leaves the register file.
template <int MW>
__device__ __forceinline__ void load_set(const uint32_t* p, int ways, uint32_t (&w)[MW]) {
#pragma unroll
  for (int i = 0; i < MW; ++i) w[i] = 0;
  if ((ways & 3) == 0) {
#pragma unroll
    for (int q = 0; q < MW / 4; ++q)
      if (q * 4 < ways) {
        uint4 v = reinterpret_cast<const uint4*>(p)[q];
        w[q * 4] = v.x;
        w[q * 4 + 1] = v.y;
        w[q * 4 + 2] = v.z;
        w[q * 4 + 3] = v.w;
      }
  } else {
#pragma unroll
    for (int i = 0; i < MW; ++i)
      if (i < ways) w[i] = p[i];
  }
}
template <int MW>
__device__ __forceinline__ void store_set(uint32_t* p, int ways, const uint32_t (&w)[MW]) {
  if ((ways & 3) == 0) {
#pragma unroll
    for (int q = 0; q < MW / 4; ++q)
      if (q * 4 < ways)
        reinterpret_cast<uint4*>(p)[q] = make_uint4(w[q * 4], w[q * 4 + 1], w[q * 4 + 2], w[q * 4 + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < MW; ++i)
      if (i < ways) p[i] = w[i];
  }
}
__device__ __forceinline__ uint32_t wrank(uint32_t v) { return (v >> W_RANK_SHIFT) & 15u; }
__device__ __forceinline__ uint32_t wset_rank(uint32_t v, uint32_t r) {
  return (v & ~(15u << W_RANK_SHIFT)) | (r << W_RANK_SHIFT);
}
// the way holding `line` and its word, or -1 (lines are below 2^26, so the
// valid bit and the line compare as one masked word)
template <int MW>
__device__ __forceinline__ int set_find(const uint32_t (&w)[MW], int ways, uint32_t line,
                                        uint32_t& word) {
  int found = -1;
  word = 0;
  const uint32_t key = W_VALID | line;
#pragma unroll
  for (int i = MW - 1; i >= 0; --i)
    if (i < ways && (w[i] & (W_VALID | W_LINE)) == key) {
      found = i;
      word = w[i];
    }
  return found;
}
template <int MW>
__device__ __forceinline__ int set_find(const uint32_t (&w)[MW], int ways, uint32_t line) {
  uint32_t word;
  return set_find(w, ways, line, word);
}
// make way `way` the most recently used (and OR `bits` into its word);
// `prev_rank` is its rank before (the number of valid ways for a way that was
// invalid).  The valid ways more recent than it age by one: with the valid bit
// and the 4-bit rank in the word's top five bits, "valid and rank < prev" is
// one unsigned compare.  The way itself may age here; its rank is reset after.
template <int MW>
__device__ __forceinline__ void set_promote(uint32_t (&w)[MW], int ways, int way, uint32_t prev_rank,
                                            uint32_t bits = 0) {
  const uint32_t lim = prev_rank << W_RANK_SHIFT;
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i < ways && (w[i] & 0xF8000000u) - W_VALID < lim) w[i] += 1u << W_RANK_SHIFT;
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i == way) w[i] = (w[i] & ~(15u << W_RANK_SHIFT)) | bits;
}
template <int MW>
__device__ __forceinline__ uint32_t set_get(const uint32_t (&w)[MW], int way) {
  uint32_t v = 0;
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i == way) v = w[i];
  return v;
}
template <int MW>
__device__ __forceinline__ void set_put(uint32_t (&w)[MW], int way, uint32_t v) {
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i == way) w[i] = v;
}
// promote a way found holding `word`
template <int MW>
__device__ __forceinline__ void set_touch(uint32_t (&w)[MW], int ways, int way, uint32_t word,
                                          uint32_t bits = 0) {
  set_promote(w, ways, way, wrank(word), bits);
}
// victim: lowest-index invalid way, else the least recently used way
template <int MW>
__device__ __forceinline__ int set_victim(const uint32_t (&w)[MW], int ways) {
  int inv = -1, lru = 0;
#pragma unroll
  for (int i = MW - 1; i >= 0; --i)
    if (i < ways) {
      if (!(w[i] & W_VALID)) inv = i;
      else if (wrank(w[i]) == (uint32_t)(ways - 1)) lru = i;
    }
  return inv >= 0 ? inv : lru;
}
template <int MW>
__device__ __forceinline__ uint32_t set_nvalid(const uint32_t (&w)[MW], int ways) {
  uint32_t n = 0;
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i < ways && (w[i] & W_VALID)) n++;
  return n;
}
// choose the way to fill: the lowest invalid way, else the least recently
// used; returns it with its old word and its rank before (for an invalid way,
// the number of valid ways), in one pass over the set
template <int MW>
__device__ __forceinline__ int set_choose(const uint32_t (&w)[MW], int ways, uint32_t& old,
                                          uint32_t& prev_rank) {
  uint32_t minv = 0, nvalid = 0, lruw = 0;
  int lru = 0;
  const uint32_t lru_top = W_VALID | ((uint32_t)(ways - 1) << W_RANK_SHIFT);
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i < ways) {
      const uint32_t v = w[i] >> 31;
      minv |= (v ^ 1u) << i;
      nvalid += v;
      if ((w[i] & 0xF8000000u) == lru_top) {
        lru = i;
        lruw = w[i];
      }
    }
  if (minv) {
    old = 0;
    prev_rank = nvalid;
    return __ffs(minv) - 1;
  }
  old = lruw;
  prev_rank = (uint32_t)(ways - 1);
  return lru;
}
// make way `way` the most recently used, replacing its word by `word`
template <int MW>
__device__ __forceinline__ void set_replace(uint32_t (&w)[MW], int ways, int way, uint32_t prev_rank,
                                            uint32_t word) {
  const uint32_t lim = prev_rank << W_RANK_SHIFT;
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i < ways && (w[i] & 0xF8000000u) - W_VALID < lim) w[i] += 1u << W_RANK_SHIFT;
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i == way) w[i] = word;
}
// remove way `way`; the ways it was more recent than move up one rank
template <int MW>
__device__ __forceinline__ void set_invalidate(uint32_t (&w)[MW], int ways, int way) {
  uint32_t rk = wrank(set_get(w, way));
#pragma unroll
  for (int i = 0; i < MW; ++i)
    if (i < ways && i != way && (w[i] & W_VALID) && wrank(w[i]) > rk)
      w[i] = wset_rank(w[i], wrank(w[i]) - 1);
  set_put(w, way, 0u);
}

__device__ __forceinline__ size_t l1_base(const Params& P, uint32_t r, uint32_t set) {
  return ((size_t)r * P.l1_sets + set) * L1WAYS(P);
}
__device__ __forceinline__ size_t l2_base(const Params& P, uint32_t r, uint32_t set) {
  return ((size_t)r * P.l2_sets + set) * L2WAYS(P);
}
// The L2 set a request or write-through for `line` will look up at tile `h`,
// pulled into the GPU's L2 cache when the message leaves.  A large mesh's
// slice tag arrays are far larger than that cache, so without this the
// lookup, some hundred simulated cycles later, would wait on DRAM inside
// Phase 3 of the home's warp.  A prefetch has no effect on any result.  The
// batch kernel, whose small instances stay in the cache, builds without it
// (NOC_PREFETCH_HOME 0).
#ifndef NOC_PREFETCH_HOME
#define NOC_PREFETCH_HOME 1
#endif
__device__ __forceinline__ void prefetch_home_set(const Params& P, uint32_t h, uint32_t line) {
#if NOC_PREFETCH_HOME
  asm volatile("prefetch.global.L2 [%0];" ::"l"(P.l2 + l2_base(P, h, l2_set(P, line))));
#endif
}


__device__ __forceinline__ uint16_t* hist_ptr(const Params& P, size_t way_index) {
  return P.l2hist + way_index * (size_t)P.hist_stride;
}

// The checked build (-DNOC_CHECKS=1, noc_set_checks) verifies the single-writer
// discipline the model relies on.  Every per-tile structure is indexed by the
// tile's own id, so the directory -- indexed by a line that a message carries
// -- is the one structure a second writer could reach: its entry for a line
// may be touched only at that line's directory tile.  The message handlers
// that touch it (DA, DINV, DIRUPD) check the tile and the line's range first
// and report ERR_OWNER or ERR_RANGE instead of touching the entry.
#ifndef NOC_CHECKS
#define NOC_CHECKS 0
#endif
__device__ __forceinline__ bool dir_owned(const Params& P, const Tile& T, uint32_t line, uint32_t t) {
#if NOC_CHECKS
  if (line >= (uint32_t)P.total_lines) {
    set_error(P, t, ERR_RANGE);
    return false;
  }
  if (dir_home(P, line) != T.r) {
    set_error(P, t, ERR_OWNER);
    return false;
  }
#endif
  return true;
}

// directory entry delete for an evicted L2 victim (Sec. 3.4)
static __device__ void send_dinv(const Params& P, Tile& T, uint32_t vline, uint32_t vepoch, uint32_t t) {
  uint32_t h = dir_home(P, vline);
  if (h == T.r) {
    if (P.dir[vline] == (T.r | (vepoch << 16))) P.dir[vline] = DIR_NONE;
  } else {
    send_svc(P, T, mkflit(T_DINV, T.r, h, vline, 0, vepoch), t);
  }
}

// install `line` in this tile's L2 slice: insert if absent (evicting the
// victim), else touch; returns the way index
template <int W2>
static __device__ int l2_install(const Params& P, Tile& T, uint32_t line, uint32_t epoch, uint32_t t) {
  uint32_t set = l2_set(P, line);
  size_t base = l2_base(P, T.r, set);
  uint32_t w[W2];
  load_set(P.l2 + base, L2WAYS(P), w);
  uint32_t fword;
  int way = set_find(w, L2WAYS(P), line, fword);
  if (way >= 0) {
    set_touch(w, L2WAYS(P), way, fword);
  } else {
    uint32_t old, prev;
    way = set_choose(w, L2WAYS(P), old, prev);
    if (old & W_VALID) {
      if (old & W_DIRTY) SMALL(S_MEMWB)++;
      if (POLICY(P) != POL_INTERLEAVED) send_dinv(P, T, old & W_LINE, P.l2ep[base + way], t);
    }
    set_replace(w, L2WAYS(P), way, prev, W_VALID | line);
    if (POLICY(P) == POL_MIGRATE) {
      uint16_t* hp = hist_ptr(P, base + way);
      hp[0] = 0;
      hp[1] = 0;
    }
  }
  store_set(P.l2 + base, L2WAYS(P), w);
  if (POLICY(P) != POL_INTERLEAVED) P.l2ep[base + way] = (uint16_t)epoch;
  return way;
}

// write-through performed at this tile's own slice
template <int W2>
static __device__ void local_wt(const Params& P, Tile& T, uint32_t line) {
  uint32_t set = l2_set(P, line);
  size_t base = l2_base(P, T.r, set);
  uint32_t w[W2];
  load_set(P.l2 + base, L2WAYS(P), w);
  uint32_t fword;
  int way = set_find(w, L2WAYS(P), line, fword);
  if (way >= 0) {
    set_touch(w, L2WAYS(P), way, fword, W_DIRTY);
    store_set(P.l2 + base, L2WAYS(P), w);
    SMALL(S_WTH)++;
  } else {
    SMALL(S_MEMW)++;
  }
}

// a write of `line` reaching the L2 that holds it: the owner recorded with the
// L1 copy (this tile's own slice, another tile through a WT message, or
// memory when no slice holds it)
template <int W2>
__device__ __forceinline__ void write_to_owner(const Params& P, Tile& T, uint32_t line, uint32_t owner,
                                               uint32_t t) {
  if (owner == T.r) local_wt<W2>(P, T, line);
  else if (owner == NO_TILE) SMALL(S_MEMW)++;
  else {
    prefetch_home_set(P, owner, line);
    send_svc(P, T, mkflit(T_WT, T.r, owner, line, 0, 0), t);
  }
}

// fill the L1 with `line` (insert if absent, else touch); `owner` is the tile
// whose L2 supplied it.  Write-through: a write is passed on to the owner
// after the fill and victims are clean.  Write-back: a write dirties the L1
// copy, and a dirty victim is written to its owner first.
template <int W1, int W2>
static __device__ void l1_fill(const Params& P, Tile& T, uint32_t line, uint32_t owner, uint32_t write,
                               uint32_t t) {
  uint32_t set = l1_set(P, line);
  size_t base = l1_base(P, T.r, set);
  uint32_t w[W1];
  load_set(P.l1 + base, L1WAYS(P), w);
  const uint32_t dirty = (L1WB(P) && write) ? W_DIRTY : 0u;
  uint32_t fword;
  int way = set_find(w, L1WAYS(P), line, fword);
  if (way >= 0) {
    set_touch(w, L1WAYS(P), way, fword, dirty);
  } else {
    uint32_t old, prev;
    way = set_choose(w, L1WAYS(P), old, prev);
    if (L1WB(P) && (old & W_VALID) && (old & W_DIRTY))
      write_to_owner<W2>(P, T, old & W_LINE, P.l1own[base + way], t);
    set_replace(w, L1WAYS(P), way, prev, W_VALID | line | dirty);
  }
  store_set(P.l1 + base, L1WAYS(P), w);
  P.l1own[base + way] = (uint16_t)owner;
  if (write && !L1WB(P)) write_to_owner<W2>(P, T, line, owner, t);
}

// record accessor `who` in the block's history of the last mig_window accessors
static __device__ void hist_push(const Params& P, size_t way_index, uint32_t who) {
  uint16_t* hp = hist_ptr(P, way_index);
  uint32_t n = hp[0];
  if (n < (uint32_t)P.mig_window) {
    hp[2 + n] = (uint16_t)who;
    hp[0] = (uint16_t)(n + 1);
  } else {
    for (int i = 0; i + 1 < P.mig_window; ++i) hp[2 + i] = hp[3 + i];
    hp[2 + P.mig_window - 1] = (uint16_t)who;
  }
}

__device__ __forceinline__ void l2lat_sample(Tile& T, uint32_t t, uint32_t start,
                                             uint32_t* sh_hist) {
  uint32_t lat = t - start;
  T.l2lsum += lat;
  SMALL(S_L2LCNT)++;
  atomicAdd(&sh_hist[HIST_BINS + (lat < HIST_BINS - 1 ? lat : HIST_BINS - 1)], 1u);
}

__device__ __forceinline__ void set_om(Tile& T, uint32_t kind, uint32_t line, uint32_t write,
                                       uint32_t start) {
  T.om_kind = kind;
  T.om_line = line;
  T.om_write = write;
  T.om_start = start;
  T.om_timer = 0;
  T.om_epoch = 0;
}

// ---------------------------------------------------------------- Phase 1
// the L1 lookup of a reference; returns false if the action was not taken
template <int W1, int W2>
static __device__ bool l1_step(const Params& P, Tile& T, uint32_t t, uint32_t line, uint32_t write) {
  uint32_t set = l1_set(P, line);
  size_t base = l1_base(P, T.r, set);
  uint32_t w[W1];
  load_set(P.l1 + base, L1WAYS(P), w);
  uint32_t fword;
  int way = set_find(w, L1WAYS(P), line, fword);
  if (way >= 0) {
    if (write && !L1WB(P)) {
      uint32_t owner = P.l1own[base + way];
      if (owner == T.r) {
        local_wt<W2>(P, T, line);
      } else if (owner == NO_TILE) {
        SMALL(S_MEMW)++;
      } else {
        if (cq_full(P, T)) {
          SMALL(S_CQST)++;
          return false;
        }
        prefetch_home_set(P, owner, line);
        send_core(P, T, mkflit(T_WT, T.r, owner, line, 0, 0));
      }
    }
    // write-back: the write dirties the L1 copy, nothing leaves the tile
    set_touch(w, L1WAYS(P), way, fword, (write && L1WB(P)) ? W_DIRTY : 0u);
    store_set(P.l1 + base, L1WAYS(P), w);
    SMALL(S_L1H)++;
    T.fsm = FSM_IDLE;
    return true;
  }
  SMALL(S_L1M)++;
  T.fsm = FSM_L2WAIT;
  T.fsm_line = line;
  T.fsm_write = write;
  T.fsm_start = t;
  T.fsm_timer = t + (uint32_t)P.l1_miss;
  return true;
}

template <int W1, int W2>
static __device__ void l2_step(const Params& P, Tile& T, uint32_t t, uint32_t* sh_hist) {
  const uint32_t line = T.fsm_line, start = T.fsm_start, write = T.fsm_write;
  const bool busy = T.om_kind != OM_NONE;
  uint32_t set = l2_set(P, line);
  size_t base = l2_base(P, T.r, set);

  if (POLICY(P) == POL_INTERLEAVED) {
    uint32_t h = home_of(P, line);
    if (h == T.r) {
      uint32_t w[W2];
      load_set(P.l2 + base, L2WAYS(P), w);
      uint32_t fword;
      int way = set_find(w, L2WAYS(P), line, fword);
      if (way >= 0) {
        SMALL(S_L2H)++;
        set_touch(w, L2WAYS(P), way, fword);
        store_set(P.l2 + base, L2WAYS(P), w);
        l1_fill<W1, W2>(P, T, line, T.r, write, t);
        l2lat_sample(T, t, start, sh_hist);
        T.fsm = FSM_IDLE;
        return;
      }
      if (busy) {
        SMALL(S_MMST)++;
        T.fsm = FSM_STALL;
        return;
      }
      SMALL(S_L2M)++;
      SMALL(S_MEMREQ)++;
      set_om(T, OM_MEM_L2, line, write, start);
      T.om_timer = t + (uint32_t)P.mem_lat;
      T.fsm = FSM_IDLE;
      return;
    }
    if (busy) {
      SMALL(S_MMST)++;
      T.fsm = FSM_STALL;
      return;
    }
    if (cq_full(P, T)) {
      SMALL(S_CQST)++;
      return;
    }
    prefetch_home_set(P, h, line);
    send_core(P, T, mkflit(T_REQ, T.r, h, line, T.r, 0));
    set_om(T, OM_WAIT_DATA, line, write, start);
    T.fsm = FSM_IDLE;
    return;
  }

  // LSPD: the requester's own slice first (local placement, Sec. 3.3)
  uint32_t w[W2];
  load_set(P.l2 + base, L2WAYS(P), w);
  uint32_t fword;
  int way = set_find(w, L2WAYS(P), line, fword);
  if (way >= 0) {
    SMALL(S_L2H)++;
    set_touch(w, L2WAYS(P), way, fword);
    store_set(P.l2 + base, L2WAYS(P), w);
    if (POLICY(P) == POL_MIGRATE) hist_push(P, base + way, T.r);
    l1_fill<W1, W2>(P, T, line, T.r, write, t);
    l2lat_sample(T, t, start, sh_hist);
    T.fsm = FSM_IDLE;
    return;
  }
  if (busy) {
    SMALL(S_MMST)++;
    T.fsm = FSM_STALL;
    return;
  }
  uint32_t h = dir_home(P, line);
  if (h == T.r) {
    uint32_t D = P.dir[line];
    if (D == DIR_NONE || (D & 0xFFFFu) == T.r) {
      SMALL(S_L2M)++;
      SMALL(S_DIRS)++;
      T.epoch = (T.epoch + 1) & 0xFFFFu;
      P.dir[line] = T.r | (T.epoch << 16);
      set_om(T, OM_MEM_L2, line, write, start);
      T.om_timer = t + (uint32_t)P.mem_lat;
      T.om_epoch = T.epoch;
      SMALL(S_MEMREQ)++;
      T.fsm = FSM_IDLE;
      return;
    }
    if (cq_full(P, T)) {
      SMALL(S_CQST)++;
      return;
    }
    SMALL(S_L2M)++;
    SMALL(S_DIRS)++;
    send_core(P, T, mkflit(T_REQ, T.r, D & 0xFFFFu, line, T.r, 0));
    set_om(T, OM_WAIT_DATA, line, write, start);
    T.fsm = FSM_IDLE;
    return;
  }
  if (cq_full(P, T)) {
    SMALL(S_CQST)++;
    return;
  }
  SMALL(S_L2M)++;
  T.epoch = (T.epoch + 1) & 0xFFFFu;
  send_core(P, T, mkflit(T_DA, T.r, h, line, 0, T.epoch));
  set_om(T, OM_WAIT_DR, line, write, start);
  T.fsm = FSM_IDLE;
}

// the line of reference k of this core (Philox stream, Sec. 6.2.3 stand-in)
static __device__ uint32_t draw_line(const Params& P, uint32_t core, uint32_t k, uint32_t& write) {
  unsigned long long w[4];
  philox4x64_10(k, core, P.stream, 0, P.seed, 0x4E4F43ull, w);
  write = (uint32_t)(w[0] >> 48) < P.write_q16 ? 1u : 0u;
  uint32_t r16 = (uint32_t)(w[1] >> 48);
  const uint32_t shared_base = P.remote_lines;
  if (r16 < P.priv_q16)
    return P.remote_lines + P.shared_lines + core * P.priv_lines +
           (uint32_t)__umul64hi(w[2], P.priv_lines);
  if (r16 < P.priv_q16 + P.shared_q16) {
    if (P.hot_side > 0 && (uint32_t)(w[3] >> 48) < P.hot_q16) {
      const uint32_t hs = (uint32_t)P.hot_side;
      uint32_t j = (uint32_t)__umul64hi(w[2], (unsigned long long)hs * hs);
      uint32_t hj = (uint32_t)(P.hot_y0 + j / hs) * (uint32_t)P.W + (uint32_t)P.hot_x0 + j % hs;
      const uint32_t N = (uint32_t)P.N;
      uint32_t i0 = (hj + N - shared_base % N) % N;
      uint32_t cnt = P.shared_lines > i0 ? (P.shared_lines - i0 + N - 1) / N : 0;
      if (cnt > 0) return shared_base + i0 + (uint32_t)__umul64hi(w[3] << 16, cnt) * N;
    }
    return shared_base + (uint32_t)__umul64hi(w[2], P.shared_lines);
  }
  return (uint32_t)__umul64hi(w[2], P.remote_lines);
}

__device__ __forceinline__ void mq_pop(const Params& P, Tile& T) {
  T.mq_head = T.mq_head + 1 == (uint32_t)P.mem_q ? 0 : T.mq_head + 1;
  T.mq_len--;
  if (T.mq_len > 0) T.mq_front = P.mq[(size_t)T.r * P.mem_q + T.mq_head];
}

// Reference k of core `core`, encoded (line | write << 31 for cache traffic,
// the destination tile for network-only probes); false past a trace's end.
// This is the definition; gen_refs_kernel and the in-place draw both use it.
static __device__ bool draw_ref(const Params& P, uint32_t core, uint32_t k, uint32_t& raw) {
  if (MODE(P) == MODE_TRACE) {
    uint32_t off = P.trace_off[core], n = P.trace_off[core + 1] - off;
    if (k >= n) return false;
    raw = P.trace[off + k];
    return true;
  }
  if (MODE(P) == MODE_NETWORK) {
    unsigned long long w[4];
    philox4x64_10(k, core, P.stream, 0, P.seed, 0x4E4F43ull, w);
    uint32_t dst = (uint32_t)__umul64hi(w[1], (unsigned long long)(P.N - 1));
    raw = dst >= core ? dst + 1 : dst;
    return true;
  }
  uint32_t write;
  uint32_t line = draw_line(P, core, k, write);
  raw = line | (write << 31);
  return true;
}

// reference next_ref from the drawn-ahead window if it is there, else drawn now
__device__ __forceinline__ bool next_ref_raw(const Params& P, const Tile& T, uint32_t& raw) {
  const uint32_t j = T.next_ref - T.rk0;
  if (j < T.rcnt) {
    raw = P.refbuf[(size_t)T.r * P.refcap + j];
    return true;
  }
  return draw_ref(P, T.r, T.next_ref, raw);
}

// start loading the next reference into a register (used cycles later)
__device__ __forceinline__ void prefetch_next_ref(const Params& P, Tile& T) {
  const uint32_t j = T.next_ref - T.rk0;
  if (j < T.rcnt) {
    T.pf_raw = P.refbuf[(size_t)T.r * P.refcap + j];
    T.pf_ok = 1;
  } else {
    T.pf_ok = 0;
  }
}

// Phase 1; returns true if the core took an action this cycle
template <int W1, int W2>
static __device__ bool phase1(const Params& P, Tile& T, uint32_t t, bool draining, uint32_t* sh_hist) {
  // (i) memory returns at an interleaved home: install, then reply
  while (T.mq_len > 0 && T.mq_front.x <= t) {
    uint32_t line = T.mq_front.y, req = T.mq_front.z;
    mq_pop(P, T);
    l2_install<W2>(P, T, line, 0, t);
    send_svc(P, T, mkflit(T_DATA, T.r, req, line, 0, 0), t);
  }
  // (ii) this core's outstanding memory fetch completes
  if ((T.om_kind == OM_MEM_L2 || T.om_kind == OM_MEM_L1) && T.om_timer <= t) {
    if (T.om_kind == OM_MEM_L2) {
      l2_install<W2>(P, T, T.om_line, T.om_epoch, t);
      l1_fill<W1, W2>(P, T, T.om_line, T.r, T.om_write, t);
    } else {
      l1_fill<W1, W2>(P, T, T.om_line, NO_TILE, T.om_write, t);
    }
    l2lat_sample(T, t, T.om_start, sh_hist);
    set_om(T, OM_NONE, 0, 0, 0);
  }
  // (iii) at most one core action
  if (T.fsm == FSM_L2WAIT) {
    if (t < T.fsm_timer) return false;
    l2_step<W1, W2>(P, T, t, sh_hist);
    return true;
  }
  if (T.fsm == FSM_STALL) {
    if (T.om_kind != OM_NONE) return false;
    l1_step<W1, W2>(P, T, t, T.fsm_line, T.fsm_write);
    return true;
  }
  if (draining || P.period <= 0) return false;
  if ((unsigned long long)t < (unsigned long long)T.next_ref * (unsigned long long)P.period) return false;

  if (MODE(P) == MODE_NETWORK && P.N < 2) return false;
  uint32_t raw;
  if (T.pf_ok) {
    raw = T.pf_raw;
  } else {
    if (!next_ref_raw(P, T, raw)) return false;
    T.pf_raw = raw;          // kept for a retry after a full core queue
    T.pf_ok = 1;
  }
  if (MODE(P) == MODE_NETWORK) {
    if (cq_full(P, T)) {
      SMALL(S_CQST)++;
      return true;
    }
    send_core(P, T, mkflit(T_PROBE, T.r, raw, 0, 0, 0));
    T.next_ref++;
    SMALL(S_REFS)++;
    prefetch_next_ref(P, T);
    return true;
  }
  if (l1_step<W1, W2>(P, T, t, raw & 0x7FFFFFFFu, raw >> 31)) {
    T.next_ref++;
    SMALL(S_REFS)++;
    prefetch_next_ref(P, T);
  }
  return true;
}

// ---------------------------------------------------------------- Phase 2
// compare-and-swap of two (key, flit) slots, smaller key first
__device__ __forceinline__ void cswap(unsigned long long& ka, uint4& fa_, unsigned long long& kb,
                                      uint4& fb_) {
  if (kb < ka) {
    unsigned long long tk = ka;
    ka = kb;
    kb = tk;
    uint4 tf = fa_;
    fa_ = fb_;
    fb_ = tf;
  }
}

// One bufferless router (Sec. 4.3): eject, inject, rank, select ports.
// `in` are this cycle's arrivals by input port, `exists` the port mask.  Each
// flit is stored straight to its output port's slot: so[p * so_stride] in
// shared memory and, for ports in `edge` (links leaving the CTA's rectangle),
// also go[p * go_stride] in global memory; unused ports get an empty flit.
// With TAGGED, `go` points at tagged slots (two uint4 each, see tag_store)
// and go_stride counts uint4.
template <bool TAGGED = false>
__device__ __forceinline__ void route(const Params& P, Tile& T, uint32_t t, uint4 (&in)[4],
                                      uint32_t exists, uint4* so, int so_stride, uint4* go,
                                      size_t go_stride, uint32_t edge) {
  const unsigned long long NOKEY = ~0ull;
  unsigned long long k[4];
  int n_arr = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    bool v = ftype(in[d]) != T_NONE;
    n_arr += v;
    k[d] = v ? fkey(P, in[d]) : NOKEY;
  }
  // eject the highest-priority arrival addressed to this tile
  int ej = -1;
  unsigned long long ejk = NOKEY;
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (k[d] != NOKEY && fdst(in[d]) == T.r && k[d] < ejk) {
      ejk = k[d];
      ej = d;
    }
  T.ej = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (d == ej) {
      T.ej = in[d];
      k[d] = NOKEY;
    }
  // rank the remaining arrivals oldest first: 4-input sorting network
  cswap(k[0], in[0], k[1], in[1]);
  cswap(k[2], in[2], k[3], in[3]);
  cswap(k[0], in[0], k[2], in[2]);
  cswap(k[1], in[1], k[3], in[3]);
  cswap(k[1], in[1], k[2], in[2]);
  // inject when an input port is free: service queue first, then core queue
  uint4 inj = make_uint4(0, 0, 0, 0);
  bool has_inj = false;
  if (n_arr < __popc(exists)) {
    if (T.sq_len > 0) {
      inj = T.sq_front;
      T.sq_head = T.sq_head + 1 == (uint32_t)P.svc_q ? 0 : T.sq_head + 1;
      T.sq_len--;
      if (T.sq_len > 0) T.sq_front = P.sq[(size_t)T.r * P.svc_q + T.sq_head];
      has_inj = true;
    } else if (T.cq_len > 0) {
      inj = T.cq_front;
      T.cq_head = T.cq_head + 1 == (uint32_t)P.core_q ? 0 : T.cq_head + 1;
      T.cq_len--;
      if (T.cq_len > 0) T.cq_front = P.cq[(size_t)T.r * P.core_q + T.cq_head];
      has_inj = true;
    }
    if (has_inj) {
      inj.x = t;
      inj.y = (inj.y & 0xFFFF0000u) | T.r;
      T.inj++;
    }
  }
  // port selection: first free port of [X-productive, Y-productive, N, S, E, W]
  uint32_t freem = exists;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    uint4 f = i < 4 ? in[i] : inj;
    const bool valid = i < 4 ? (k[i] != NOKEY) : has_inj;
    if (!valid) continue;
    const uint32_t dst = fdst(f);
    const uint32_t dsty = P.mW32 ? __umulhi(dst, P.mW32) : dst;
    const int dx = (int)(dst - dsty * (uint32_t)P.W) - (int)T.x;
    const int dy = (int)dsty - (int)T.y;
    const uint32_t xb = dx > 0 ? (1u << P_E) : (dx < 0 ? (1u << P_W) : 0u);
    const uint32_t yb = dy > 0 ? (1u << P_S) : (dy < 0 ? (1u << P_N) : 0u);
    uint32_t pick;
    if (freem & xb) pick = xb;
    else if (freem & yb) pick = yb;
    else {
      pick = freem & (0u - freem);  // lowest free port: N, S, E, W order
      T.defl++;
      if (AGE1(P)) age_deflected(P, f, t);
    }
    freem &= ~pick;
    const int p = __ffs(pick) - 1;
    so[p * so_stride] = f;
    if (edge & pick) {
      if (TAGGED) tag_store(&go[p * go_stride], f, link_tag(t));
      else __stcg(&go[p * go_stride], f);
    }
  }
  // the ports no flit took carry nothing this cycle
  const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (freem & (1u << d) || !(exists & (1u << d))) {
      so[d * so_stride] = z;
      if (edge & (1u << d)) {
        if (TAGGED) tag_store(&go[d * go_stride], z, link_tag(t));
        else __stcg(&go[d * go_stride], z);
      }
    }
}

// The productive ports of a flit at tile (x, y): X direction in bits 0-3, Y
// direction in bits 4-7 (one port bit each, or none when aligned).
__device__ __forceinline__ uint32_t prod_ports(const Params& P, uint32_t dst, uint32_t x, uint32_t y) {
  const uint32_t dy_ = P.mW32 ? __umulhi(dst, P.mW32) : dst;
  const uint32_t dx_ = dst - dy_ * (uint32_t)P.W;
  const uint32_t xb = dx_ > x ? (1u << P_E) : (dx_ < x ? (1u << P_W) : 0u);
  const uint32_t yb = dy_ > y ? (1u << P_S) : (dy_ < y ? (1u << P_N) : 0u);
  return xb | (yb << 4);
}
// first free port of [X-productive, Y-productive, N, S, E, W] for a flit
// whose productive ports are `prod` (prod_ports), counting a deflection when
// neither productive port is free; with `on` = 0 (no such flit) nothing is
// picked or counted.  Branch-free: lanes differ in how many flits they place.
__device__ __forceinline__ uint32_t pick_port(uint32_t prod, uint32_t freem, uint32_t on, uint32_t& defl) {
  const uint32_t xb = prod & 15u, yb = prod >> 4;
  const uint32_t low = freem & (0u - freem);
  const bool px = (freem & xb) != 0, py = (freem & yb) != 0;
  defl += (!px && !py) ? (on & 1u) : 0u;
  return (px ? xb : (py ? yb : low)) & on;
}

// The flit a tile would inject this cycle if an input port is free (the
// service-queue head, else the core-queue head) with its productive ports.
// It depends on the tile's own state only, so the plain cycle loop takes it
// before waiting for the neighbours' outputs.
struct InjCand {
  uint4 f;
  uint32_t prod;  // prod_ports() of its destination
  int q;          // 0: none, 1: service queue, 2: core queue
};
__device__ __forceinline__ InjCand inj_candidate(const Params& P, const Tile& T) {
  InjCand c;
  c.q = T.sq_len > 0 ? 1 : (T.cq_len > 0 ? 2 : 0);
  c.f = c.q == 1 ? T.sq_front : T.cq_front;
  c.prod = c.q ? prod_ports(P, fdst(c.f), T.x, T.y) : 0u;
  return c;
}

// Copy this tile's outputs of cycle t on the links in `edge` (leaving the CTA
// rectangle) from their shared-memory slots to the tagged global slots.
__device__ __forceinline__ void store_edges(const uint4* so, int so_stride, uint4* go, size_t go_stride,
                                            uint32_t edge, uint32_t t) {
  if (edge) {
    const uint32_t tag = link_tag(t);
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if ((edge >> d) & 1u) tag_store(&go[d * go_stride], so[d * so_stride], tag);
  }
}

// The router of Sec. 4.3 as route() computes it, for the plain cycle loop:
// arrivals are ranked by pairwise key comparisons instead of being sorted, so
// flits never move between registers; the ejected flit is the lowest-ranked
// arrival addressed here, and the others' ranks close up behind it.  Each flit
// is stored once, to its port's slot, after all four slots were cleared.
// Links in `edge` (leaving the CTA rectangle) are then copied from the slots
// to tagged global slots (store_edges; the single-simulation plain loop
// passes none and copies them after publishing its warp's flag).  `ic` is
// inj_candidate() of the tile's state.
__device__ __forceinline__ void route_ranked(const Params& P, Tile& T, uint32_t t, const uint4 (&in)[4],
                                             uint32_t exists, uint4* so, int so_stride, uint4* go,
                                             size_t go_stride, uint32_t edge, const InjCand& ic) {
  uint32_t vm = 0;
  unsigned long long k[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    vm |= (ftype(in[d]) != T_NONE ? 1u : 0u) << d;
    k[d] = fkey(P, in[d]);
  }
  const int n_arr = __popc(vm);
  // rank of each arrival among the valid ones: how many are older (keys are
  // unique: a tile injects at most one flit per cycle)
  uint32_t rk[4] = {0, 0, 0, 0};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a + 1; b < 4; ++b) {
      const bool lt = k[a] < k[b];
      rk[b] += (((vm >> a) & 1u) && lt) ? 1u : 0u;
      rk[a] += (((vm >> b) & 1u) && !lt) ? 1u : 0u;
    }
  uint32_t prod[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) prod[d] = prod_ports(P, fdst(in[d]), T.x, T.y);
  // eject the highest-priority arrival addressed to this tile: bit r of emr
  // is set when the arrival of rank r is addressed here
  uint32_t emr = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (((vm >> d) & 1u) && fdst(in[d]) == T.r) emr |= 1u << rk[d];
  // the lowest set bit's index; ~0u (above every rank) when none is set
  const uint32_t rej = 31u - (uint32_t)__clz(emr & (0u - emr));
  T.ej = make_uint4(0, 0, 0, 0);
  uint32_t rm = vm;
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (((vm >> d) & 1u) && rk[d] == rej) {
      T.ej = in[d];
      rm &= ~(1u << d);
    }
#pragma unroll
  for (int d = 0; d < 4; ++d) rk[d] -= rk[d] > rej ? 1u : 0u;
  // inject when an input port is free: the candidate taken off its queue
  uint4 inj = make_uint4(0, 0, 0, 0);
  const bool has_inj = ic.q != 0 && n_arr < __popc(exists);
  if (has_inj) {
    inj = ic.f;
    if (ic.q == 1) {
      T.sq_head = T.sq_head + 1 == (uint32_t)P.svc_q ? 0 : T.sq_head + 1;
      T.sq_len--;
      if (T.sq_len > 0) T.sq_front = P.sq[(size_t)T.r * P.svc_q + T.sq_head];
    } else {
      T.cq_head = T.cq_head + 1 == (uint32_t)P.core_q ? 0 : T.cq_head + 1;
      T.cq_len--;
      if (T.cq_len > 0) T.cq_front = P.cq[(size_t)T.r * P.core_q + T.cq_head];
    }
    inj.x = t;
    inj.y = (inj.y & 0xFFFF0000u) | T.r;
    T.inj++;
  }
  // ports in priority order: arrivals oldest first, then the injected flit.
  // The productive-port bytes are packed in rank order (byte r = the flit of
  // rank r), the grants come back packed by rank (nibble r), then by flit.
  uint32_t rp = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if ((rm >> d) & 1u) rp |= prod[d] << (8u * rk[d]);
  const uint32_t n_rem = __popc(rm);
  // over all four ranks: a rank past the remaining arrivals picks nothing
  uint32_t freem = exists, defl = 0, pkp = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint32_t pick = pick_port((rp >> (8 * r)) & 0xFFu, freem, (uint32_t)r < n_rem ? ~0u : 0u, defl);
    freem &= ~pick;
    pkp |= pick << (4 * r);
  }
  // grants are one-hot: a port's index is the position of its bit (31 - clz)
  uint32_t pk[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) pk[d] = (pkp >> (4u * rk[d])) & 15u;
  const uint32_t pki = pick_port(ic.prod, freem, has_inj ? ~0u : 0u, defl);
  freem &= ~pki;
  T.defl += defl;
  // every slot cleared, then each flit stored to the slot of its port
  const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int d = 0; d < 4; ++d) so[d * so_stride] = z;
  if (AGE1(P)) {
    // age_mode 1: a flit whose port is neither productive one ages by one
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if ((rm >> d) & 1u) {
        uint4 f = in[d];
        if (!(pk[d] & (prod[d] | (prod[d] >> 4)))) age_deflected(P, f, t);
        so[(31 - __clz(pk[d])) * so_stride] = f;
      }
    if (has_inj && !(pki & (ic.prod | (ic.prod >> 4)))) age_deflected(P, inj, t);
  } else {
#pragma unroll
    for (int d = 0; d < 4; ++d)
      if ((rm >> d) & 1u) so[(31 - __clz(pk[d])) * so_stride] = in[d];
  }
  if (has_inj) so[(31 - __clz(pki)) * so_stride] = inj;
  store_edges(so, so_stride, go, go_stride, edge, t);
}

// ---------------------------------------------------------------- Phase 3
template <int W1, int W2>
static __device__ void phase3(const Params& P, Tile& T, uint32_t t, uint32_t* sh_hist) {
  uint4 f = T.ej;
  uint32_t ty = ftype(f);
  if (ty == T_NONE) return;
  uint32_t lat = t - finject(P, f);
  T.ejc++;
  T.latsum += lat;
  if (lat > T.latmax) T.latmax = lat;
  atomicAdd(&sh_hist[lat < HIST_BINS - 1 ? lat : HIST_BINS - 1], 1u);

  // packet mode: the handler runs once, when the last flit of a packet is in
  if (PACKETS(P) && fe(f) > 1 && packet_flits(P, ty) > 1) {
    uint32_t* rb = P.rob + (size_t)T.r * P.rob_entries * 2;
    const uint32_t key = W_VALID | fline(f) | (ty << 26), src = fsrc(f);
    int hit = -1, free_slot = -1;
    for (int i = 0; i < P.rob_entries; ++i) {
      const uint32_t w0 = rb[2 * i];
      if (w0 == key && (rb[2 * i + 1] & 0xFFFFu) == src) hit = i;
      else if (!(w0 & W_VALID) && free_slot < 0) free_slot = i;
    }
    if (hit < 0) {
      if (free_slot < 0) {
        set_error(P, t, ERR_OVERFLOW);
        return;
      }
      hit = free_slot;
      rb[2 * hit] = key;
      rb[2 * hit + 1] = src;
    }
    const uint32_t cnt = (rb[2 * hit + 1] >> 16) + 1;
    if (cnt < fe(f)) {
      rb[2 * hit + 1] = src | (cnt << 16);
      return;
    }
    rb[2 * hit] = 0;
    rb[2 * hit + 1] = 0;
  }

  const uint32_t line = fline(f);
  const uint32_t set = l2_set(P, line);
  const size_t base = l2_base(P, T.r, set);
  switch (ty) {
    case T_PROBE:
      break;

    case T_REQ: {
      uint32_t q = fa(f);
      SMALL(S_REQR)++;
      uint32_t w[W2];
      load_set(P.l2 + base, L2WAYS(P), w);
      uint32_t fword;
      int way = set_find(w, L2WAYS(P), line, fword);
      if (way >= 0) {
        SMALL(S_L2H)++;
        set_touch(w, L2WAYS(P), way, fword);
        store_set(P.l2 + base, L2WAYS(P), w);
        send_svc(P, T, mkflit(T_DATA, T.r, q, line, 0, 0), t);
        if (POLICY(P) == POL_MIGRATE) {
          hist_push(P, base + way, q);
          uint16_t* hp = hist_ptr(P, base + way);
          uint32_t n = hp[0], cnt = 0;
          for (uint32_t i = 0; i < n; ++i) cnt += hp[2 + i] == q;
          if (n == (uint32_t)P.mig_window && cnt >= (uint32_t)P.mig_threshold && !hp[1]) {
            hp[1] = 1;
            SMALL(S_MIGS)++;
            send_svc(P, T, mkflit(T_MIG, T.r, q, line, 0, 0), t);
          }
        }
        break;
      }
      SMALL(S_L2M)++;
      if (POLICY(P) == POL_INTERLEAVED) {
        if (T.mq_len >= (uint32_t)P.mem_q) {
          set_error(P, t, ERR_OVERFLOW);
          break;
        }
        uint32_t slot = T.mq_head + T.mq_len;
        if (slot >= (uint32_t)P.mem_q) slot -= P.mem_q;
        uint4 m = make_uint4(t + (uint32_t)P.mem_lat, line, q, 0);
        P.mq[(size_t)T.r * P.mem_q + slot] = m;
        if (T.mq_len == 0) T.mq_front = m;
        T.mq_len++;
        SMALL(S_MEMREQ)++;
        break;
      }
      if (POLICY(P) == POL_MIGRATE) {
        // redirection (Sec. 3.3): the newest forward entry for the line
        const uint32_t* fw = P.fwd + (size_t)T.r * P.fwd_cap * 2;
        for (uint32_t i = 0; i < T.fwd_n; ++i) {
          int slot = ((int)T.fwd_next - 1 - (int)i) % P.fwd_cap;
          if (slot < 0) slot += P.fwd_cap;
          if (fw[slot * 2] == line) {
            uint32_t m = fw[slot * 2 + 1];
            if (m != q) {
              SMALL(S_REDIR)++;
              send_svc(P, T, mkflit(T_REQ, T.r, m, line, q, 0), t);
              return;
            }
            break;
          }
        }
      }
      SMALL(S_TRAP)++;
      send_svc(P, T, mkflit(T_NACK, T.r, q, line, 0, 0), t);
      break;
    }

    case T_DATA:
      SMALL(S_REPR)++;
      if (T.om_kind != OM_WAIT_DATA || T.om_line != line) {
        set_error(P, t, ERR_PROTOCOL);
        break;
      }
      l1_fill<W1, W2>(P, T, line, fsrc(f), T.om_write, t);
      l2lat_sample(T, t, T.om_start, sh_hist);
      set_om(T, OM_NONE, 0, 0, 0);
      break;

    case T_WT: {
      uint32_t w[W2];
      load_set(P.l2 + base, L2WAYS(P), w);
      uint32_t fword;
      int way = set_find(w, L2WAYS(P), line, fword);
      if (way >= 0) {
        set_touch(w, L2WAYS(P), way, fword, W_DIRTY);
        store_set(P.l2 + base, L2WAYS(P), w);
        SMALL(S_WTH)++;
      } else {
        SMALL(S_MEMW)++;
      }
      break;
    }

#if NOC_WITH_LSPD
    case T_DA: {
      if (!dir_owned(P, T, line, t)) break;
      uint32_t q = fsrc(f), D = P.dir[line];
      SMALL(S_DIRS)++;
      if (D == DIR_NONE || (D & 0xFFFFu) == q) {
        P.dir[line] = q | (fe(f) << 16);
        send_svc(P, T, mkflit(T_DRNEG, T.r, q, line, 0, fe(f)), t);
      } else {
        send_svc(P, T, mkflit(T_DRPOS, T.r, q, line, D & 0xFFFFu, 0), t);
      }
      break;
    }

    case T_DRNEG:
      SMALL(S_REPR)++;
      if (T.om_kind != OM_WAIT_DR || T.om_line != line) {
        set_error(P, t, ERR_PROTOCOL);
        break;
      }
      T.om_kind = OM_MEM_L2;
      T.om_timer = t + (uint32_t)P.mem_lat;
      T.om_epoch = fe(f);
      SMALL(S_MEMREQ)++;
      break;

    case T_DRPOS:
      SMALL(S_REPR)++;
      if (T.om_kind != OM_WAIT_DR || T.om_line != line) {
        set_error(P, t, ERR_PROTOCOL);
        break;
      }
      send_svc(P, T, mkflit(T_REQ, T.r, fa(f), line, T.r, 0), t);
      T.om_kind = OM_WAIT_DATA;
      break;

    case T_NACK:
      SMALL(S_REPR)++;
      if (T.om_kind != OM_WAIT_DATA || T.om_line != line) {
        set_error(P, t, ERR_PROTOCOL);
        break;
      }
      T.om_kind = OM_MEM_L1;
      T.om_timer = t + (uint32_t)P.mem_lat;
      SMALL(S_MEMREQ)++;
      break;

    case T_DINV:
      if (!dir_owned(P, T, line, t)) break;
      if (P.dir[line] == (fsrc(f) | (fe(f) << 16))) P.dir[line] = DIR_NONE;
      break;

    case T_MIG: {
      uint32_t o = fsrc(f);
      T.epoch = (T.epoch + 1) & 0xFFFFu;
      int way = l2_install<W2>(P, T, line, T.epoch, t);
      uint16_t* hp = hist_ptr(P, base + way);
      hp[0] = 0;
      hp[1] = 0;
      uint32_t h = dir_home(P, line);
      if (h == T.r) {
        P.dir[line] = T.r | (T.epoch << 16);
        SMALL(S_MIGR)++;
        send_svc(P, T, mkflit(T_INV, T.r, o, line, T.r, 0), t);
      } else {
        send_svc(P, T, mkflit(T_DIRUPD, T.r, h, line, o, T.epoch), t);
      }
      break;
    }

    case T_DIRUPD:
    case T_INV: {
      uint32_t m;
      if (ty == T_DIRUPD) {
        if (!dir_owned(P, T, line, t)) break;
        m = fsrc(f);
        uint32_t o = fa(f);
        P.dir[line] = m | (fe(f) << 16);
        SMALL(S_MIGR)++;
        if (o != T.r) {
          send_svc(P, T, mkflit(T_INV, T.r, o, line, m, 0), t);
          break;
        }
      } else {
        m = fa(f);
      }
      // invalidate the source copy and remember where the block went
      uint32_t w[W2];
      load_set(P.l2 + base, L2WAYS(P), w);
      uint32_t fword;
      int way = set_find(w, L2WAYS(P), line, fword);
      if (way >= 0) {
        if (fword & W_DIRTY) SMALL(S_MEMWB)++;
        set_invalidate(w, L2WAYS(P), way);
        store_set(P.l2 + base, L2WAYS(P), w);
        P.l2ep[base + way] = 0;
        uint16_t* hp = hist_ptr(P, base + way);
        hp[0] = 0;
        hp[1] = 0;
      }
      uint32_t* fw = P.fwd + (size_t)T.r * P.fwd_cap * 2;
      fw[T.fwd_next * 2] = line;
      fw[T.fwd_next * 2 + 1] = m;
      T.fwd_next = T.fwd_next + 1 == (uint32_t)P.fwd_cap ? 0 : T.fwd_next + 1;
      if (T.fwd_n < (uint32_t)P.fwd_cap) T.fwd_n++;
      break;
    }

#endif
    default:
      set_error(P, t, ERR_PROTOCOL);
  }
}

// ---------------------------------------------------------------- hash
// the dynamic-hash terms of a tile's partly received packets (packet mode):
// one fold(0x1A, r, line | type << 26, src | count << 16) per entry, summed
static __device__ unsigned long long rob_hash(const Params& P, uint32_t r) {
  unsigned long long h = 0;
  if (!PACKETS(P)) return 0;
  const uint32_t* rb = P.rob + (size_t)r * P.rob_entries * 2;
  for (int i = 0; i < P.rob_entries; ++i)
    if (rb[2 * i] & W_VALID)
      h += hfold(hfold(hfold(hstart(0x1A), r), rb[2 * i] & ~W_VALID), rb[2 * i + 1]);
  return h;
}
// whether a tile has no partly received packet
static __device__ bool rob_empty(const Params& P, uint32_t r) {
  if (!PACKETS(P)) return true;
  const uint32_t* rb = P.rob + (size_t)r * P.rob_entries * 2;
  for (int i = 0; i < P.rob_entries; ++i)
    if (rb[2 * i] & W_VALID) return false;
  return true;
}
// dynamic hash of one tile after a cycle: fold(r, its four output flits, its
// core record words C0..C6, injected, ejected, deflections); fields that mean
// nothing in the current FSM / outstanding-miss state hash as 0
static __device__ unsigned long long tile_hash(const Params& P, const Tile& T, const uint4 (&out)[4]) {
  unsigned long long h = hstart(T.r);
#pragma unroll
  for (int d = 0; d < 4; ++d) h = hflit(P, h, out[d]);
  bool busy = T.fsm != FSM_IDLE, wait = T.fsm == FSM_L2WAIT, om = T.om_kind != OM_NONE;
  bool mem = T.om_kind == OM_MEM_L2 || T.om_kind == OM_MEM_L1;
  h = hfold(h, T.next_ref);
  h = hfold(h, (unsigned long long)T.fsm | ((unsigned long long)(busy ? T.fsm_write : 0) << 8) |
                   ((unsigned long long)T.om_kind << 16) |
                   ((unsigned long long)(om ? T.om_write : 0) << 24) |
                   ((unsigned long long)T.epoch << 32));
  h = hfold(h, (unsigned long long)(busy ? T.fsm_line : 0) |
                   ((unsigned long long)(wait ? T.fsm_timer : 0) << 32));
  h = hfold(h, (unsigned long long)(wait ? T.fsm_start : 0) |
                   ((unsigned long long)(T.om_kind == OM_MEM_L2 ? T.om_epoch : 0) << 32));
  h = hfold(h, (unsigned long long)(om ? T.om_line : 0) |
                   ((unsigned long long)(mem ? T.om_timer : 0) << 32));
  h = hfold(h, om ? T.om_start : 0);
  h = hfold(h, (unsigned long long)T.cq_len | ((unsigned long long)T.sq_len << 16) |
                   ((unsigned long long)T.mq_len << 32) | ((unsigned long long)T.fwd_n << 48));
  h = hfold(h, T.inj);
  h = hfold(h, T.ejc);
  return hfold(h, T.defl);
}

}  // namespace noc
