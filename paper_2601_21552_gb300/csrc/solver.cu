// solver.cu -- GPU DPLL over batches of CNFs (the satisfiability step of
// Sec. V-B, step 10, applied to one query per static memory instruction).
//
// Layout in HBM (per batch, built by the prep kernels from the caller's CSR):
//   norm[L]        u32  normalised literal code per literal slot (2(v-1)+neg),
//                       NONE for dropped slots, UNIT_BIT for unit clauses
//   occ_begin[..]  u32  per instance 2V+1 offsets: occurrence list of each
//                       literal code (clauses that contain it)
//   ent[L]         u64  occurrence entries, in clause order within a list:
//                       binary (x|y) in x's list = {y, NONE}; ternary
//                       (x|y|z) in x's list = {y, z}; longer clauses =
//                       {LONG_CLAUSE|local clause index, 0}
//   units[C]       u32  unit-clause literal codes, compacted per instance
// Per worker slot (one warp): trail[Vmax], dstack[Vmax], act[Vmax] in global
// memory; the assignment (2 bits per variable) in shared memory.
//
// Search per instance (complete DPLL): unit propagation to a fixpoint over
// occurrence lists, frontier-parallel across the 32 lanes; on conflict bump
// the activity of the falsified clause's variables and backtrack
// chronologically to the deepest decision not yet flipped; otherwise decide
// the unassigned variable of highest activity (ties: lowest id), value false
// first. A busy warp hands the untried branch of its shallowest open decision
// to an idle warp (subtree splitting) so that hard instances spread over the
// whole GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/scuba.h"
#include "learn.cuh"
#include "scuba_internal.h"

namespace scuba {
namespace dev {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
constexpr uint32_t LONG_CLAUSE = 0x80000000u;
constexpr uint32_t UNIT_BIT = 0x40000000u;
constexpr uint32_t FLIP = 0x80000000u;
constexpr uint32_t F_EMPTY = 1u, F_BAD = 2u;
constexpr int MAX_PREFIX = 248;   // literals in a split job's prefix
// Learned clauses a clause-learning donor attaches to a cube: [count, words
// used, offset of each clause (JOB_CLS_MAX), records {len, lbd, literals}].
constexpr uint32_t JOB_CLS_MAX = 256, JOB_CLS_WORDS = 4096;
// Clause-learning records shared between the jobs of one instance: {seq,
// instance, len | lbd << 8, producer slot, up to SHARE_MAXLEN literals}.
constexpr uint32_t SHARE_REC = 16, SHARE_MAXLEN = 12;

__device__ __forceinline__ uint32_t code_of(int32_t l) {
  int32_t v = l > 0 ? l : -l;
  return 2u * (uint32_t)(v - 1) + (l < 0 ? 1u : 0u);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// --------------------------------------------------------------------------
// Prep
// --------------------------------------------------------------------------

struct Ctrl {
  uint32_t next_inst;   // fresh-instance counter
  uint32_t inst_left;   // instances not finished yet
  uint32_t idle;        // warps waiting for work
  int32_t status;       // first error (scuba status code)
  uint32_t q_head, q_tail;
  uint64_t t0;          // globaltimer at launch
  uint32_t jobs_split;  // statistics
  int32_t check_site;   // checked build: site of the first failed bounds check (0: none)
  uint64_t check_index; // ... the index it saw
  uint64_t check_limit; // ... and the bound it broke
};

__device__ void fail_batch(Ctrl* c, int32_t st) { atomicCAS(&c->status, 0, st); }

// Bounds checks of the checked build (-DSCUBA_CHECKED; compute-sanitizer is
// not available everywhere). SCUBA_IDX(ctrl, i, limit, site) is i when
// i < limit; otherwise the first failure records its site, index and bound,
// the call's status becomes SCUBA_ERR_INTERNAL and the access goes to index 0
// instead, so it stays inside its buffer (the call's results are void from
// then on). Without SCUBA_CHECKED the macro is the index itself.
#ifdef SCUBA_CHECKED
__device__ __noinline__ uint64_t check_fail(Ctrl* c, uint64_t i, uint64_t lim, int site) {
  if (atomicCAS(&c->check_site, 0, site) == 0) {
    c->check_index = i;
    c->check_limit = lim;
  }
  fail_batch(c, -8 /* SCUBA_ERR_INTERNAL */);
  return 0;
}
// The index expression is evaluated exactly once (it may be an atomicAdd).
template <class T>
__device__ __forceinline__ T checked_idx(Ctrl* c, T i, uint64_t lim, int site) {
  return (uint64_t)i < lim ? i : (T)check_fail(c, (uint64_t)i, lim, site);
}
#define SCUBA_IDX(ctrl, i, lim, site) \
  ::scuba::dev::checked_idx((ctrl), (i), (uint64_t)(lim), (site))
#else
#define SCUBA_IDX(ctrl, i, lim, site) (i)
#endif

__device__ __forceinline__ bool batch_failed(Ctrl* c) {
  return *(volatile int32_t*)&c->status != 0;
}

struct Prep {
  int n;
  int64_t C, L;
  int64_t total_vars;  // model size promised by the caller
  int64_t occ_cap;     // allocated occurrence-offset entries
  int32_t vmax;
  const int64_t* vb;
  Ctrl* ctrl;
  const int64_t* icb;
  const int64_t* cb;
  const int32_t* lits;
  const int32_t* nv;
  int64_t* occ_base;   // [n+1]
  uint32_t* norm;      // [L]
  uint32_t* occ_cnt;   // [occ_total] counts, then fill cursors
  uint32_t* occ_begin; // [occ_total]
  uint64_t* ent;       // [L]
  uint32_t* units;     // [C]
  uint32_t* nunits;    // [n]
  uint32_t* flags;     // [n]
};

__device__ __forceinline__ int32_t clamp_nv(int32_t v, int32_t vmax) {
  return v < 0 ? 0 : (v > vmax ? vmax : v);
}

// occ_base[i] = sum_{j<i} (2 nv[j] + 1); single block, chunked scan. Also
// validates the batch header: clause ranges monotonic and covering exactly
// [0, total_clauses), 0 <= nv <= max_vars, model ranges inside total_vars.
// Instances that fail get F_BAD; a header that cannot be trusted at all
// stops the whole batch with SCUBA_ERR_MALFORMED.
__global__ void k_occ_base(Prep P) {
  __shared__ int64_t part[1024];
  __shared__ int bad_header;
  const int n = P.n, t = threadIdx.x, T = blockDim.x;
  if (t == 0) bad_header = (P.icb[0] != 0 || P.icb[n] != P.C);
  __syncthreads();
  const int per = (n + T - 1) / T;
  const int b = min(n, t * per), e = min(n, b + per);
  int64_t s = 0;
  for (int i = b; i < e; i++) {
    const int32_t v = P.nv[i];
    if (P.icb[i] > P.icb[i + 1]) bad_header = 1;
    uint32_t f = 0;
    if (v < 0 || v > P.vmax) f |= F_BAD;
    // occurrence offsets are 32-bit within an instance
    const int64_t ca = P.icb[i], cz = P.icb[i + 1];
    if (ca >= 0 && cz >= ca && cz <= P.C && P.cb[cz] - P.cb[ca] >= (1LL << 32)) f |= F_BAD;
    if (P.vb[i] < 0 || P.vb[i] + (int64_t)(v < 0 ? 0 : v) > P.total_vars) f |= F_BAD;
    if (f) atomicOr(&P.flags[i], f);
    s += 2 * (int64_t)clamp_nv(v, P.vmax) + 1;
  }
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int k = 0; k < T; k++) {
      int64_t v = part[k];
      part[k] = acc;
      acc += v;
    }
    P.occ_base[n] = acc;
    if (acc > P.occ_cap) bad_header = 1;
  }
  __syncthreads();
  int64_t acc = part[t];
  for (int i = b; i < e; i++) {
    P.occ_base[i] = acc;
    acc += 2 * (int64_t)clamp_nv(P.nv[i], P.vmax) + 1;
  }
  if (t == 0 && bad_header) fail_batch(P.ctrl, SCUBA_ERR_MALFORMED);
}

__device__ __forceinline__ int find_inst(const int64_t* icb, int n, int64_t c) {
  int lo = 0, hi = n - 1;  // largest i with icb[i] <= c
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (icb[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One thread per clause: validate, normalise clauses of length <= 3
// (duplicates removed, tautologies dropped), count occurrences.
__global__ void k_normalize(Prep P) {
  if (batch_failed(P.ctrl)) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < P.C;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i = find_inst(P.icb, P.n, c);
    while (i + 1 < P.n && P.icb[i + 1] <= c) i++;  // skip empty instances
    const int V = clamp_nv(P.nv[i], P.vmax);
    const int64_t b = P.cb[c], e = P.cb[c + 1];
    if (b < 0 || e < b || e > P.L) { atomicOr(&P.flags[i], F_BAD); continue; }
    const int64_t len = e - b;
    bool bad = false;
    for (int64_t k = b; k < e; k++) {
      int32_t l = P.lits[k];
      if (l == 0 || l > V || l < -V) bad = true;
    }
    if (bad) {
      atomicOr(&P.flags[i], F_BAD);
      for (int64_t k = b; k < e; k++) P.norm[k] = NONE;
      continue;
    }
    if (len == 0) { atomicOr(&P.flags[i], F_EMPTY); continue; }
    uint32_t* cnt = P.occ_cnt + P.occ_base[i];
    if (len <= 3) {
      uint32_t u[3];
      int k = 0;
      bool taut = false;
      for (int64_t q = b; q < e; q++) {
        uint32_t x = code_of(P.lits[q]);
        bool dup = false;
        for (int r = 0; r < k; r++) {
          if (u[r] == x) dup = true;
          if (u[r] == (x ^ 1u)) taut = true;
        }
        P.norm[q] = dup ? NONE : x;
        if (!dup) u[k++] = x;
      }
      if (taut) {
        for (int64_t q = b; q < e; q++) P.norm[q] = NONE;
      } else if (k == 1) {
        for (int64_t q = b; q < e; q++)
          if (P.norm[q] != NONE) P.norm[q] |= UNIT_BIT;
      } else {
        for (int r = 0; r < k; r++) atomicAdd(&cnt[u[r]], 1u);
      }
    } else {
      for (int64_t q = b; q < e; q++) {
        uint32_t x = code_of(P.lits[q]);
        P.norm[q] = x;
        atomicAdd(&cnt[x], 1u);
      }
    }
  }
}

// One warp per instance: exclusive scan of the 2V counts -> occ_begin; the
// counts become fill cursors.
__global__ void k_occ_scan(Prep P) {
  if (batch_failed(P.ctrl)) return;
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int W = (gridDim.x * blockDim.x) >> 5;
  for (int i = w; i < P.n; i += W) {
    const int64_t base = P.occ_base[i];
    const uint32_t m = 2u * (uint32_t)clamp_nv(P.nv[i], P.vmax);
    uint32_t run = 0;
    for (uint32_t s = 0; s < m; s += 32) {
      uint32_t k = s + lane;
      uint32_t v = k < m ? P.occ_cnt[base + k] : 0u;
      uint32_t inc = v;
      for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, inc, d);
        if (lane >= d) inc += y;
      }
      if (k < m) {
        P.occ_begin[base + k] = run + inc - v;
        P.occ_cnt[base + k] = run + inc - v;
      }
      run += __shfl_sync(FULL, inc, 31);
    }
    if (lane == 0) P.occ_begin[base + m] = run;
  }
}

// One warp per instance: fill occurrence entries in clause order
// (deterministic), and compact the unit literals.
__global__ void k_fill(Prep P) {
  if (batch_failed(P.ctrl)) return;
  __shared__ uint32_t sbase[32 * 8];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t* my_base = sbase + 32 * wib;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int W = (gridDim.x * blockDim.x) >> 5;
  for (int i = w; i < P.n; i += W) {
    if (P.flags[i] & F_BAD) continue;
    const int64_t c0 = P.icb[i], c1 = P.icb[i + 1];
    const int64_t lbase = c0 < c1 ? P.cb[c0] : 0;
    uint32_t* cur = P.occ_cnt + P.occ_base[i];
    uint32_t nunit = 0;
    for (int64_t cs = c0; cs < c1; cs += 32) {
      const int64_t c = cs + lane;
      const bool valid = c < c1;
      int64_t b = 0, e = 0;
      uint32_t lits3[3] = {NONE, NONE, NONE};
      int nk = 0;
      bool is_long = false, is_unit = false;
      uint32_t unit_code = 0;
      if (valid) {
        b = P.cb[c];
        e = P.cb[c + 1];
        if (e - b > 3) {
          is_long = true;
          nk = (int)(e - b);
        } else {
          for (int64_t q = b; q < e; q++) {
            uint32_t x = P.norm[q];
            if (x == NONE) continue;
            if (x & UNIT_BIT) { is_unit = true; unit_code = x & ~UNIT_BIT; continue; }
            lits3[nk++] = x;
          }
          if (nk < 2) nk = 0;
        }
      }
      // units, in clause order
      uint32_t ub = __ballot_sync(FULL, is_unit);
      if (is_unit) P.units[c0 + nunit + __popc(ub & ((1u << lane) - 1u))] = unit_code;
      nunit += __popc(ub);
      int rounds = __reduce_max_sync(FULL, (unsigned)nk);
      for (int k = 0; k < rounds; k++) {
        const bool has = k < nk;
        uint32_t code = 0x80000000u | (uint32_t)lane;  // unique dummy
        uint64_t entry = 0;
        if (has) {
          if (is_long) {
            code = P.norm[b + k];
            entry = (uint64_t)(LONG_CLAUSE | (uint32_t)(c - c0));
          } else {
            code = lits3[k];
            uint32_t o1 = lits3[k == 0 ? 1 : 0];
            uint32_t o2 = nk == 3 ? lits3[k == 2 ? 1 : 2] : NONE;
            entry = (uint64_t)o1 | ((uint64_t)o2 << 32);
          }
        }
        uint32_t grp = __match_any_sync(FULL, code);
        int leader = __ffs(grp) - 1;
        if (has && lane == leader) {
          my_base[lane] = cur[code];
          cur[code] += __popc(grp);
        }
        __syncwarp();
        if (has) {
          uint32_t pos = my_base[leader] + __popc(grp & ((1u << lane) - 1u));
          P.ent[lbase + pos] = entry;
        }
        __syncwarp();
      }
    }
    if (lane == 0) P.nunits[i] = nunit;
  }
}

// --------------------------------------------------------------------------
// Solve
// --------------------------------------------------------------------------

struct Job {            // a DPLL subtree: the instance plus assumed literals
  int32_t inst;
  int32_t len;
  uint32_t lit[MAX_PREFIX];
  uint32_t seq;         // ring-buffer sequence number (Vyukov MPMC queue)
  float inc;            // donor's activity increment; its activities are in job_act
};

// Decision-trace buffers (training data for the branching network).
struct TraceDev {
  unsigned long long* cursor;  // [2]: nodes, rows reserved
  int64_t max_nodes, max_rows;
  int32_t* node_inst;
  int32_t* node_depth;
  int64_t* node_row;
  int32_t* node_nrows;
  int32_t* node_closed;
  __nv_bfloat16* x;            // [max_rows][NFEAT]
  float* target;               // [max_rows]
  int32_t* var;                // [max_rows]
};

enum { MODE_PLAIN = 0, MODE_TRACE = 1, MODE_LEARNED = 2, MODE_CDCL = 3 };

struct WList;  // a learned watch list (clause-learning mode)

struct Solve {
  int n;
  int32_t vmax;
  uint32_t assign_words;   // per-warp shared words (2 bits per variable)
  const int64_t* icb;
  const int64_t* cb;
  const int32_t* lits;
  const int32_t* nv;
  const int64_t* vb;
  const int64_t* occ_base;
  const uint32_t* occ_begin;
  const uint64_t* ent;
  const uint32_t* units;
  const uint32_t* nunits;
  const uint32_t* flags;
  const int32_t* order;
  // units: instance + assumption literals (solve_units); without a unit table
  // every instance is one unit with no assumptions
  int n_units;
  const int32_t* unit_inst;        // [n_units] or NULL (unit u is instance u)
  const int64_t* unit_asm_begin;   // [n_units+1] or NULL
  const int32_t* unit_asm;         // DIMACS assumption literals
  const int64_t* unit_vb;          // [n_units] model offset of each unit, or NULL
  uint8_t* verdict;
  uint8_t* model;
  int64_t* stats;
  // per instance bookkeeping
  uint32_t* pending;       // open jobs of an instance
  uint32_t* done;          // 1 once the verdict is final
  unsigned long long* inst_dec;  // decisions so far (budget)
  // per slot
  uint32_t* trail;
  uint32_t* dstack;
  float* act;
  // job ring
  Job* ring;
  float* job_act;          // [ring_cap x vmax] donor activity snapshot per cell
  uint32_t* prefix;        // [slots x MAX_PREFIX] the running job's assumptions
  uint32_t ring_cap;       // power of two
  int32_t split_min;       // decisions a job makes before it may donate
  int32_t split_depth;     // CDCL: cube levels below the instance a donor may reach
  Ctrl* ctrl;
  int64_t budget;
  uint64_t time_ns;
  const volatile int32_t* abort_flag;
  int split;
  int split_interval;
  int trail_smem;          // 1: each warp's trail lives in shared memory
  int64_t* finish_ns;      // optional [n]: completion time of each instance
  unsigned long long* prof;  // optional [8]: search counters
  // learned branching and trace recording
  const learn::MlpWeights* mlp;
  int learned_depth;           // MLP decides at decision depth < learned_depth
  const int32_t* inst_num_inputs;  // optional [n]: input bits (numbered first)
  int trace_depth;             // record decisions at depth < trace_depth
  TraceDev tr;
  uint32_t* lvlcnt;            // [slots][MAX_TRACE_DEPTH][vmax] conflict counts
  int64_t* lvl_node;           // [slots][MAX_TRACE_DEPTH] node of each open level
  // conflict-driven clause learning (per slot)
  uint4* cd_var;               // [slots][vmax] reason, trail position, level (16 B)
  uint8_t* cd_mark;            // [slots][vmax]
  WList* cd_wl;                // [slots][2 vmax] learned watch lists
  uint64_t* cd_pool;           // [slots][cd_pool_cap] watch entries
  uint32_t* cd_learnt;         // [slots][vmax]
  uint32_t* cd_arena;          // [slots][cd_arena_words]
  uint32_t* cd_clidx;          // [slots][cd_arena_words / 8] clause offsets
  int64_t cd_arena_words, cd_pool_cap;
  uint32_t* job_cls;           // [ring_cap][JOB_CLS_WORDS] clauses shared with a cube
  uint32_t* cls_copy;          // [slots][JOB_CLS_WORDS] a taken cube's clauses
  int restart_unit;            // conflicts per Luby unit
  // clauses shared between the jobs (cubes, units) of one instance: pool
  // (inst & share_mask) is a ring of share_cap records of SHARE_REC words
  uint32_t* share;             // [pools][share_cap][SHARE_REC]
  unsigned long long* share_cur;  // [pools] records reserved so far
  uint32_t share_mask;         // pools - 1 (a power of two)
  uint32_t share_cap;          // records per pool (a power of two)
  uint32_t share_lbd;          // publish learned clauses of LBD <= this; 0: off
};

struct WarpShared {
  uint32_t tail;
  uint32_t conflict;
  uint32_t cl[3];
  uint32_t pad[3];
  // per-job work counters (lane 0 updates them; kept out of registers)
  unsigned long long decisions, conflicts, props, visits, act_reads, undone;
  // clause-learning profile (cycles of lane 0 per phase; counts)
  unsigned long long cyc[8];
};

enum : uint32_t { LV_U = 0, LV_T = 1, LV_F = 2, LV_X = 3 };

__device__ __forceinline__ uint32_t lit_value(const uint32_t* asg, uint32_t l) {
  uint32_t v = l >> 1;
  uint32_t bits = (asg[v >> 4] >> ((v & 15u) * 2u)) & 3u;
  if (bits == 0u || bits == 3u) return bits == 0u ? LV_U : LV_X;
  // bits 1 = variable true, 2 = variable false
  bool lit_true = (bits == 1u) ^ ((l & 1u) != 0u);
  return lit_true ? LV_T : LV_F;
}

struct Warp {
  const Solve* S;
  uint32_t* asg;
  WarpShared* ws;
  uint32_t* trail;
  uint32_t* dstack;
  float* act;
  int lane;
  int inst;
  uint32_t V;
  const uint32_t* occ;
  const uint64_t* ent;
  const int64_t* cb;       // the caller's clause_begin (long clauses)
  const int32_t* lits;     // the caller's literals (long clauses)
  int64_t c0;
  uint32_t head;
  uint32_t nd;
  uint32_t nd_fixed;       // decisions below this index are assumptions
  float inc;
  uint32_t decisions;      // decisions of the current job
  uint32_t* lvlcnt;        // trace: per-level conflict counts of this slot
  int64_t* lvl_node;       // trace: node of each open level
  __nv_bfloat16* xtile;    // learned: 32 x NFEAT feature tile in shared memory
#ifdef SCUBA_CHECKED
  Ctrl* ck;                // where a failed bounds check is recorded
  uint32_t ent_end;        // occurrence entries of the instance (occ[2V])
#endif
};

// A checked index into a buffer of the current warp's instance.
#define WIDX(w, i, lim, site) SCUBA_IDX((w).ck, (i), (lim), (site))

// Checked build: the instance's bounds for WIDX (a no-op otherwise).
__device__ __forceinline__ void warp_checks(Warp& w, Ctrl* c) {
#ifdef SCUBA_CHECKED
  w.ck = c;
  w.ent_end = __ldg(&w.occ[2u * w.V]);
#else
  (void)w;
  (void)c;
#endif
}

#define WCOUNT(w, field, amount)                 \
  do {                                           \
    if ((w).lane == 0) (w).ws->field += (amount); \
  } while (0)

__device__ __forceinline__ void record_conflict(Warp& w, uint32_t a, uint32_t b, uint32_t c) {
  if (atomicCAS(&w.ws->conflict, 0u, 1u) == 0u) {
    w.ws->cl[0] = a;
    w.ws->cl[1] = b;
    w.ws->cl[2] = c;
  }
}

// Assign literal l true. Returns false on a clash with the opposite value.
__device__ __forceinline__ bool imply(Warp& w, uint32_t l) {
  uint32_t v = WIDX(w, l >> 1, w.V, 1);
  uint32_t sh = (v & 15u) * 2u;
  uint32_t mask = ((l & 1u) ? 2u : 1u) << sh;
  uint32_t old = atomicOr(&w.asg[v >> 4], mask);
  uint32_t ob = (old >> sh) & 3u;
  if (ob == 0u) {
    uint32_t pos = atomicAdd(&w.ws->tail, 1u);
    w.trail[WIDX(w, pos, w.V, 2)] = l;
    return true;
  }
  if (ob == (mask >> sh)) return true;
  if ((old & mask) == 0u) atomicAnd(&w.asg[v >> 4], ~mask);  // undo our bit
  return false;
}

__device__ void eval_long(Warp& w, uint32_t local, uint32_t f) {
  const int64_t c = w.c0 + local;
  const int64_t b = w.cb[c], e = w.cb[c + 1];
  uint32_t open_lit = NONE;
  int n_open = 0;
  for (int64_t q = b; q < e; q++) {
    uint32_t x = code_of(__ldg(&w.lits[q]));
    uint32_t vx = lit_value(w.asg, x);
    if (vx == LV_T || vx == LV_X) return;
    if (vx == LV_U && x != open_lit) {
      n_open++;
      open_lit = x;
      if (n_open > 1) return;
    }
  }
  if (n_open == 0) {
    record_conflict(w, LONG_CLAUSE | local, NONE, NONE);
  } else if (!imply(w, open_lit)) {
    record_conflict(w, LONG_CLAUSE | local, NONE, NONE);
  }
}

// Visit one occurrence entry of the falsified literal f.
__device__ __forceinline__ void eval_entry(Warp& w, uint32_t f, uint64_t e) {
  const uint32_t a0 = (uint32_t)e, b0 = (uint32_t)(e >> 32);
  if (a0 & LONG_CLAUSE) {
    eval_long(w, a0 & ~LONG_CLAUSE, f);
    return;
  }
  const uint32_t a = WIDX(w, a0, 2u * w.V, 3);
  const uint32_t b = b0 == NONE ? NONE : WIDX(w, b0, 2u * w.V, 3);
  const uint32_t va = lit_value(w.asg, a);
  if (b == NONE) {  // binary (f | a)
    if (va == LV_T || va == LV_X) return;
    if (va == LV_F || !imply(w, a)) record_conflict(w, f, a, NONE);
    return;
  }
  const uint32_t vb = lit_value(w.asg, b);  // ternary (f | a | b)
  if (va == LV_T || vb == LV_T || va == LV_X || vb == LV_X) return;
  if (va == LV_F && vb == LV_F) {
    record_conflict(w, f, a, b);
  } else if (va == LV_F) {
    if (!imply(w, b)) record_conflict(w, f, a, b);
  } else if (vb == LV_F) {
    if (!imply(w, a)) record_conflict(w, f, a, b);
  }
}

// Unit propagation to a fixpoint. Returns true on conflict.
// Each round takes the trail literals assigned in the previous round (the
// frontier) and spreads their occurrence entries over the 32 lanes:
// visit(f, entry) evaluates one occurrence entry of the falsified literal f;
// on_round(lo, hi) runs at the start of each round (frontier trail[lo, hi))
// and after_batch(base, count) after each batch of up to 32 frontier
// literals (all lanes, both).
template <class Visit, class Round, class Batch>
__device__ __forceinline__ bool bcp_rounds(Warp& w, Visit&& visit, Round&& on_round,
                                           Batch&& after_batch) {
  for (;;) {
    __syncwarp();
    const uint32_t hi = *(volatile uint32_t*)&w.ws->tail;
    if (w.head >= hi) return false;
    const uint32_t lo = w.head;
    w.head = hi;
    on_round(lo, hi);
    WCOUNT(w, props, hi - lo);
    for (uint32_t base = lo; base < hi; base += 32) {
      const uint32_t nlit = min(32u, hi - base);
      if (nlit == 1) {
        // one literal: every lane reads the same list bounds (broadcast)
        const uint32_t f = WIDX(w, w.trail[base] ^ 1u, 2u * w.V, 4);
        const uint32_t beg = __ldg(&w.occ[f]);
        const uint32_t cnt = __ldg(&w.occ[f + 1]) - beg;
        WCOUNT(w, visits, cnt);
        for (uint32_t e = w.lane; e < cnt; e += 32)
          visit(f, __ldg(&w.ent[WIDX(w, beg + e, w.ent_end, 5)]));
      } else {
        uint32_t f = 0, beg = 0, cnt = 0;
        if (w.lane < nlit) {
          f = WIDX(w, w.trail[base + w.lane] ^ 1u, 2u * w.V, 4);  // the literal that became false
          beg = __ldg(&w.occ[f]);
          cnt = __ldg(&w.occ[f + 1]) - beg;
        }
        uint32_t inc = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          uint32_t y = __shfl_up_sync(FULL, inc, d);
          if (w.lane >= d) inc += y;
        }
        const uint32_t excl = inc - cnt;
        const uint32_t total = __shfl_sync(FULL, inc, 31);
        WCOUNT(w, visits, total);
        if (total <= 32) {
          // owner of entry e = the lane whose segment starts at the last
          // segment start <= e: segment starts as a bit mask, ranks by popc
          const bool has = cnt > 0;
          const uint32_t starts = __reduce_or_sync(FULL, has ? (1u << excl) : 0u);
          const uint32_t nz = __ballot_sync(FULL, has);
          const uint32_t e = w.lane;
          int j = 0;
          if (e < total) {
            const int rank = __popc(starts & ((2u << e) - 1u)) - 1;
            j = __fns(nz, 0, rank + 1);
          }
          const uint32_t jbeg = __shfl_sync(FULL, beg, j);
          const uint32_t jex = __shfl_sync(FULL, excl, j);
          const uint32_t jf = __shfl_sync(FULL, f, j);
          if (e < total) visit(jf, __ldg(&w.ent[WIDX(w, jbeg + (e - jex), w.ent_end, 5)]));
        } else {
          for (uint32_t e0 = 0; e0 < total; e0 += 32) {
            const uint32_t e = e0 + w.lane;
            // owner = smallest lane j with inc_j > e
            int lo_j = 0, hi_j = 31;
#pragma unroll
            for (int s2 = 0; s2 < 5; s2++) {
              int mid = (lo_j + hi_j) >> 1;
              uint32_t v = __shfl_sync(FULL, inc, mid);
              if (v > e) hi_j = mid; else lo_j = mid + 1;
              if (lo_j > hi_j) lo_j = hi_j;
            }
            const int j = lo_j;
            const uint32_t jbeg = __shfl_sync(FULL, beg, j);
            const uint32_t jex = __shfl_sync(FULL, excl, j);
            const uint32_t jf = __shfl_sync(FULL, f, j);
            if (e < total) visit(jf, __ldg(&w.ent[WIDX(w, jbeg + (e - jex), w.ent_end, 5)]));
          }
        }
      }
      after_batch(base, nlit);
      __syncwarp();
      if (*(volatile uint32_t*)&w.ws->conflict) return true;
    }
  }
}

__device__ bool bcp(Warp& w) {
  return bcp_rounds(
      w, [&](uint32_t f, uint64_t e) { eval_entry(w, f, e); }, [](uint32_t, uint32_t) {},
      [](uint32_t, uint32_t) {});
}

template <int MODE>
__device__ void bump(Warp& w) {
  // activity += inc for the variables of the falsified clause
  const uint32_t a = w.ws->cl[0], b = w.ws->cl[1], c = w.ws->cl[2];
  if (MODE == MODE_TRACE) {
    // every open traced level counts the falsified clause's variables
    const uint32_t levels = min(w.nd, (uint32_t)w.S->trace_depth);
    if ((uint32_t)w.lane < levels) {
      uint32_t* cnt = w.lvlcnt + (size_t)w.lane * w.S->vmax;
      if (a & LONG_CLAUSE) {
        const int64_t cl = w.c0 + (a & ~LONG_CLAUSE);
        for (int64_t q = w.cb[cl]; q < w.cb[cl + 1]; q++) cnt[code_of(w.lits[q]) >> 1]++;
      } else {
        if (a != NONE) cnt[a >> 1]++;
        if (b != NONE) cnt[b >> 1]++;
        if (c != NONE) cnt[c >> 1]++;
      }
    }
    __syncwarp();
  }
  bool big = false;
  if (w.lane == 0) {
    if (a & LONG_CLAUSE) {
      const int64_t cl = w.c0 + (a & ~LONG_CLAUSE);
      for (int64_t q = w.cb[cl]; q < w.cb[cl + 1]; q++) {
        uint32_t v = code_of(w.lits[q]) >> 1;
        w.act[v] += w.inc;
        big |= w.act[v] > 1e20f;
      }
    } else {
      uint32_t x[3] = {a, b, c};
      for (int k = 0; k < 3; k++)
        if (x[k] != NONE) {
          uint32_t v = x[k] >> 1;
          w.act[v] += w.inc;
          big |= w.act[v] > 1e20f;
        }
    }
  }
  w.inc *= (1.0f / 0.95f);
  big = __shfl_sync(FULL, (int)big, 0) || w.inc > 1e20f;
  __syncwarp();
  if (big) {
    for (uint32_t v = w.lane; v < w.V; v += 32) w.act[v] *= 1e-20f;
    w.inc *= 1e-20f;
    __syncwarp();
  }
}

// ---- features of the residual formula (learned branching, traces) -------
//
// For variable v (0-based) and each polarity: how many clauses containing the
// literal are not yet satisfied with 2 / 3 open literals, its static
// occurrence count, plus activity, input-bit flags and search progress.
template <class Out>
__device__ void var_features(const Warp& w, uint32_t v, uint32_t ninputs, Out&& put) {
  uint32_t c2[2] = {0, 0}, c3[2] = {0, 0}, occn[2];
#pragma unroll
  for (int pol = 0; pol < 2; pol++) {
    const uint32_t lit = 2u * v + (uint32_t)pol;
    const uint32_t beg = __ldg(&w.occ[lit]), end = __ldg(&w.occ[lit + 1]);
    occn[pol] = end - beg;
    for (uint32_t e = beg; e < end; e++) {
      const uint64_t en = __ldg(&w.ent[e]);
      const uint32_t a = (uint32_t)en, b = (uint32_t)(en >> 32);
      if (a & LONG_CLAUSE) continue;
      const uint32_t va = lit_value(w.asg, a);
      if (va == LV_T || va == LV_X) continue;
      uint32_t open = 1 + (va == LV_U);
      if (b != NONE) {
        const uint32_t vb = lit_value(w.asg, b);
        if (vb == LV_T || vb == LV_X) continue;
        open += (vb == LV_U);
      }
      if (open == 2) c2[pol]++;
      else if (open == 3) c3[pol]++;
    }
  }
  const float tail = (float)*(volatile uint32_t*)&w.ws->tail;
  put(0, c2[0] * 0.25f);
  put(1, c3[0] * 0.25f);
  put(2, c2[1] * 0.25f);
  put(3, c3[1] * 0.25f);
  put(4, occn[0] * 0.125f);
  put(5, occn[1] * 0.125f);
  put(6, fminf(w.act[v] / w.inc, 16.0f) * 0.0625f);
  put(7, v < ninputs ? 1.0f : 0.0f);
  put(8, v < ninputs ? (float)v / (float)ninputs : 0.0f);
  put(9, (float)w.nd * (1.0f / 32.0f));
  put(10, w.V ? tail / (float)w.V : 0.0f);
  put(11, (c2[0] + c2[1]) * 0.125f);
  put(12, (c3[0] + c3[1]) * 0.125f);
  put(13, log2f(1.0f + occn[0] + occn[1]) * (1.0f / 6.0f));
  put(14, ((float)(c2[0] + c3[0]) - (float)(c2[1] + c3[1])) * 0.125f);
  put(15, 1.0f);
}

__device__ __forceinline__ bool var_unassigned(const uint32_t* asg, uint32_t v) {
  return ((asg[v >> 4] >> ((v & 15u) * 2u)) & 3u) == 0u;
}

// Trace: open a node for the decision about to be made at level `depth`.
__device__ void trace_open(Warp& w, uint32_t depth) {
  const Solve& S = *w.S;
  const TraceDev& T = S.tr;
  uint32_t nun = 0;
  for (uint32_t base = 0; base < w.V; base += 32) {
    const uint32_t v = base + w.lane;
    nun += __popc(__ballot_sync(FULL, v < w.V && var_unassigned(w.asg, v)));
  }
  long long node = -1, row0 = 0;
  if (w.lane == 0) {
    node = (long long)atomicAdd(&T.cursor[0], 1ull);
    row0 = (long long)atomicAdd(&T.cursor[1], (unsigned long long)nun);
    if (node >= T.max_nodes || row0 + nun > T.max_rows) node = -1;
  }
  node = __shfl_sync(FULL, node, 0);
  row0 = __shfl_sync(FULL, row0, 0);
  if (w.lane == 0) w.lvl_node[depth] = node;
  if (node < 0) return;
  if (w.lane == 0) {
    T.node_inst[node] = w.inst;
    T.node_depth[node] = (int32_t)depth;
    T.node_row[node] = row0;
    T.node_nrows[node] = (int32_t)nun;
    T.node_closed[node] = 0;
  }
  const uint32_t ni = S.inst_num_inputs ? (uint32_t)S.inst_num_inputs[w.inst] : 0u;
  long long r = row0;
  for (uint32_t base = 0; base < w.V; base += 32) {
    const uint32_t v = base + w.lane;
    const bool un = v < w.V && var_unassigned(w.asg, v);
    const uint32_t m = __ballot_sync(FULL, un);
    if (un) {
      const long long row = r + __popc(m & ((1u << w.lane) - 1u));
      __nv_bfloat16* xr = T.x + row * learn::NFEAT;
      var_features(w, v, ni, [&](int k, float x) { xr[k] = __float2bfloat16(x); });
      T.var[row] = (int32_t)v;
      T.target[row] = 0.0f;
    }
    r += __popc(m);
  }
  __syncwarp();
}

// Trace: the subtree of level l is finished; write its conflict counts.
__device__ void trace_close(Warp& w, uint32_t l) {
  const TraceDev& T = w.S->tr;
  const long long node = w.lvl_node[l];
  uint32_t* cnt = w.lvlcnt + (size_t)l * w.S->vmax;
  if (node >= 0) {
    const long long row0 = T.node_row[node];
    const int32_t nr = T.node_nrows[node];
    for (int k = w.lane; k < nr; k += 32) T.target[row0 + k] = (float)cnt[T.var[row0 + k]];
    __syncwarp();
    if (w.lane == 0) T.node_closed[node] = 1;
  }
  for (uint32_t v = w.lane; v < w.V; v += 32) cnt[v] = 0u;
  __syncwarp();
  if (w.lane == 0) w.lvl_node[l] = -1;
  __syncwarp();
}

// Learned decision: the unassigned variable with the highest MLP score
// (ties: higher activity, then lower id). NONE if all are assigned.
__device__ uint32_t pick_learned(Warp& w) {
  const Solve& S = *w.S;
  const uint32_t ni = S.inst_num_inputs ? (uint32_t)S.inst_num_inputs[w.inst] : 0u;
  float best_s = -INFINITY, best_a = -1.0f;
  uint32_t best_v = NONE;
  for (uint32_t base = 0; base < w.V; base += 32) {
    const uint32_t v = base + w.lane;
    const bool un = v < w.V && var_unassigned(w.asg, v);
    if (!__any_sync(FULL, un)) continue;
    __nv_bfloat16* xr = w.xtile + w.lane * learn::NFEAT;
    if (un) {
      var_features(w, v, ni, [&](int k, float x) { xr[k] = __float2bfloat16(x); });
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) xr[k] = __float2bfloat16(0.0f);
    }
    __syncwarp();
    float a_lo, a_hi, b_lo, b_hi;
    learn::mlp_tile_scores(S.mlp, w.xtile, w.lane, a_lo, a_hi);
    learn::mlp_tile_scores(S.mlp, w.xtile + 16 * learn::NFEAT, w.lane, b_lo, b_hi);
    // lane 4g holds rows g, g+8 (first tile) and 16+g, 24+g (second tile)
    const int src = 4 * (w.lane & 7);
    const float r0 = __shfl_sync(FULL, a_lo, src), r1 = __shfl_sync(FULL, a_hi, src);
    const float r2 = __shfl_sync(FULL, b_lo, src), r3 = __shfl_sync(FULL, b_hi, src);
    const float sc = w.lane < 8 ? r0 : (w.lane < 16 ? r1 : (w.lane < 24 ? r2 : r3));
    if (un) {
      const float a = w.act[v];
      if (sc > best_s || (sc == best_s && (a > best_a || (a == best_a && v < best_v)))) {
        best_s = sc;
        best_a = a;
        best_v = v;
      }
    }
    __syncwarp();
  }
  for (int d = 16; d > 0; d >>= 1) {
    const float os = __shfl_xor_sync(FULL, best_s, d), oa = __shfl_xor_sync(FULL, best_a, d);
    const uint32_t ov = __shfl_xor_sync(FULL, best_v, d);
    if (os > best_s || (os == best_s && (oa > best_a || (oa == best_a && ov < best_v)))) {
      best_s = os;
      best_a = oa;
      best_v = ov;
    }
  }
  return best_v;
}

// Chronological backtrack after a conflict. Returns false when no decision
// above the assumptions is left to flip (the subtree is refuted).
template <int MODE>
__device__ bool backtrack(Warp& w) {
  uint32_t nd = w.nd;
  if (w.lane == 0)
    while (nd > w.nd_fixed && (w.dstack[nd - 1] & FLIP)) nd--;
  nd = __shfl_sync(FULL, nd, 0);
  __syncwarp();
  if (nd <= w.nd_fixed) return false;
  if (MODE == MODE_TRACE) {
    // levels nd .. w.nd-1 are popped: their subtrees are complete
    const uint32_t hi_l = min(w.nd, (uint32_t)w.S->trace_depth);
    for (uint32_t l = nd; l < hi_l; l++) trace_close(w, l);
  }
  const uint32_t pos = w.dstack[nd - 1] & ~FLIP;
  const uint32_t tail = *(volatile uint32_t*)&w.ws->tail;
  const uint32_t d = w.trail[pos];
  WCOUNT(w, undone, tail - pos);
  for (uint32_t t = pos + w.lane; t < tail; t += 32) {
    uint32_t v = w.trail[t] >> 1;
    atomicAnd(&w.asg[v >> 4], ~(3u << ((v & 15u) * 2u)));
  }
  __syncwarp();
  if (w.lane == 0) {
    w.dstack[nd - 1] |= FLIP;
    w.ws->tail = pos;
    w.ws->conflict = 0;
  }
  __syncwarp();
  w.nd = nd;
  w.head = pos;
  if (w.lane == 0) imply(w, d ^ 1u);
  __syncwarp();
  return true;
}

// Highest-activity unassigned variable (ties: lowest id); NONE if all assigned.
__device__ uint32_t pick(Warp& w) {
  float best_a = -1.0f;
  uint32_t best_v = NONE;
  const uint32_t nwords = (w.V + 15u) >> 4;
  for (uint32_t k = w.lane; k < nwords; k += 32) {
    const uint32_t word = w.asg[k];
    uint32_t un = ~(word | (word >> 1)) & 0x55555555u;  // 00 pairs
    const uint32_t lim = w.V - 16u * k;
    if (lim < 16u) un &= (1u << (2u * lim)) - 1u;
    while (un) {
      const uint32_t bitpos = __ffs(un) - 1;
      un &= un - 1u;
      const uint32_t v = 16u * k + (bitpos >> 1);
      const float a = w.act[v];
      if (a > best_a || (a == best_a && v < best_v)) {
        best_a = a;
        best_v = v;
      }
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    float oa = __shfl_xor_sync(FULL, best_a, d);
    uint32_t ov = __shfl_xor_sync(FULL, best_v, d);
    if (oa > best_a || (oa == best_a && ov < best_v)) {
      best_a = oa;
      best_v = ov;
    }
  }
  return best_v;
}

__device__ __forceinline__ void set_status(const Solve& S, int32_t st) {
  atomicCAS(&S.ctrl->status, 0, st);
}

// ---- job ring (bounded MPMC queue, Vyukov) --------------------------------

// extra(cell) runs (all lanes) after the cell is filled and before it is
// published: the clause-learning search attaches learned clauses there.
template <class Extra>
__device__ bool ring_push(const Solve& S, const Warp& w, int inst, uint32_t plen,
                          const uint32_t* prefix_src_trail, const uint32_t* dpos,
                          uint32_t flip_index, Extra&& extra) {
  // called by all lanes; lane 0 reserves
  Ctrl* C = S.ctrl;
  uint32_t slot = NONE;
  if (w.lane == 0) {
    for (int it = 0; it < 64; it++) {
      uint32_t pos = *(volatile uint32_t*)&C->q_tail;
      Job* cell = &S.ring[pos & (S.ring_cap - 1)];
      uint32_t seq = *(volatile uint32_t*)&cell->seq;
      int32_t dif = (int32_t)(seq - pos);
      if (dif == 0) {
        if (atomicCAS(&C->q_tail, pos, pos + 1) == pos) { slot = pos; break; }
      } else if (dif < 0) {
        break;  // full
      }
    }
  }
  slot = __shfl_sync(FULL, slot, 0);
  if (slot == NONE) return false;
  Job* cell = &S.ring[slot & (S.ring_cap - 1)];
  // prefix = decision literals 0..flip_index-1 as assigned now, then the
  // negation of decision flip_index
  for (uint32_t k = w.lane; k < plen; k += 32) {
    uint32_t lit = prefix_src_trail[dpos[k] & ~FLIP];
    if (k == flip_index) lit ^= 1u;
    cell->lit[k] = lit;
  }
  // the thief continues with the donor's activity ordering
  float* snap = S.job_act + (size_t)(slot & (S.ring_cap - 1)) * S.vmax;
  for (uint32_t v = w.lane; v < w.V; v += 32) snap[v] = w.act[v];
  if (w.lane == 0) {
    cell->inst = inst;
    cell->len = (int32_t)plen;
    cell->inc = w.inc;
  }
  extra(slot & (S.ring_cap - 1));
  __threadfence();
  __syncwarp();
  if (w.lane == 0) atomicExch(&cell->seq, slot + 1);
  __syncwarp();
  return true;
}

__device__ bool ring_push(const Solve& S, const Warp& w, int inst, uint32_t plen,
                          const uint32_t* prefix_src_trail, const uint32_t* dpos,
                          uint32_t flip_index) {
  return ring_push(S, w, inst, plen, prefix_src_trail, dpos, flip_index, [](uint32_t) {});
}

// Try to take a job; returns slot or NONE.
__device__ uint32_t ring_pop(const Solve& S, int lane) {
  Ctrl* C = S.ctrl;
  uint32_t slot = NONE;
  if (lane == 0) {
    for (int it = 0; it < 64; it++) {
      uint32_t pos = *(volatile uint32_t*)&C->q_head;
      Job* cell = &S.ring[pos & (S.ring_cap - 1)];
      uint32_t seq = *(volatile uint32_t*)&cell->seq;
      int32_t dif = (int32_t)(seq - (pos + 1));
      if (dif == 0) {
        if (atomicCAS(&C->q_head, pos, pos + 1) == pos) { slot = pos; break; }
      } else if (dif < 0) {
        break;  // empty
      }
    }
    __threadfence();  // acquire: the cell's contents after its sequence number
  }
  slot = __shfl_sync(FULL, slot, 0);
  __syncwarp();
  return slot;
}

__device__ void ring_release(const Solve& S, uint32_t slot, int lane) {
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    atomicExch(&S.ring[slot & (S.ring_cap - 1)].seq, slot + S.ring_cap);
  }
  __syncwarp();
}

// A unit's job finished with result r (SCUBA_SAT / SCUBA_UNSAT /
// SCUBA_UNKNOWN). The last open job of a unit (an instance, or an instance
// under assumptions) writes its verdict.
__device__ void finish_job(const Solve& S, Warp& w, int unit, int r) {
  if (w.lane == 0) {
    if (r == SCUBA_SAT) {
      S.verdict[unit] = SCUBA_SAT;
      atomicOr(&S.done[unit], 1u);
    } else if (r == SCUBA_UNKNOWN) {
      atomicOr(&S.done[unit], 2u);  // mark: some subtree gave up
    }
    uint32_t left = atomicSub(&S.pending[unit], 1u) - 1u;
    if (left == 0u) {
      uint32_t d = atomicOr(&S.done[unit], 4u);
      if (!(d & 1u)) S.verdict[unit] = (d & 2u) ? SCUBA_UNKNOWN : SCUBA_UNSAT;
      atomicSub(&S.ctrl->inst_left, 1u);
      if (S.finish_ns) S.finish_ns[unit] = (int64_t)(globaltimer() - S.ctrl->t0);
    }
    if (S.prof) {
      atomicAdd(&S.prof[1], 1ull);  // jobs run
      for (int k = 0; k < 8; k++)
        if (w.ws->cyc[k]) atomicAdd(&S.prof[8 + k], w.ws->cyc[k]);
    }
    if (S.stats) {
      unsigned long long* st = (unsigned long long*)&S.stats[SCUBA_NSTATS * (int64_t)unit];
      atomicAdd(st + 0, w.ws->decisions);
      atomicAdd(st + 1, w.ws->conflicts);
      atomicAdd(st + 2, w.ws->props);
      atomicAdd(st + 3, w.ws->visits);
      atomicAdd(st + 4, w.ws->act_reads);
      atomicAdd(st + 5, w.ws->undone);
    }
  }
  __syncwarp();
}

// Solve one subtree (inst + assumptions). Returns SAT / UNSAT / UNKNOWN.
// A taken job (a shared subtree) in slot-private memory: the ring cell is
// released as soon as it has been copied.
struct TakenJob {
  const uint32_t* lit;  // assumptions, in order
  int32_t len;
  float inc;            // activities were copied into the warp's act[] already
  const uint32_t* cls;  // clause learning: the donor's clauses (slot copy), or NULL
};

template <int MODE>
__device__ int run_job_body(const Solve& S, Warp& w, int unit, int inst, const TakenJob* job,
                            int& abort_code);

// A unit's assumption literals as the job of a fresh search (all lanes):
// converted into the slot's prefix buffer, activities zeroed. Returns true
// if a literal is out of range or there are more than MAX_PREFIX of them.
__device__ __noinline__ bool unit_job(const Solve& S, int unit, int inst, int64_t slot, int lane,
                                      float* act, TakenJob* out) {
  const int64_t ab = S.unit_asm_begin[unit], ae = S.unit_asm_begin[unit + 1];
  const int32_t V = min(S.nv[inst], S.vmax);
  bool bad = ae - ab > MAX_PREFIX;
  uint32_t* pre = S.prefix + slot * MAX_PREFIX;
  for (int64_t q = ab + lane; !bad && q < ae; q += 32) {
    const int32_t l = S.unit_asm[q];
    if (l == 0 || l > V || l < -V) bad = true;
    else pre[q - ab] = code_of(l);
  }
  bad = __any_sync(FULL, bad);
  for (int v = lane; v < V; v += 32) act[v] = 0.0f;  // fresh activities
  out->lit = pre;
  out->len = (int32_t)(ae - ab < MAX_PREFIX ? ae - ab : MAX_PREFIX);
  out->inc = 1.0f;
  out->cls = nullptr;
  __syncwarp();
  return bad;
}

// Runs one job; in trace mode every level still open at the end is closed.
template <int MODE>
__device__ int run_job(const Solve& S, Warp& w, int unit, int inst, const TakenJob* job,
                       int& abort_code) {
  const int r = run_job_body<MODE>(S, w, unit, inst, job, abort_code);
  if (MODE == MODE_TRACE) {
    const uint32_t hi_l = min(w.nd, (uint32_t)S.trace_depth);
    for (uint32_t l = 0; l < hi_l; l++) trace_close(w, l);
  }
  return r;
}

template <int MODE>
__device__ int run_job_body(const Solve& S, Warp& w, int unit, int inst, const TakenJob* job,
                            int& abort_code) {
  w.inst = inst;
  w.V = (uint32_t)S.nv[inst];
  w.c0 = S.icb[inst];
  w.occ = S.occ_begin + S.occ_base[inst];
  const int64_t lbase = S.icb[inst] < S.icb[inst + 1] ? S.cb[S.icb[inst]] : 0;
  w.ent = S.ent + lbase;
  warp_checks(w, S.ctrl);
  w.head = 0;
  w.nd = 0;
  w.nd_fixed = 0;
  w.inc = 1.0f;
  const uint32_t nwords = (w.V + 15u) >> 4;
  for (uint32_t k = w.lane; k < nwords; k += 32) w.asg[k] = 0u;
  if (job) {
    w.inc = job->inc;
  } else {
    for (uint32_t v = w.lane; v < w.V; v += 32) w.act[v] = 0.0f;
  }
  if (w.lane == 0) {
    w.ws->tail = 0;
    w.ws->conflict = 0;
  }
  __syncwarp();
  if (S.flags[inst] & F_EMPTY) return SCUBA_UNSAT;
  // level 0: unit clauses, then the job's assumptions as fixed decisions
  const uint32_t nu = S.nunits[inst];
  const uint32_t* un = S.units + w.c0;
  for (uint32_t k = w.lane; k < nu; k += 32)
    if (!imply(w, un[k])) record_conflict(w, un[k], NONE, NONE);
  __syncwarp();
  if (w.ws->conflict) return SCUBA_UNSAT;
  if (job) {
    for (int k = 0; k < job->len; k++) {
      if (bcp(w)) return SCUBA_UNSAT;
      const uint32_t l = job->lit[k];
      const uint32_t val = lit_value(w.asg, l);
      if (val == LV_F) return SCUBA_UNSAT;
      if (val == LV_T) continue;
      if (w.lane == 0) {
        w.dstack[WIDX(w, w.nd, (uint32_t)w.S->vmax, 6)] = *(volatile uint32_t*)&w.ws->tail | FLIP;
        imply(w, l);
      }
      w.nd++;
      __syncwarp();
    }
    w.nd_fixed = w.nd;
  }
  uint32_t iter = 0;
  for (;;) {
    if ((++iter & 63u) == 0u) {
      int stop = 0;
      if (w.lane == 0) {
        if (S.abort_flag && *S.abort_flag) stop = 1;
        else if (globaltimer() - S.ctrl->t0 > S.time_ns) stop = 2;
        else if (*(volatile uint32_t*)&S.done[unit] & 1u) stop = 3;  // solved elsewhere
#ifdef SCUBA_CHECKED
        else if (batch_failed(S.ctrl)) stop = 4;  // a bounds check failed: stop
#endif
      }
      stop = __shfl_sync(FULL, stop, 0);
      if (stop == 4) { abort_code = SCUBA_ERR_INTERNAL; return SCUBA_UNKNOWN; }
      if (stop == 1) { abort_code = SCUBA_ERR_ABORTED; return SCUBA_UNKNOWN; }
      if (stop == 2) { abort_code = SCUBA_ERR_TIMEOUT; return SCUBA_UNKNOWN; }
      if (stop == 3) return SCUBA_UNSAT;  // the instance is SAT already; this subtree is moot
    }
    if (bcp(w)) {
      WCOUNT(w, conflicts, 1);
      bump<MODE>(w);
      if (!backtrack<MODE>(w)) return SCUBA_UNSAT;
      continue;
    }
    WCOUNT(w, act_reads, w.V - *(volatile uint32_t*)&w.ws->tail);
    uint32_t v;
    if (MODE == MODE_LEARNED && w.nd < (uint32_t)S.learned_depth) v = pick_learned(w);
    else v = pick(w);
    if (MODE == MODE_TRACE && v != NONE && w.nd < (uint32_t)S.trace_depth) trace_open(w, w.nd);
    if (v == NONE) {
      // the first subtree of the instance to reach a model writes it
      uint32_t won = 0;
      if (w.lane == 0) won = !(atomicOr(&S.done[unit], 8u) & 8u);
      won = __shfl_sync(FULL, won, 0);
      if (won && S.model)
        for (uint32_t x = w.lane; x < w.V; x += 32) {
          uint32_t bits = (w.asg[x >> 4] >> ((x & 15u) * 2u)) & 3u;
          S.model[(S.unit_vb ? S.unit_vb[unit] : S.vb[inst]) + x] = bits == 1u ? 1 : 0;
        }
      __syncwarp();
      return SCUBA_SAT;
    }
    // budget: decisions of the instance across all of its subtrees
    if (S.budget > 0 && (w.decisions & 255) == 0) {
      unsigned long long tot = 0;
      if (w.lane == 0) tot = atomicAdd(&S.inst_dec[unit], 256ull);
      tot = __shfl_sync(FULL, tot, 0);
      if ((int64_t)tot >= S.budget) return SCUBA_UNKNOWN;
    }
    // share the untried branch of the shallowest open decision
    if (S.split && w.decisions >= S.split_min && (w.decisions % S.split_interval) == 0 &&
        w.nd > w.nd_fixed) {
      uint32_t idle = 0;
      if (w.lane == 0) idle = *(volatile uint32_t*)&S.ctrl->idle;
      idle = __shfl_sync(FULL, idle, 0);
      if (idle > 0) {
        uint32_t k = w.nd_fixed;
        if (w.lane == 0)
          while (k < w.nd && (w.dstack[k] & FLIP)) k++;
        k = __shfl_sync(FULL, k, 0);
        if (k < w.nd && k + 1 <= (uint32_t)MAX_PREFIX) {
          if (w.lane == 0) atomicAdd(&S.pending[unit], 1u);
          __syncwarp();
          if (ring_push(S, w, unit, k + 1, w.trail, w.dstack, k)) {
            if (w.lane == 0) {
              w.dstack[k] |= FLIP;
              atomicAdd(&S.ctrl->jobs_split, 1u);
              if (S.prof) {
                atomicAdd(&S.prof[0], 1ull);                       // jobs shared
                atomicAdd(&S.prof[2], (unsigned long long)(k + 1)); // prefix literals
                atomicAdd(&S.prof[3], (unsigned long long)(w.nd - k)); // depth left
              }
            }
          } else if (w.lane == 0) {
            atomicSub(&S.pending[unit], 1u);
            if (S.prof) atomicAdd(&S.prof[4], 1ull);  // ring full
          }
          __syncwarp();
        }
      }
    }
    w.decisions++;
    WCOUNT(w, decisions, 1);
    if (w.lane == 0) {
      w.dstack[WIDX(w, w.nd, (uint32_t)w.S->vmax, 6)] = *(volatile uint32_t*)&w.ws->tail;
      imply(w, 2u * v + 1u);  // false first
    }
    w.nd++;
    __syncwarp();
  }
}

#include "cdcl.cuh"

// Plain search: 48 registers per thread, 5 blocks x 8 warps = 40 resident
// warps per SM. The learned variant (MLP on the tensor cores) defaults to 4
// blocks (64 registers); SCUBA_LEARNED_MINBLOCKS=5 trades spills for warps
// (measured slower). The clause-learning variant runs 2 blocks (116
// registers, no spills): measured faster than 3 (80 registers) or 4 (64,
// spilling) on partition queries and on random 3-SAT.
#ifndef SCUBA_LEARNED_MINBLOCKS
#define SCUBA_LEARNED_MINBLOCKS 4
#endif
#ifndef SCUBA_CDCL_MINBLOCKS
#define SCUBA_CDCL_MINBLOCKS 2
#endif
template <int MODE>
__global__ void __launch_bounds__(256, MODE == MODE_LEARNED ? SCUBA_LEARNED_MINBLOCKS
                                       : MODE == MODE_CDCL  ? SCUBA_CDCL_MINBLOCKS
                                                            : 5)
    k_solve(const __grid_constant__ Solve S) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t slot = (int64_t)blockIdx.x * wpb + wib;
  WarpShared* wsh = reinterpret_cast<WarpShared*>(smem);
  Warp w;
  w.S = &S;
  w.ws = &wsh[wib];
  w.asg = smem + (sizeof(WarpShared) / 4) * wpb + (size_t)S.assign_words * wib;
  w.trail = S.trail_smem
                ? smem + (sizeof(WarpShared) / 4) * wpb + (size_t)S.assign_words * wpb +
                      (size_t)S.vmax * wib
                : S.trail + slot * S.vmax;
  w.dstack = S.dstack + slot * S.vmax;
  w.act = S.act + slot * S.vmax;
  w.cb = S.cb;
  w.lits = S.lits;
  w.lane = lane;
  w.lvlcnt = nullptr;
  w.lvl_node = nullptr;
  w.xtile = nullptr;
  if (MODE == MODE_TRACE) {
    w.lvlcnt = S.lvlcnt + (size_t)slot * learn::MAX_TRACE_DEPTH * S.vmax;
    w.lvl_node = S.lvl_node + (size_t)slot * learn::MAX_TRACE_DEPTH;
  }
  if (MODE == MODE_LEARNED) {
    // feature tile after the per-warp assignment (and trail) areas
    unsigned char* tiles = reinterpret_cast<unsigned char*>(
        smem + (sizeof(WarpShared) / 4) * wpb + (size_t)S.assign_words * wpb +
        (S.trail_smem ? (size_t)S.vmax * wpb : 0));
    w.xtile = reinterpret_cast<__nv_bfloat16*>(tiles) + (size_t)wib * 32 * learn::NFEAT;
  }
  uint2* ring = nullptr;
  if (MODE == MODE_CDCL) {
    // recent-trail ring and analysis queue after the per-warp assignment (and
    // trail) areas, 16-byte aligned
    const size_t off = ((sizeof(WarpShared) / 4) * wpb + (size_t)S.assign_words * wpb +
                        (S.trail_smem ? (size_t)S.vmax * wpb : 0)) * 4;
    ring = reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(smem) +
                                    ((off + 15) & ~(size_t)15) + (size_t)wib * CD_SMEM_WARP);
  }
  if (batch_failed(S.ctrl)) return;
  bool counted_idle = false;
  for (;;) {
    // 1) a shared subtree, 2) a fresh unit (an instance, possibly under
    // assumptions), 3) wait for shared work
    int inst = -1, unit = -1;
    bool bad_unit = false;
    uint32_t slot_j = ring_pop(S, lane);
    TakenJob taken;
    const TakenJob* job = nullptr;
    if (slot_j != NONE) {
      // copy the cell out (prefix, activity snapshot) and release it at once
      const Job* cell = &S.ring[slot_j & (S.ring_cap - 1)];
      unit = cell->inst;
      inst = S.unit_inst ? S.unit_inst[unit] : unit;
      const int32_t len = cell->len;
      uint32_t* pre = S.prefix + slot * MAX_PREFIX;
      for (int k = lane; k < len; k += 32) pre[k] = cell->lit[k];
      const float* snap = S.job_act + (size_t)(slot_j & (S.ring_cap - 1)) * S.vmax;
      const int32_t V = min(S.nv[inst], S.vmax);
      for (int v = lane; v < V; v += 32) w.act[v] = snap[v];
      taken.lit = pre;
      taken.len = len;
      taken.inc = cell->inc;
      taken.cls = nullptr;
      if (MODE == MODE_CDCL) {  // the donor's learned clauses, copied out too
        const uint32_t* src = S.job_cls + (size_t)(slot_j & (S.ring_cap - 1)) * JOB_CLS_WORDS;
        uint32_t* dst = S.cls_copy + slot * JOB_CLS_WORDS;
        const uint32_t words = min(src[1], JOB_CLS_WORDS);
        for (uint32_t k = lane; k < words; k += 32) dst[k] = src[k];
        taken.cls = dst;
      }
      __syncwarp();
      ring_release(S, slot_j, lane);
      job = &taken;
    } else {
      uint32_t k = 0;
      if (lane == 0) k = atomicAdd(&S.ctrl->next_inst, 1u);
      k = __shfl_sync(FULL, k, 0);
      if (k < (uint32_t)S.n_units) {
        unit = S.order ? S.order[k] : (int)k;
        inst = S.unit_inst ? S.unit_inst[unit] : unit;
        if (inst < 0 || inst >= S.n) {
          bad_unit = true;
          inst = 0;
        } else if (S.unit_asm_begin &&
                   S.unit_asm_begin[unit + 1] > S.unit_asm_begin[unit]) {
          bad_unit = unit_job(S, unit, inst, slot, lane, w.act, &taken);
          job = &taken;
        }
      } else {
        if (!counted_idle) {
          if (lane == 0) atomicAdd(&S.ctrl->idle, 1u);
          counted_idle = true;
        }
        int stop = 0;
        if (lane == 0) {
          if (*(volatile uint32_t*)&S.ctrl->inst_left == 0u) stop = 1;
          else if (*(volatile int32_t*)&S.ctrl->status != 0) stop = 1;
          else if (S.abort_flag && *S.abort_flag) { stop = 1; set_status(S, SCUBA_ERR_ABORTED); }
          else if (globaltimer() - S.ctrl->t0 > S.time_ns) { stop = 1; set_status(S, SCUBA_ERR_TIMEOUT); }
          else {
            if (S.prof) atomicAdd(&S.prof[5], 1ull);  // idle polls
            __nanosleep(2000);
          }
        }
        stop = __shfl_sync(FULL, stop, 0);
        if (stop) break;
        continue;
      }
    }
    if (counted_idle) {
      if (lane == 0) atomicSub(&S.ctrl->idle, 1u);
      counted_idle = false;
    }
    int abort_code = 0;
    int r;
    w.decisions = 0;
    if (lane == 0) {
      w.ws->decisions = w.ws->conflicts = w.ws->props = 0;
      w.ws->visits = w.ws->act_reads = w.ws->undone = 0;
      for (int k = 0; k < 8; k++) w.ws->cyc[k] = 0;
    }
    __syncwarp();
    uint32_t moot = 0;
    if (lane == 0) moot = *(volatile uint32_t*)&S.done[unit] & 1u;
    moot = __shfl_sync(FULL, moot, 0);
    if (bad_unit) {  // an instance index or assumption literal out of range
      r = SCUBA_UNKNOWN;
      if (lane == 0) set_status(S, SCUBA_ERR_MALFORMED);
    } else if (S.flags[inst] & F_BAD) {
      r = SCUBA_UNKNOWN;
      if (lane == 0) set_status(S, SCUBA_ERR_MALFORMED);
    } else if (S.nv[inst] > S.vmax) {
      r = SCUBA_UNKNOWN;
      if (lane == 0) set_status(S, SCUBA_ERR_TOO_LARGE);
    } else if (moot) {
      r = SCUBA_UNSAT;  // moot: another subtree already found a model
    } else if constexpr (MODE == MODE_CDCL) {
      r = run_cdcl(S, w, slot, unit, inst, job, ring, abort_code);
    } else {
      r = run_job<MODE>(S, w, unit, inst, job, abort_code);
    }
    finish_job(S, w, unit, r);
    if (abort_code) {
      if (lane == 0) set_status(S, abort_code);
      break;
    }
  }
  if (counted_idle && lane == 0) atomicSub(&S.ctrl->idle, 1u);
}

// Unit-propagation closure of each instance under its unit clauses and the
// caller's assumption literals: one warp per instance, the same BCP as the
// search. values[vb[i] + v] = 0 open, 1 true, 2 false; conflict[i] = 1 when
// propagation falsifies a clause (values are then unspecified).
struct PropArgs {
  int n;
  int32_t vmax;
  uint32_t assign_words;
  const int64_t* icb;
  const int64_t* cb;
  const int32_t* lits;
  const int32_t* nv;
  const int64_t* vb;
  const int64_t* occ_base;
  const uint32_t* occ_begin;
  const uint64_t* ent;
  const uint32_t* units;
  const uint32_t* nunits;
  const uint32_t* flags;
  const int64_t* asm_begin;   // [n+1]
  const int32_t* asm_lits;    // DIMACS
  uint32_t* trail;            // [slots][vmax]
  uint8_t* values;
  uint8_t* conflict;
  Ctrl* ctrl;
};

__global__ void __launch_bounds__(256) k_propagate(const __grid_constant__ PropArgs A) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  WarpShared* wsh = reinterpret_cast<WarpShared*>(smem);
  Warp w;
  w.S = nullptr;  // the propagate kernel has no search state; BCP reads only w.*
  w.cb = A.cb;
  w.lits = A.lits;
  w.ws = &wsh[wib];
  w.asg = smem + (sizeof(WarpShared) / 4) * wpb + (size_t)A.assign_words * wib;
  w.lane = lane;
  const int64_t slot = (int64_t)blockIdx.x * wpb + wib;
  w.trail = A.trail + slot * A.vmax;
  if (batch_failed(A.ctrl)) return;
  for (int i = (int)(blockIdx.x * wpb + wib); i < A.n; i += gridDim.x * wpb) {
    if (A.flags[i] & F_BAD) continue;
    w.V = (uint32_t)A.nv[i];
    w.c0 = A.icb[i];
    w.occ = A.occ_begin + A.occ_base[i];
    const int64_t lbase = A.icb[i] < A.icb[i + 1] ? A.cb[A.icb[i]] : 0;
    w.ent = A.ent + lbase;
    warp_checks(w, A.ctrl);
    w.head = 0;
    const uint32_t nwords = (w.V + 15u) >> 4;
    for (uint32_t k = lane; k < nwords; k += 32) w.asg[k] = 0u;
    if (lane == 0) {
      w.ws->tail = 0;
      w.ws->conflict = 0;
      w.ws->props = w.ws->visits = 0;
    }
    __syncwarp();
    bool confl = (A.flags[i] & F_EMPTY) != 0;
    for (uint32_t k = lane; k < A.nunits[i] && !confl; k += 32)
      if (!imply(w, A.units[w.c0 + k])) record_conflict(w, 0, NONE, NONE);
    for (int64_t k = A.asm_begin[i] + lane; k < A.asm_begin[i + 1]; k += 32) {
      const int32_t l = A.asm_lits[k];
      if (l == 0 || l > (int32_t)w.V || l < -(int32_t)w.V) continue;
      if (!imply(w, code_of(l))) record_conflict(w, 0, NONE, NONE);
    }
    __syncwarp();
    confl = confl || w.ws->conflict != 0;
    if (!confl) confl = bcp(w);
    if (lane == 0) A.conflict[i] = confl ? 1 : 0;
    for (uint32_t x = lane; x < w.V; x += 32) {
      const uint32_t bits = (w.asg[x >> 4] >> ((x & 15u) * 2u)) & 3u;
      A.values[A.vb[i] + x] = (uint8_t)(bits == 3u ? 0u : bits);
    }
    __syncwarp();
  }
}

// Instances still open when the kernel stopped (timeout / abort) -> UNKNOWN.
__global__ void k_finalize(Solve S) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n_units;
       i += gridDim.x * blockDim.x) {
    uint32_t d = S.done[i];
    if (!(d & 5u)) S.verdict[i] = SCUBA_UNKNOWN;
  }
}

__global__ void k_init_ring(Job* ring, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
    ring[i].seq = i;
}

__global__ void k_init_inst(uint32_t* pending, uint32_t* done, unsigned long long* dec, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    pending[i] = 1u;
    done[i] = 0u;
    dec[i] = 0ull;
  }
}

__global__ void k_start_clock(Ctrl* c) { c->t0 = globaltimer(); }

__global__ void k_init_ctrl(Ctrl* c, uint32_t n) {
  c->next_inst = 0;
  c->inst_left = n;
  c->idle = 0;
  c->status = 0;
  c->q_head = 0;
  c->q_tail = 0;
  c->t0 = globaltimer();
  c->jobs_split = 0;
  c->check_site = 0;
  c->check_index = 0;
  c->check_limit = 0;
}

}  // namespace dev

// --------------------------------------------------------------------------
// Host side: scratch, launch
// --------------------------------------------------------------------------

namespace {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Scratch {
  Buf occ_base, norm, occ_cnt, occ_begin, ent, units, nunits, flags;
  Buf pending, done, inst_dec, trail, dstack, act, ring, job_act, prefix, ctrl;
  Buf lvlcnt, lvl_node;
  Buf cd_var, cd_mark, cd_wl, cd_pool, cd_learnt, cd_arena, cd_clidx;
  Buf share, share_cur;
  Buf job_cls, cls_copy;
  Buf h_icb, h_cb, h_lits, h_nv, h_vb, h_verdict, h_model, h_stats;  // for the host entry
  int sms = 0;
  int32_t last_status = 0;
  int smem_set[4] = {0, 0, 0, 0};  // dynamic shared memory granted per search mode
  int smem_prop = 0;
};

std::map<int, Scratch>& scratch_map() {
  static std::map<int, Scratch> m;
  return m;
}

int ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return 0;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t want = bytes + bytes / 4;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    want = bytes;
  }
  b.cap = want;
  return 0;
}

template <class T>
T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

int cuda_fail(const char* what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SCUBA_ERR_CUDA;
}

}  // namespace

}  // namespace scuba

using namespace scuba;

extern "C" int scuba_abi_sizes(int64_t* out) {
  if (!out) return SCUBA_ERR_ARG;
  out[0] = (int64_t)sizeof(scuba_cnf_batch);
  out[1] = (int64_t)sizeof(scuba_options);
  return SCUBA_OK;
}

extern "C" int scuba_options_init(scuba_options* o) {
  if (!o) return SCUBA_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->heuristic = SCUBA_HEUR_ACTIVITY;
  o->learned_depth = 0;
  o->decision_budget = 0;
  o->time_budget_ms = 0;
  o->split = 1;
  o->split_interval = 0;
  return SCUBA_OK;
}

// Units for scuba_solve_units: unit u is instance inst[u] under the
// assumption literals asm_lits[asm_begin[u] .. asm_begin[u+1]).
struct UnitArgs {
  int32_t n;
  const int32_t* inst;
  const int64_t* asm_begin;
  const int32_t* asm_lits;
  const int64_t* model_begin;
};

// clause-sharing pools of the clause-learning search: instance i uses pool
// i & (kSharePools - 1), a ring of kShareCap records of 64 bytes (128 MiB)
constexpr uint32_t kSharePools = 1024, kShareCap = 2048;

static int solve_impl(const scuba_cnf_batch* b, uint8_t* verdict, uint8_t* model,
                      cudaStream_t st, const scuba_options* opt, const UnitArgs* ua = nullptr) {
  if (!b || b->num_instances < 0 || b->total_clauses < 0 || b->total_lits < 0 ||
      b->max_vars < 0 || b->total_vars < 0) {
    set_error("scuba_solve_batch: bad arguments");
    return SCUBA_ERR_ARG;
  }
  scuba_options defaults;
  scuba_options_init(&defaults);
  if (!opt) opt = &defaults;
  const int n = b->num_instances;
  const int n_units = ua ? ua->n : n;
  if (n_units == 0) return SCUBA_OK;
  if (n == 0 || n_units < 0 || (ua && (!ua->inst || (ua->asm_begin && !ua->asm_lits)))) {
    set_error("scuba_solve_units: units need instances, a unit table and assumption literals");
    return SCUBA_ERR_ARG;
  }
  if (!verdict) {
    set_error("scuba_solve_batch: NULL verdict array");
    return SCUBA_ERR_ARG;
  }
  if (!b->inst_clause_begin || !b->clause_begin || !b->inst_num_vars || !b->inst_var_begin ||
      (b->total_lits > 0 && !b->lits)) {
    set_error("scuba_solve_batch: NULL batch array");
    return SCUBA_ERR_ARG;
  }
  if (opt->heuristic != SCUBA_HEUR_ACTIVITY && opt->heuristic != SCUBA_HEUR_LEARNED) {
    set_error("scuba_solve_batch: unknown heuristic");
    return SCUBA_ERR_ARG;
  }
  if (opt->search != SCUBA_SEARCH_DPLL && opt->search != SCUBA_SEARCH_CDCL) {
    set_error("scuba_solve_batch: unknown search algorithm");
    return SCUBA_ERR_ARG;
  }
  if (opt->search == SCUBA_SEARCH_CDCL &&
      (opt->trace || opt->heuristic != SCUBA_HEUR_ACTIVITY || opt->restart_unit < 0 ||
       opt->learnt_words < 0 || opt->learnt_words >= (1LL << 30))) {
    set_error("scuba_solve_batch: CDCL takes activity branching, no trace, restart_unit >= 0 "
              "and 0 <= learnt_words < 2^30");
    return SCUBA_ERR_ARG;
  }
  if (b->max_vars >= (1 << 29)) {
    set_error("scuba_solve_batch: instance too large (max_vars >= 2^29)");
    return SCUBA_ERR_TOO_LARGE;
  }
  int mode = dev::MODE_PLAIN;
  if (opt->trace) {
    const scuba_trace* T = opt->trace;
    if (T->depth < 1 || T->depth > learn::MAX_TRACE_DEPTH || T->max_nodes < 0 ||
        T->max_rows < 0 || !T->counts || !T->node_inst || !T->node_depth || !T->node_row ||
        !T->node_nrows || !T->node_closed || !T->x || !T->target || !T->var) {
      set_error("scuba_solve_batch: bad trace buffers (depth 1..8, all arrays set)");
      return SCUBA_ERR_ARG;
    }
    if (ua) {
      set_error("scuba_solve_units: trace recording takes whole instances");
      return SCUBA_ERR_ARG;
    }
    mode = dev::MODE_TRACE;
  } else if (opt->heuristic == SCUBA_HEUR_LEARNED) {
    if (!opt->mlp_weights || opt->learned_depth < 0) {
      set_error("scuba_solve_batch: learned branching needs mlp_weights and learned_depth >= 0");
      return SCUBA_ERR_ARG;
    }
    mode = dev::MODE_LEARNED;
  } else if (opt->search == SCUBA_SEARCH_CDCL) {
    mode = dev::MODE_CDCL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  Scratch& S = scratch_map()[dev];
  if (!S.sms) {
    e = cudaDeviceGetAttribute(&S.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute", e);
  }
  const int64_t C = b->total_clauses, L = b->total_lits;
  const int vmax = std::max(1, (int)b->max_vars);
  // occurrence offsets: sum over instances of (2V+1)
  const int64_t occ_total = 2LL * b->total_vars + n;

  // shape: warps per block x blocks per SM (shared memory bounds the warps).
  // The trail goes to shared memory when that still leaves >= 16 warps/SM.
  int wpb = opt->warps_per_block > 0 ? opt->warps_per_block : 8;
  int bps = opt->blocks_per_sm > 0 ? opt->blocks_per_sm : 5;
  wpb = std::min(wpb, 8);
  // 2 bits per variable; the clause-learning search keeps 4 (value + fresh)
  const uint32_t assign_words = mode == dev::MODE_CDCL ? (uint32_t)((vmax + 7) / 8)
                                                       : (uint32_t)((vmax + 15) / 16);
  const size_t smem_cap = 227 * 1024, sm_cap = 228 * 1024;
  const size_t per_warp_g = sizeof(dev::WarpShared) + (size_t)assign_words * 4;
  const size_t per_warp_s = per_warp_g + (size_t)vmax * 4;
  // Global memory by default: a small shared-memory carve-out leaves a larger L1
  // for the read-only occurrence lists, which measured faster.
  int trail_smem = opt->trail_placement == 1 ? 1 : 0;
  (void)per_warp_s;
  size_t per_warp = trail_smem ? per_warp_s : per_warp_g;
  if (mode == dev::MODE_LEARNED) per_warp += 32 * learn::NFEAT * sizeof(__nv_bfloat16);
  if (mode == dev::MODE_CDCL) per_warp += dev::CD_SMEM_WARP;
  size_t smem = per_warp * wpb + (mode == dev::MODE_CDCL ? 16 : 0);  // ring alignment
  while (wpb > 1 && smem > smem_cap) {
    wpb--;
    smem = per_warp * wpb + (mode == dev::MODE_CDCL ? 16 : 0);
  }
  if (smem > smem_cap) {
    set_error("scuba_solve_batch: instance too large for the shared-memory assignment");
    return SCUBA_ERR_TOO_LARGE;
  }
  while (bps > 1 && (smem + 1024) * bps > sm_cap) bps--;
  if (mode == dev::MODE_LEARNED) bps = std::min(bps, SCUBA_LEARNED_MINBLOCKS);
  if (mode == dev::MODE_CDCL) bps = std::min(bps, SCUBA_CDCL_MINBLOCKS);
  const int64_t slots = (int64_t)S.sms * bps * wpb;
  const uint32_t ring_cap = 2048;

  if (ensure(S.occ_base, 8 * (size_t)(n + 1)) || ensure(S.norm, 4 * (size_t)L) ||
      ensure(S.occ_cnt, 4 * (size_t)occ_total) || ensure(S.occ_begin, 4 * (size_t)occ_total) ||
      ensure(S.ent, 8 * (size_t)L) || ensure(S.units, 4 * (size_t)std::max<int64_t>(C, 1)) ||
      ensure(S.nunits, 4 * (size_t)n) || ensure(S.flags, 4 * (size_t)n) ||
      ensure(S.pending, 4 * (size_t)n_units) || ensure(S.done, 4 * (size_t)n_units) ||
      ensure(S.inst_dec, 8 * (size_t)n_units) || ensure(S.trail, 4 * (size_t)slots * vmax) ||
      ensure(S.dstack, 4 * (size_t)slots * vmax) || ensure(S.act, 4 * (size_t)slots * vmax) ||
      ensure(S.ring, sizeof(dev::Job) * (size_t)ring_cap) ||
      ensure(S.job_act, 4 * (size_t)ring_cap * vmax) ||
      ensure(S.prefix, 4 * (size_t)slots * dev::MAX_PREFIX) || ensure(S.ctrl, sizeof(dev::Ctrl))) {
    set_error("scuba_solve_batch: out of device memory for scratch");
    return SCUBA_ERR_NOMEM;
  }
  if (mode == dev::MODE_TRACE &&
      (ensure(S.lvlcnt, 4 * (size_t)slots * learn::MAX_TRACE_DEPTH * vmax) ||
       ensure(S.lvl_node, 8 * (size_t)slots * learn::MAX_TRACE_DEPTH))) {
    set_error("scuba_solve_batch: out of device memory for trace scratch");
    return SCUBA_ERR_NOMEM;
  }
  int64_t arena_words = 0;
  if (mode == dev::MODE_CDCL) {
    arena_words = (opt->learnt_words > 0 ? opt->learnt_words : (1LL << 18)) & ~3LL;
    if (arena_words < std::max<int64_t>((int64_t)vmax + 2 * dev::CD_HDR, 64)) {
      set_error("scuba_solve_batch: learnt_words must be at least max(max_vars + 8, 64)");
      return SCUBA_ERR_ARG;
    }
    if (ensure(S.cd_var, 16 * (size_t)slots * vmax) ||
        ensure(S.cd_mark, (size_t)slots * vmax) ||
        ensure(S.cd_wl, 32 * (size_t)slots * vmax) ||
        ensure(S.cd_pool, 8 * (size_t)slots * arena_words) ||
        ensure(S.cd_learnt, 4 * (size_t)slots * vmax) ||
        ensure(S.cd_arena, 4 * (size_t)slots * arena_words) ||
        ensure(S.cd_clidx, 4 * (size_t)slots * (arena_words / 8)) ||
        ensure(S.job_cls, 4 * (size_t)ring_cap * dev::JOB_CLS_WORDS) ||
        ensure(S.cls_copy, 4 * (size_t)slots * dev::JOB_CLS_WORDS) ||
        ensure(S.share, 4 * (size_t)kSharePools * kShareCap * dev::SHARE_REC) ||
        ensure(S.share_cur, 8 * (size_t)kSharePools)) {
      set_error("scuba_solve_batch: out of device memory for clause-learning scratch");
      return SCUBA_ERR_NOMEM;
    }
  }
  dev::Prep pr;
  pr.n = n;
  pr.C = C;
  pr.L = L;
  pr.icb = b->inst_clause_begin;
  pr.cb = b->clause_begin;
  pr.lits = b->lits;
  pr.nv = b->inst_num_vars;
  pr.occ_base = P<int64_t>(S.occ_base);
  pr.norm = P<uint32_t>(S.norm);
  pr.occ_cnt = P<uint32_t>(S.occ_cnt);
  pr.occ_begin = P<uint32_t>(S.occ_begin);
  pr.ent = P<uint64_t>(S.ent);
  pr.units = P<uint32_t>(S.units);
  pr.nunits = P<uint32_t>(S.nunits);
  pr.flags = P<uint32_t>(S.flags);
  pr.total_vars = b->total_vars;
  pr.occ_cap = occ_total;
  pr.vmax = vmax;
  pr.vb = b->inst_var_begin;
  pr.ctrl = P<dev::Ctrl>(S.ctrl);

  NvtxRange prep_range("scuba prep + search launch");
  dev::k_init_ctrl<<<1, 1, 0, st>>>(pr.ctrl, (uint32_t)n_units);
  cudaMemsetAsync(pr.occ_cnt, 0, 4 * (size_t)occ_total, st);
  cudaMemsetAsync(pr.flags, 0, 4 * (size_t)n, st);
  dev::k_occ_base<<<1, 1024, 0, st>>>(pr);
  if (C > 0) {
    int grid = (int)std::min<int64_t>((C + 255) / 256, (int64_t)S.sms * 32);
    dev::k_normalize<<<grid, 256, 0, st>>>(pr);
  }
  int wgrid = (int)std::min<int64_t>((n + 7) / 8, (int64_t)S.sms * 16);
  dev::k_occ_scan<<<wgrid, 256, 0, st>>>(pr);
  dev::k_fill<<<wgrid, 256, 0, st>>>(pr);

  dev::Solve sv;
  sv.n = n;
  sv.vmax = vmax;
  sv.assign_words = assign_words;
  sv.icb = b->inst_clause_begin;
  sv.cb = b->clause_begin;
  sv.lits = b->lits;
  sv.nv = b->inst_num_vars;
  sv.vb = b->inst_var_begin;
  sv.occ_base = pr.occ_base;
  sv.occ_begin = pr.occ_begin;
  sv.ent = pr.ent;
  sv.units = pr.units;
  sv.nunits = pr.nunits;
  sv.flags = pr.flags;
  sv.order = opt->order;
  sv.n_units = n_units;
  sv.unit_inst = ua ? ua->inst : nullptr;
  sv.unit_asm_begin = ua ? ua->asm_begin : nullptr;
  sv.unit_asm = ua ? ua->asm_lits : nullptr;
  sv.unit_vb = ua ? ua->model_begin : nullptr;
  sv.verdict = verdict;
  sv.model = model;
  sv.stats = opt->stats;
  sv.pending = P<uint32_t>(S.pending);
  sv.done = P<uint32_t>(S.done);
  sv.inst_dec = P<unsigned long long>(S.inst_dec);
  sv.trail = P<uint32_t>(S.trail);
  sv.dstack = P<uint32_t>(S.dstack);
  sv.act = P<float>(S.act);
  sv.ring = P<dev::Job>(S.ring);
  sv.ring_cap = ring_cap;
  sv.job_act = P<float>(S.job_act);
  sv.prefix = P<uint32_t>(S.prefix);
  sv.split_min = opt->split_min > 0 ? opt->split_min : 256;
  sv.split_depth = opt->split_depth > 0 ? opt->split_depth : dev::MAX_PREFIX;
  sv.ctrl = P<dev::Ctrl>(S.ctrl);
  sv.budget = opt->decision_budget;
  int64_t tb = opt->time_budget_ms > 0 ? opt->time_budget_ms : 600000;
  sv.time_ns = (uint64_t)tb * 1000000ull;
  sv.abort_flag = opt->abort_flag;
  sv.split = opt->split ? 1 : 0;
  sv.split_interval = opt->split_interval > 0 ? opt->split_interval : 16;
  sv.trail_smem = trail_smem;
  sv.finish_ns = opt->finish_ns;
  sv.prof = reinterpret_cast<unsigned long long*>(opt->profile);
  sv.mlp = static_cast<const learn::MlpWeights*>(opt->mlp_weights);
  sv.learned_depth = opt->learned_depth;
  sv.inst_num_inputs = opt->inst_num_inputs;
  sv.trace_depth = 0;
  sv.lvlcnt = nullptr;
  sv.lvl_node = nullptr;
  sv.cd_var = P<uint4>(S.cd_var);
  sv.cd_mark = P<uint8_t>(S.cd_mark);
  sv.cd_wl = P<dev::WList>(S.cd_wl);
  sv.cd_pool = P<uint64_t>(S.cd_pool);
  sv.cd_pool_cap = arena_words;
  sv.cd_learnt = P<uint32_t>(S.cd_learnt);
  sv.cd_arena = P<uint32_t>(S.cd_arena);
  sv.cd_clidx = P<uint32_t>(S.cd_clidx);
  sv.job_cls = P<uint32_t>(S.job_cls);
  sv.cls_copy = P<uint32_t>(S.cls_copy);
  sv.cd_arena_words = arena_words;
  sv.restart_unit = opt->restart_unit > 0 ? opt->restart_unit : 100;
  sv.share = nullptr;
  sv.share_cur = nullptr;
  sv.share_mask = 0;
  sv.share_cap = 0;
  sv.share_lbd = 0;
  if (mode == dev::MODE_CDCL && opt->share_lbd >= 0) {
    // the pools start empty every call: a record left by an earlier batch must
    // never pass for one of this batch
    sv.share = P<uint32_t>(S.share);
    sv.share_cur = P<unsigned long long>(S.share_cur);
    sv.share_mask = kSharePools - 1;
    sv.share_cap = kShareCap;
    sv.share_lbd = opt->share_lbd > 0 ? (uint32_t)opt->share_lbd : 2u;
    cudaMemsetAsync(sv.share, 0, 4 * (size_t)kSharePools * kShareCap * dev::SHARE_REC, st);
    cudaMemsetAsync(sv.share_cur, 0, 8 * (size_t)kSharePools, st);
  }
  std::memset(&sv.tr, 0, sizeof(sv.tr));
  if (mode == dev::MODE_TRACE) {
    const scuba_trace* T = opt->trace;
    sv.trace_depth = T->depth;
    sv.split = 0;  // a traced subtree must be explored by one warp
    sv.tr.cursor = reinterpret_cast<unsigned long long*>(T->counts);
    sv.tr.max_nodes = T->max_nodes;
    sv.tr.max_rows = T->max_rows;
    sv.tr.node_inst = T->node_inst;
    sv.tr.node_depth = T->node_depth;
    sv.tr.node_row = T->node_row;
    sv.tr.node_nrows = T->node_nrows;
    sv.tr.node_closed = T->node_closed;
    sv.tr.x = reinterpret_cast<__nv_bfloat16*>(T->x);
    sv.tr.target = T->target;
    sv.tr.var = T->var;
    sv.lvlcnt = P<uint32_t>(S.lvlcnt);
    sv.lvl_node = P<int64_t>(S.lvl_node);
    cudaMemsetAsync(sv.lvlcnt, 0, 4 * (size_t)slots * learn::MAX_TRACE_DEPTH * vmax, st);
    cudaMemsetAsync(sv.lvl_node, 0xff, 8 * (size_t)slots * learn::MAX_TRACE_DEPTH, st);
  }

  dev::k_init_ring<<<16, 256, 0, st>>>(sv.ring, ring_cap);
  dev::k_init_inst<<<(n_units + 255) / 256, 256, 0, st>>>(sv.pending, sv.done, sv.inst_dec,
                                                          n_units);
  dev::k_start_clock<<<1, 1, 0, st>>>(sv.ctrl);
  auto kern = mode == dev::MODE_TRACE     ? dev::k_solve<dev::MODE_TRACE>
              : mode == dev::MODE_LEARNED ? dev::k_solve<dev::MODE_LEARNED>
              : mode == dev::MODE_CDCL    ? dev::k_solve<dev::MODE_CDCL>
                                          : dev::k_solve<dev::MODE_PLAIN>;
  // raise the dynamic shared-memory limit only when it grows, so that a
  // repeated call (for example while a CUDA graph is being captured) issues
  // no attribute change
  if ((int)smem > S.smem_set[mode]) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail("cudaFuncSetAttribute", e);
    S.smem_set[mode] = (int)smem;
  }
  if (opt->search_event_begin) cudaEventRecord((cudaEvent_t)opt->search_event_begin, st);
  kern<<<S.sms * bps, 32 * wpb, smem, st>>>(sv);
  if (opt->search_event_end) cudaEventRecord((cudaEvent_t)opt->search_event_end, st);
  dev::k_finalize<<<(n_units + 255) / 256, 256, 0, st>>>(sv);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("kernel launch", e);
  return SCUBA_OK;
}

extern "C" int scuba_solve_batch_ex(const scuba_cnf_batch* b, uint8_t* verdict, uint8_t* model,
                                    void* stream, const scuba_options* opt) {
  return solve_impl(b, verdict, model, (cudaStream_t)stream, opt);
}

extern "C" int scuba_solve_units(const scuba_cnf_batch* b, int32_t n_units,
                                 const int32_t* unit_inst, const int64_t* asm_begin,
                                 const int32_t* asm_lits, const int64_t* unit_model_begin,
                                 uint8_t* verdict, uint8_t* model, void* stream,
                                 const scuba_options* opt) {
  if (n_units < 0 || (n_units > 0 && (!unit_inst || !verdict)) || (model && !unit_model_begin)) {
    set_error("scuba_solve_units: bad arguments");
    return SCUBA_ERR_ARG;
  }
  UnitArgs ua{n_units, unit_inst, asm_begin, asm_lits, unit_model_begin};
  return solve_impl(b, verdict, model, (cudaStream_t)stream, opt, &ua);
}

extern "C" int scuba_solve_batch(const scuba_cnf_batch* b, uint8_t* verdict, uint8_t* model,
                                 void* stream) {
  return solve_impl(b, verdict, model, (cudaStream_t)stream, nullptr);
}

extern "C" int scuba_sync_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = scratch_map().find(dev);
  if (it == scratch_map().end() || !it->second.ctrl.p) return SCUBA_OK;
  dev::Ctrl c;
  e = cudaMemcpy(&c, it->second.ctrl.p, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("cudaMemcpy", e);
  if (c.status != 0) {
    std::string msg = "device status " + std::to_string(c.status);
    if (c.check_site != 0)
      msg += " (bounds check " + std::to_string(c.check_site) + " failed: index " +
             std::to_string(c.check_index) + ", limit " + std::to_string(c.check_limit) + ")";
    set_error(msg);
  }
  return c.status;
}

extern "C" int scuba_solve_batch_host(const scuba_cnf_batch* hb, uint8_t* verdict,
                                      uint8_t* model, void* stream, const scuba_options* opt) {
  if (!hb || !verdict || hb->num_instances < 0) return SCUBA_ERR_ARG;
  const int n = hb->num_instances;
  if (n == 0) return SCUBA_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  Scratch& S = scratch_map()[dev];
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t C = hb->total_clauses, L = hb->total_lits;
  const int64_t nvars = hb->inst_var_begin[n];
  if (ensure(S.h_icb, 8 * (size_t)(n + 1)) || ensure(S.h_cb, 8 * (size_t)(C + 1)) ||
      ensure(S.h_lits, 4 * (size_t)L) || ensure(S.h_nv, 4 * (size_t)n) ||
      ensure(S.h_vb, 8 * (size_t)(n + 1)) || ensure(S.h_verdict, (size_t)n) ||
      ensure(S.h_model, (size_t)std::max<int64_t>(nvars, 1)) ||
      ensure(S.h_stats, 8 * SCUBA_NSTATS * (size_t)n))
    return SCUBA_ERR_NOMEM;
  cudaError_t e;
  NvtxRange range("scuba host-buffer solve (upload, solve, download)");
  e = cudaMemcpyAsync(S.h_icb.p, hb->inst_clause_begin, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.h_cb.p, hb->clause_begin, 8 * (size_t)(C + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && L > 0) e = cudaMemcpyAsync(S.h_lits.p, hb->lits, 4 * (size_t)L, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.h_nv.p, hb->inst_num_vars, 4 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.h_vb.p, hb->inst_var_begin, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync H2D", e);
  scuba_cnf_batch db = *hb;
  db.inst_clause_begin = P<int64_t>(S.h_icb);
  db.clause_begin = P<int64_t>(S.h_cb);
  db.lits = P<int32_t>(S.h_lits);
  db.inst_num_vars = P<int32_t>(S.h_nv);
  db.inst_var_begin = P<int64_t>(S.h_vb);
  scuba_options o;
  if (opt) o = *opt; else scuba_options_init(&o);
  int64_t* host_stats = o.stats;
  if (host_stats) {
    cudaMemsetAsync(S.h_stats.p, 0, 8 * SCUBA_NSTATS * (size_t)n, st);
    o.stats = P<int64_t>(S.h_stats);
  }
  int r = solve_impl(&db, P<uint8_t>(S.h_verdict), model ? P<uint8_t>(S.h_model) : nullptr, st, &o);
  if (r != SCUBA_OK) return r;
  e = cudaMemcpyAsync(verdict, S.h_verdict.p, (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && model && nvars > 0)
    e = cudaMemcpyAsync(model, S.h_model.p, (size_t)nvars, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && host_stats)
    e = cudaMemcpyAsync(host_stats, S.h_stats.p, 8 * SCUBA_NSTATS * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync D2H", e);
  return scuba_sync_status(stream);
}

extern "C" void scuba_release(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  auto it = scratch_map().find(dev);
  if (it == scratch_map().end()) return;
  Scratch& S = it->second;
  Buf* all[] = {&S.occ_base, &S.norm, &S.occ_cnt, &S.occ_begin, &S.ent, &S.units, &S.nunits,
                &S.flags, &S.pending, &S.done, &S.inst_dec, &S.trail, &S.dstack, &S.act,
                &S.ring, &S.job_act, &S.prefix, &S.ctrl, &S.lvlcnt, &S.lvl_node,
                &S.cd_var, &S.cd_mark, &S.cd_wl, &S.cd_pool,
                &S.cd_learnt, &S.cd_arena, &S.cd_clidx, &S.job_cls, &S.cls_copy,
                &S.share, &S.share_cur, &S.h_icb,
                &S.h_cb, &S.h_lits,
                &S.h_nv, &S.h_vb,
                &S.h_verdict, &S.h_model, &S.h_stats};
  for (Buf* x : all) {
    if (x->p) cudaFree(x->p);
    x->p = nullptr;
    x->cap = 0;
  }
  scratch_map().erase(it);
}

// --------------------------------------------------------------------------
// Allocation-free variant
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, inside a plugin whose host
// forbids device allocation, or on a path where a synchronous allocation would
// stall other streams. For them scuba_solve_batch_noalloc runs the same
// preparation and search kernels with every scratch buffer carved out of one
// file-scope device array of fixed size. Every GPU that loads this library
// holds that array until the process exits.
// --------------------------------------------------------------------------

namespace scuba {
namespace {
constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB
constexpr int kNoAllocWarpsPerBlock = 4;
constexpr uint32_t kNoAllocRingCap = 256;
constexpr int kMaxDevices = 256;
void* g_noalloc_scratch_addr[kMaxDevices];  // device address of the array, per device
std::mutex g_noalloc_mu;  // guards the per-device set-up and the shared attribute cache
}  // namespace
}  // namespace scuba

static __device__ __align__(256) unsigned char g_noalloc_scratch[scuba::kNoAllocScratchBytes];

extern "C" int scuba_solve_batch_noalloc(const scuba_cnf_batch* b, uint8_t* verdict,
                                         uint8_t* model, void* stream,
                                         const scuba_options* opt) {
  using namespace scuba;
  if (!b || b->num_instances < 0 || b->total_clauses < 0 || b->total_lits < 0 ||
      b->max_vars < 0 || b->total_vars < 0) {
    set_error("scuba_solve_batch_noalloc: bad arguments");
    return SCUBA_ERR_ARG;
  }
  scuba_options defaults;
  scuba_options_init(&defaults);
  if (!opt) opt = &defaults;
  const int n = b->num_instances;
  if (n == 0) return SCUBA_OK;
  if (!verdict || !b->inst_clause_begin || !b->clause_begin || !b->inst_num_vars ||
      !b->inst_var_begin || (b->total_lits > 0 && !b->lits)) {
    set_error("scuba_solve_batch_noalloc: NULL array");
    return SCUBA_ERR_ARG;
  }
  if (opt->heuristic != SCUBA_HEUR_ACTIVITY || opt->search != SCUBA_SEARCH_DPLL) {
    set_error("scuba_solve_batch_noalloc: only DPLL with activity branching is supported");
    return SCUBA_ERR_ARG;
  }
  if (b->max_vars >= (1 << 29) || b->total_lits >= (1LL << 32)) {
    set_error("scuba_solve_batch_noalloc: instance too large");
    return SCUBA_ERR_TOO_LARGE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("scuba_solve_batch_noalloc: device ordinal out of range");
    return SCUBA_ERR_ARG;
  }
  // set-up, once per device, with that device current: the host-side name of
  // the array is not a device address, so ask the runtime for it
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail("cudaGetSymbolAddress", e);
      g_noalloc_scratch_addr[dev] = p;
    }
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute", e);

  const int64_t C = b->total_clauses, L = b->total_lits;
  const int vmax = std::max(1, (int)b->max_vars);
  const int64_t occ_total = 2LL * b->total_vars + n;
  const int wpb = kNoAllocWarpsPerBlock;
  const uint32_t assign_words = (uint32_t)((vmax + 15) / 16);
  const size_t smem = (sizeof(dev::WarpShared) + (size_t)assign_words * 4) * wpb;
  if (smem > 227 * 1024) {
    set_error("scuba_solve_batch_noalloc: instance too large for the shared-memory assignment");
    return SCUBA_ERR_TOO_LARGE;
  }
  const int64_t slots = (int64_t)sms * wpb;  // one block per SM
  const uint32_t ring_cap = kNoAllocRingCap;

  // carve every buffer out of the static array, 256-byte aligned
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t at = off;
    off += (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
    return at;
  };
  const size_t o_occ_base = carve(8 * (size_t)(n + 1)), o_norm = carve(4 * (size_t)L),
               o_occ_cnt = carve(4 * (size_t)occ_total), o_occ_begin = carve(4 * (size_t)occ_total),
               o_ent = carve(8 * (size_t)L), o_units = carve(4 * (size_t)std::max<int64_t>(C, 1)),
               o_nunits = carve(4 * (size_t)n), o_flags = carve(4 * (size_t)n),
               o_pending = carve(4 * (size_t)n), o_done = carve(4 * (size_t)n),
               o_inst_dec = carve(8 * (size_t)n), o_trail = carve(4 * (size_t)slots * vmax),
               o_dstack = carve(4 * (size_t)slots * vmax), o_act = carve(4 * (size_t)slots * vmax),
               o_ring = carve(sizeof(dev::Job) * (size_t)ring_cap),
               o_job_act = carve(4 * (size_t)ring_cap * vmax),
               o_prefix = carve(4 * (size_t)slots * dev::MAX_PREFIX),
               o_ctrl = carve(sizeof(dev::Ctrl));
  if (off > kNoAllocScratchBytes) {
    set_error("scuba_solve_batch_noalloc: batch needs " + std::to_string(off) +
              " bytes of scratch, more than the fixed " +
              std::to_string(kNoAllocScratchBytes) + " bytes");
    return SCUBA_ERR_TOO_LARGE;
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_scratch_addr[dev]);
  auto at = [&](size_t o) { return static_cast<void*>(base + o); };

  dev::Prep pr;
  pr.n = n;
  pr.C = C;
  pr.L = L;
  pr.icb = b->inst_clause_begin;
  pr.cb = b->clause_begin;
  pr.lits = b->lits;
  pr.nv = b->inst_num_vars;
  pr.occ_base = static_cast<int64_t*>(at(o_occ_base));
  pr.norm = static_cast<uint32_t*>(at(o_norm));
  pr.occ_cnt = static_cast<uint32_t*>(at(o_occ_cnt));
  pr.occ_begin = static_cast<uint32_t*>(at(o_occ_begin));
  pr.ent = static_cast<uint64_t*>(at(o_ent));
  pr.units = static_cast<uint32_t*>(at(o_units));
  pr.nunits = static_cast<uint32_t*>(at(o_nunits));
  pr.flags = static_cast<uint32_t*>(at(o_flags));
  pr.total_vars = b->total_vars;
  pr.occ_cap = occ_total;
  pr.vmax = vmax;
  pr.vb = b->inst_var_begin;
  pr.ctrl = static_cast<dev::Ctrl*>(at(o_ctrl));

  // the array keeps the previous call's contents: everything that must start
  // at zero is cleared here, the rest is written before it is read
  dev::k_init_ctrl<<<1, 1, 0, st>>>(pr.ctrl, (uint32_t)n);
  cudaMemsetAsync(pr.occ_cnt, 0, 4 * (size_t)occ_total, st);
  cudaMemsetAsync(pr.flags, 0, 4 * (size_t)n, st);
  dev::k_occ_base<<<1, 1024, 0, st>>>(pr);
  if (C > 0) {
    int grid = (int)std::min<int64_t>((C + 255) / 256, (int64_t)sms * 32);
    dev::k_normalize<<<grid, 256, 0, st>>>(pr);
  }
  int wgrid = (int)std::min<int64_t>((n + 7) / 8, (int64_t)sms * 16);
  dev::k_occ_scan<<<wgrid, 256, 0, st>>>(pr);
  dev::k_fill<<<wgrid, 256, 0, st>>>(pr);

  dev::Solve sv;
  std::memset(&sv, 0, sizeof(sv));
  sv.n = n;
  sv.vmax = vmax;
  sv.assign_words = assign_words;
  sv.icb = b->inst_clause_begin;
  sv.cb = b->clause_begin;
  sv.lits = b->lits;
  sv.nv = b->inst_num_vars;
  sv.vb = b->inst_var_begin;
  sv.occ_base = pr.occ_base;
  sv.occ_begin = pr.occ_begin;
  sv.ent = pr.ent;
  sv.units = pr.units;
  sv.nunits = pr.nunits;
  sv.flags = pr.flags;
  sv.n_units = n;
  sv.order = opt->order;
  sv.verdict = verdict;
  sv.model = model;
  sv.stats = opt->stats;
  sv.pending = static_cast<uint32_t*>(at(o_pending));
  sv.done = static_cast<uint32_t*>(at(o_done));
  sv.inst_dec = static_cast<unsigned long long*>(at(o_inst_dec));
  sv.trail = static_cast<uint32_t*>(at(o_trail));
  sv.dstack = static_cast<uint32_t*>(at(o_dstack));
  sv.act = static_cast<float*>(at(o_act));
  sv.ring = static_cast<dev::Job*>(at(o_ring));
  sv.ring_cap = ring_cap;
  sv.job_act = static_cast<float*>(at(o_job_act));
  sv.prefix = static_cast<uint32_t*>(at(o_prefix));
  sv.split_min = opt->split_min > 0 ? opt->split_min : 256;
  sv.split_depth = opt->split_depth > 0 ? opt->split_depth : dev::MAX_PREFIX;
  sv.ctrl = pr.ctrl;
  sv.budget = opt->decision_budget;
  int64_t tb = opt->time_budget_ms > 0 ? opt->time_budget_ms : 600000;
  sv.time_ns = (uint64_t)tb * 1000000ull;
  sv.abort_flag = opt->abort_flag;
  sv.split = opt->split ? 1 : 0;
  sv.split_interval = opt->split_interval > 0 ? opt->split_interval : 16;
  sv.trail_smem = 0;
  sv.finish_ns = nullptr;
  sv.prof = nullptr;

  dev::k_init_ring<<<4, 256, 0, st>>>(sv.ring, ring_cap);
  dev::k_init_inst<<<(n + 255) / 256, 256, 0, st>>>(sv.pending, sv.done, sv.inst_dec, n);
  dev::k_start_clock<<<1, 1, 0, st>>>(sv.ctrl);
  // the kernel attribute is shared with the regular entry points: only ever
  // raise it, through the same per-device cache, so that a later regular
  // call that needs more shared memory still finds its own grant in place
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    int& granted = scratch_map()[dev].smem_set[dev::MODE_PLAIN];
    if ((int)smem > granted) {
      e = cudaFuncSetAttribute(dev::k_solve<dev::MODE_PLAIN>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return cuda_fail("cudaFuncSetAttribute", e);
      granted = (int)smem;
    }
  }
  dev::k_solve<dev::MODE_PLAIN><<<sms, 32 * wpb, smem, st>>>(sv);
  dev::k_finalize<<<(n + 255) / 256, 256, 0, st>>>(sv);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("kernel launch", e);
  // report the device-side status of this call (the control block lives in
  // the static array, so the normal status query cannot see it)
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
  int32_t status = 0;
  e = cudaMemcpy(&status, reinterpret_cast<unsigned char*>(pr.ctrl) + offsetof(dev::Ctrl, status),
                 sizeof(status), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("cudaMemcpy", e);
  if (status != 0) set_error("scuba_solve_batch_noalloc: device status " + std::to_string(status));
  return status;
}

extern "C" int scuba_propagate_batch(const scuba_cnf_batch* b, const int64_t* asm_begin,
                                     const int32_t* asm_lits, uint8_t* values,
                                     uint8_t* conflict, void* stream) {
  using namespace scuba;
  if (!b || b->num_instances < 0 || b->max_vars < 0 || b->total_vars < 0 ||
      b->total_clauses < 0 || b->total_lits < 0) {
    set_error("scuba_propagate_batch: bad arguments");
    return SCUBA_ERR_ARG;
  }
  const int n = b->num_instances;
  if (n == 0) return SCUBA_OK;
  if (!asm_begin || !values || !conflict || !b->inst_clause_begin || !b->clause_begin ||
      !b->inst_num_vars || !b->inst_var_begin || (b->total_lits > 0 && !b->lits)) {
    set_error("scuba_propagate_batch: NULL array");
    return SCUBA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  Scratch& S = scratch_map()[dev];
  if (!S.sms) {
    e = cudaDeviceGetAttribute(&S.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute", e);
  }
  const int64_t C = b->total_clauses, L = b->total_lits;
  const int vmax = std::max(1, (int)b->max_vars);
  const int64_t occ_total = 2LL * b->total_vars + n;
  const int wpb = 8;
  const uint32_t assign_words = (uint32_t)((vmax + 15) / 16);
  const size_t smem = (sizeof(dev::WarpShared) + (size_t)assign_words * 4) * wpb;
  if (smem > 227 * 1024) return SCUBA_ERR_TOO_LARGE;
  const int blocks = S.sms;
  const int64_t slots = (int64_t)blocks * wpb;
  if (ensure(S.occ_base, 8 * (size_t)(n + 1)) || ensure(S.norm, 4 * (size_t)L) ||
      ensure(S.occ_cnt, 4 * (size_t)occ_total) || ensure(S.occ_begin, 4 * (size_t)occ_total) ||
      ensure(S.ent, 8 * (size_t)L) || ensure(S.units, 4 * (size_t)std::max<int64_t>(C, 1)) ||
      ensure(S.nunits, 4 * (size_t)n) || ensure(S.flags, 4 * (size_t)n) ||
      ensure(S.trail, 4 * (size_t)slots * vmax) || ensure(S.ctrl, sizeof(dev::Ctrl)))
    return SCUBA_ERR_NOMEM;
  dev::Prep pr;
  pr.n = n;
  pr.C = C;
  pr.L = L;
  pr.icb = b->inst_clause_begin;
  pr.cb = b->clause_begin;
  pr.lits = b->lits;
  pr.nv = b->inst_num_vars;
  pr.occ_base = P<int64_t>(S.occ_base);
  pr.norm = P<uint32_t>(S.norm);
  pr.occ_cnt = P<uint32_t>(S.occ_cnt);
  pr.occ_begin = P<uint32_t>(S.occ_begin);
  pr.ent = P<uint64_t>(S.ent);
  pr.units = P<uint32_t>(S.units);
  pr.nunits = P<uint32_t>(S.nunits);
  pr.flags = P<uint32_t>(S.flags);
  pr.total_vars = b->total_vars;
  pr.occ_cap = occ_total;
  pr.vmax = vmax;
  pr.vb = b->inst_var_begin;
  pr.ctrl = P<dev::Ctrl>(S.ctrl);
  dev::k_init_ctrl<<<1, 1, 0, st>>>(pr.ctrl, (uint32_t)n);
  cudaMemsetAsync(pr.occ_cnt, 0, 4 * (size_t)occ_total, st);
  cudaMemsetAsync(pr.flags, 0, 4 * (size_t)n, st);
  dev::k_occ_base<<<1, 1024, 0, st>>>(pr);
  if (C > 0) {
    int grid = (int)std::min<int64_t>((C + 255) / 256, (int64_t)S.sms * 32);
    dev::k_normalize<<<grid, 256, 0, st>>>(pr);
  }
  int wgrid = (int)std::min<int64_t>((n + 7) / 8, (int64_t)S.sms * 16);
  dev::k_occ_scan<<<wgrid, 256, 0, st>>>(pr);
  dev::k_fill<<<wgrid, 256, 0, st>>>(pr);
  dev::PropArgs A;
  A.n = n;
  A.vmax = vmax;
  A.assign_words = assign_words;
  A.icb = b->inst_clause_begin;
  A.cb = b->clause_begin;
  A.lits = b->lits;
  A.nv = b->inst_num_vars;
  A.vb = b->inst_var_begin;
  A.occ_base = pr.occ_base;
  A.occ_begin = pr.occ_begin;
  A.ent = pr.ent;
  A.units = pr.units;
  A.nunits = pr.nunits;
  A.flags = pr.flags;
  A.asm_begin = asm_begin;
  A.asm_lits = asm_lits;
  A.trail = P<uint32_t>(S.trail);
  A.values = values;
  A.conflict = conflict;
  A.ctrl = pr.ctrl;
  if ((int)smem > S.smem_prop) {
    e = cudaFuncSetAttribute(dev::k_propagate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return cuda_fail("cudaFuncSetAttribute", e);
    S.smem_prop = (int)smem;
  }
  dev::k_propagate<<<blocks, 32 * wpb, smem, st>>>(A);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("kernel launch", e);
  return SCUBA_OK;
}
