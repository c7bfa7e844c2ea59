// cdcl.cuh -- conflict-driven clause learning mode of the persistent search
// (included by solver.cu after the DPLL search; same prep layout, shared
// assignment, BCP frontier rounds and worker loop).
//
// The paper's solver (Sec. V-B, OR-Tools' SAT solver) learns clauses
// internally and says no more about it; this mode puts the textbook
// first-UIP scheme on top of the GPU propagation of the DPLL mode:
//
//  * The assignment takes 4 bits per variable in shared memory: value (true,
//    false) and a "fresh" bit, set by the same compare-and-swap that claims
//    the variable during a BCP round and cleared when the round after it
//    starts. Every assigned variable keeps its reason (the occurrence entry or
//    clause reference that implied it) and its decision level.
//  * Propagation rounds are frontier-parallel, so two lanes can assign
//    variables of the same round in either trail order. An implication may
//    therefore only rely on false literals assigned BEFORE the current round;
//    a clause whose unit-ness depends on a literal falsified during the round
//    is left for the next round, where that literal's own occurrence list
//    brings it back. Every reason then precedes its literal on the trail, and
//    the trail is a topological order of the implication graph. Conflicts
//    need no such rule: a falsified clause is a conflict whenever found.
//  * Learned clauses live in a per-warp arena with two watched literals per
//    clause. Each literal's watch list is an array in a per-warp pool (grown
//    by doubling); an entry is {clause, blocker}, the blocker being a literal
//    of the clause (the other watch when the entry was made) whose truth
//    settles the clause without reading it. After the static occurrence
//    entries of each frontier batch, the watchers of every literal in the
//    batch are spread over the 32 lanes like the static entries. A clause
//    can sit on two lists of one batch only when both its watches are false;
//    a lane then takes a per-clause lock first, and the loser retries after
//    the winner has moved its watch. Moved watches are appended to their new
//    lists one at a time (the warp copies a list when it grows) and the
//    batch's own lists are compacted afterwards.
//  * Conflict analysis resolves the falsified clause with the reasons of
//    current-level literals, newest first on the trail, until one
//    current-level literal (the first UIP) is left; the lanes take the
//    literals of each clause, and the next literal to resolve is the newest
//    of the waiting ones, kept with their trail positions in shared memory
//    (a warp-wide backward scan of the trail if more than CAND wait). Every
//    variable met is bumped.
//  * Hard instances are shared cube-and-conquer style through the DPLL mode's
//    job ring: a busy warp that sees idle warps gives away the negation of
//    its first free decision, together with the assumptions above it, as a
//    cube, and keeps that decision as one more assumption itself (backjumps
//    and restarts never undo assumptions). An instance is UNSAT once every
//    cube is; a cube starts from its donor's activities and its short,
//    low-LBD learned clauses. A unit of scuba_solve_units (an instance under
//    the caller's assumptions) starts the same way, as a job with a prefix.
//  * The search backjumps to the second-highest level of the learned clause
//    and asserts its UIP literal there; decisions take the saved phase (the
//    variable's last value, false at first); restarts follow the Luby
//    sequence times `restart_unit` conflicts. The first restart after 2000
//    conflicts (then 2300, 2600, ... more) also halves the learned clauses,
//    keeping the newer half and every clause of LBD <= 3 (the number of
//    distinct decision levels in it at learning time, after Glucose). When
//    the arena or the watch pool runs out the same reduction happens at once;
//    if even that does not fit, every learned clause is dropped (all of them
//    are implied by the formula, so any of this is sound).
//
// Clause arena layout (32-bit words, 16-byte aligned clauses): [len, lock, 0,
// 0, lit0 .. lit_{len-1}, padding to a multiple of 4]; lit0 and lit1 are the
// watched literals.

constexpr uint32_t LEARNT_REF = 0xC0000000u;  // clause reference: learned clause at offset
constexpr uint32_t CD_HDR = 4;
constexpr uint64_t WATCH_GONE = ~0ull;     // tombstone of a moved watch entry
constexpr uint32_t NB_T = 1u, NB_F = 2u, NB_FRESH = 4u;  // assignment nibble bits
constexpr uint32_t RING = 128;  // recent-trail entries per warp in shared memory
constexpr uint32_t CAND = 96;   // current-level literals awaiting resolution, per warp
// shared memory per warp for the clause-learning search (16-byte multiple)
constexpr uint32_t CD_SMEM_WARP = RING * 8 + CAND * 8;
constexpr uint8_t MK_PHASE = 1, MK_SEEN = 2;

// Profile counters (only when the caller passed a profile array): lane 0
// adds the clock cycles of each phase to its warp's WarpShared::cyc.
enum { PF_BCP = 0, PF_LEARNED = 1, PF_ANALYZE = 2, PF_DECIDE = 3, PF_DB = 4, PF_NDB = 5,
       PF_NLEARNT = 6 };

__device__ __forceinline__ long long pf_now(const Solve& S) {
  return S.prof ? clock64() : 0;
}

__device__ __forceinline__ void pf_add(const Solve& S, Warp& w, int k, long long t0) {
  if (S.prof && w.lane == 0) w.ws->cyc[k] += (unsigned long long)(clock64() - t0);
}

__device__ __forceinline__ bool is_learnt_ref(uint32_t a) {
  return a != NONE && (a & LEARNT_REF) == LEARNT_REF;
}

struct WList {       // one literal's learned watch list in the pool
  uint32_t off, len, cap, pad;
};

// Per assigned variable, one 16-byte record written by one store: the reason
// (the occurrence entry {a, b} that implied it, or a clause reference in the
// low word, ~0 for decisions and assumptions), its trail position and level.
struct VarInfo {
  uint32_t reason_lo, reason_hi, pos, level;
};

struct CdWarp {
  VarInfo* var;       // [V] reason, trail position, decision level
  uint8_t* mark;      // [V] MK_PHASE saved phase, MK_SEEN during analysis
  WList* wl;          // [2V] learned watch list per literal code
  uint64_t* pool;     // [pool_cap] watch entries {clause, blocker}
  uint32_t* arena;    // [arena_words]
  uint32_t* cl_off;   // [arena_words / 8] arena offset of each learned clause, oldest first
  uint32_t* learnt;   // [V] clause under construction
  uint2* ring;        // [RING] shared memory: {literal, trail position} of recent claims
  uint2* cand;        // [CAND] shared memory: analysis queue {trail position, literal}
  uint32_t arena_words, pool_cap;
  uint32_t top;       // first free arena word
  uint32_t ncl;       // learned clauses in the arena
  uint32_t pool_top;  // first free pool entry
  uint32_t full;      // the pool ran out during propagation: drop the learned clauses
};

// The nibble of variable v (value bits and fresh bit).
__device__ __forceinline__ uint32_t nib(const uint32_t* asg, uint32_t v) {
  return (asg[v >> 3] >> ((v & 7u) * 4u)) & 7u;
}

// Value (LV_U, LV_T, LV_F) of literal l whose variable has nibble n.
__device__ __forceinline__ uint32_t nib_value(uint32_t n, uint32_t l) {
  const uint32_t b = n & 3u;
  if (b == 0u) return LV_U;
  return ((b == NB_T) != ((l & 1u) != 0u)) ? LV_T : LV_F;
}

__device__ __forceinline__ uint32_t lit_value_cd(const uint32_t* asg, uint32_t l) {
  return nib_value(nib(asg, l >> 1), l);
}

// Assign l with reason `why` at the current level; fresh marks a claim made
// inside a BCP round. One compare-and-swap claims value and fresh bit
// together. Returns false on a clash with the opposite value.
__device__ __forceinline__ bool imply_cd(Warp& w, CdWarp& cd, uint32_t l, uint64_t why,
                                         uint32_t fresh = NB_FRESH) {
  const uint32_t v = WIDX(w, l >> 1, w.V, 11), wi = v >> 3, sh = (v & 7u) * 4u;
  const uint32_t val = (l & 1u) ? NB_F : NB_T;
  uint32_t old = w.asg[wi];
  for (;;) {
    const uint32_t cur = (old >> sh) & 3u;
    if (cur) return cur == val;
    const uint32_t prev = atomicCAS(&w.asg[wi], old, old | ((val | fresh) << sh));
    if (prev == old) break;
    old = prev;
  }
  const uint32_t pos = WIDX(w, atomicAdd(&w.ws->tail, 1u), w.V, 12);
  w.trail[pos] = l;
  cd.ring[pos & (RING - 1u)] = make_uint2(l, pos);
  *reinterpret_cast<uint4*>(&cd.var[v]) =
      make_uint4((uint32_t)why, (uint32_t)(why >> 32), pos, w.nd);
  return true;
}

// trail[p], from the shared-memory ring when its slot still holds position p.
__device__ __forceinline__ uint32_t trail_at(const Warp& w, const CdWarp& cd, uint32_t p) {
  const uint2 e = cd.ring[p & (RING - 1u)];
  return e.y == p ? e.x : w.trail[p];
}

__device__ void eval_long_cd(Warp& w, CdWarp& cd, uint32_t local) {
  const int64_t c = w.c0 + local;
  const int64_t b = w.cb[c], e = w.cb[c + 1];
  uint32_t open_lit = NONE;
  int n_open = 0;
  bool fresh_false = false;
  for (int64_t q = b; q < e; q++) {
    const uint32_t x = code_of(__ldg(&w.lits[q]));
    const uint32_t n = nib(w.asg, x >> 1);
    const uint32_t vx = nib_value(n, x);
    if (vx == LV_T) return;
    if (vx == LV_U) {
      if (x != open_lit) {
        n_open++;
        open_lit = x;
        if (n_open > 1) return;
      }
    } else if (n & NB_FRESH) {
      fresh_false = true;
    }
  }
  if (n_open == 1 && fresh_false) return;  // a literal falsified this round: next round
  if (n_open == 0 || !imply_cd(w, cd, open_lit, (uint64_t)(LONG_CLAUSE | local)))
    record_conflict(w, LONG_CLAUSE | local, NONE, NONE);
}

// One occurrence entry of the falsified (old) literal f: (f | a) with b ==
// NONE, (f | a | b), or a long clause. One claim site and one conflict site.
__device__ __forceinline__ void eval_entry_cd(Warp& w, CdWarp& cd, uint32_t f, uint64_t e) {
  const uint32_t a0 = (uint32_t)e, b0 = (uint32_t)(e >> 32);
  if (a0 & LONG_CLAUSE) {
    eval_long_cd(w, cd, a0 & ~LONG_CLAUSE);
    return;
  }
  const uint32_t a = WIDX(w, a0, 2u * w.V, 13);
  const uint32_t b = b0 == NONE ? NONE : WIDX(w, b0, 2u * w.V, 13);
  const uint32_t na = nib(w.asg, a >> 1);
  const uint32_t va = nib_value(na, a);
  uint32_t nb = 0, vb = LV_F;  // a binary entry has no third literal: read it as false
  if (b != NONE) {
    nb = nib(w.asg, b >> 1);
    vb = nib_value(nb, b);
  }
  if (va == LV_T || vb == LV_T) return;
  uint32_t unit = NONE, other = NONE;  // the literal to imply, the false one beside f
  if (va == LV_U && vb == LV_F) {
    if (nb & NB_FRESH) return;  // b falsified this round: next round
    unit = a;
    other = b;
  } else if (vb == LV_U && va == LV_F) {
    if (na & NB_FRESH) return;
    unit = b;
    other = a;
  } else if (va == LV_U || vb == LV_U) {
    return;  // two open literals
  }
  if (unit == NONE ||
      !imply_cd(w, cd, unit, (uint64_t)f | ((uint64_t)other << 32)))
    record_conflict(w, f, a, b);
}

// Append entry e to literal g's watch list (all lanes, uniform arguments).
__device__ void wl_append(Warp& w, CdWarp& cd, uint32_t g, uint64_t e) {
  if (cd.full) return;
  WList L = cd.wl[g];  // last written before a __syncwarp
  if (L.len == L.cap) {
    const uint32_t ncap = L.cap ? 2u * L.cap : 8u;
    if ((uint64_t)cd.pool_top + ncap > cd.pool_cap) {
      cd.full = 1;
      if (w.lane == 0) record_conflict(w, NONE, NONE, NONE);  // ends this BCP
      __syncwarp();
      return;
    }
    const uint32_t noff = cd.pool_top;
    cd.pool_top += ncap;
    for (uint32_t k = w.lane; k < L.len; k += 32) cd.pool[noff + k] = cd.pool[L.off + k];
    L.off = noff;
    L.cap = ncap;
  }
  __syncwarp();
  if (w.lane == 0) {
    cd.pool[L.off + L.len] = e;
    L.len++;
    cd.wl[g] = L;
  }
  __syncwarp();
}

// A new watch for a learned clause: the first position >= 2 whose literal is
// not false, else the first whose literal was falsified during this round
// (its own list brings the clause back next round), else NONE. Literals are
// read 4 at a time (16-byte loads; clauses are 16-byte aligned and padded).
__device__ __forceinline__ uint32_t new_watch(const uint32_t* asg, const uint32_t* lits,
                                              uint32_t len) {
  const uint4* L4 = reinterpret_cast<const uint4*>(lits);
  uint32_t fresh_pos = NONE;
  for (uint32_t q = 0; q < len; q += 4) {
    const uint4 a = L4[q >> 2];
    const uint32_t x[4] = {a.x, a.y, a.z, a.w};
    uint32_t open = 0, fr = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (q + i < 2 || q + i >= len) continue;
      const uint32_t n = nib(asg, x[i] >> 1);
      if (nib_value(n, x[i]) != LV_F) open |= 1u << i;
      else if (n & NB_FRESH) fr |= 1u << i;
    }
    if (open) return q + __ffs(open) - 1;
    if (fr && fresh_pos == NONE) fresh_pos = q + __ffs(fr) - 1;
  }
  return fresh_pos;
}

// One watch entry (clause c, blocker) of the falsified literal f, at pool
// index at. Returns the literal the watch moved to (NONE if it stayed) and
// the entry for that literal's list.
__device__ uint32_t visit_learnt(Warp& w, CdWarp& cd, uint32_t f, uint32_t at, uint32_t c,
                                 uint64_t& moved_entry) {
  uint32_t* C = cd.arena + c;
  const uint32_t l0 = C[CD_HDR], l1 = C[CD_HDR + 1];
  const uint32_t which = l0 == f ? 0u : 1u;
  const uint32_t other = which ? l0 : l1;
  const uint32_t vo = lit_value_cd(w.asg, other);
  if (vo == LV_T) {
    cd.pool[at] = (uint64_t)c | ((uint64_t)other << 32);  // new blocker
    return NONE;
  }
  const uint32_t k = new_watch(w.asg, C + CD_HDR, C[0]);
  if (k != NONE) {
    const uint32_t g = C[CD_HDR + k];
    C[CD_HDR + k] = f;
    C[CD_HDR + which] = g;
    cd.pool[at] = WATCH_GONE;
    moved_entry = (uint64_t)c | ((uint64_t)other << 32);
    return g;
  }
  if (vo == LV_F) {
    record_conflict(w, LEARNT_REF | c, NONE, NONE);
  } else if (vo == LV_U) {
    if (!imply_cd(w, cd, other, (uint64_t)(LEARNT_REF | c)))
      record_conflict(w, LEARNT_REF | c, NONE, NONE);
  }
  return NONE;
}

// Learned clauses watching the literals falsified in this batch: lane j <
// nlit holds falsified literal f and its watch list pool[beg, beg + cnt).
__device__ void learned_batch(Warp& w, CdWarp& cd, uint32_t nlit, uint32_t f, uint32_t beg,
                              uint32_t cnt) {
  __syncwarp();
  if (cd.top == 0) return;  // no learned clauses
  const long long t0 = pf_now(*w.S);
  uint32_t inc = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, d);
    if (w.lane >= d) inc += y;
  }
  const uint32_t excl = inc - cnt;
  const uint32_t total = __shfl_sync(FULL, inc, 31);
  WCOUNT(w, visits, total);
  uint32_t dirty = 0;  // lists that lost an entry
  for (uint32_t e0 = 0; e0 < total; e0 += 32) {
    const uint32_t e = e0 + w.lane;
    int lo_j = 0, hi_j = 31;  // owner: smallest lane j with inc_j > e
#pragma unroll
    for (int s2 = 0; s2 < 5; s2++) {
      const int mid = (lo_j + hi_j) >> 1;
      const uint32_t v = __shfl_sync(FULL, inc, mid);
      if (v > e) hi_j = mid; else lo_j = mid + 1;
      if (lo_j > hi_j) lo_j = hi_j;
    }
    const uint32_t jbeg = __shfl_sync(FULL, beg, lo_j);
    const uint32_t jex = __shfl_sync(FULL, excl, lo_j);
    const uint32_t jf = __shfl_sync(FULL, f, lo_j);
    bool pending = false;
    uint32_t at = 0, c = 0;
    if (e < total) {
      at = WIDX(w, jbeg + (e - jex), cd.pool_cap, 16);
      const uint64_t ent = cd.pool[at];
      c = WIDX(w, (uint32_t)ent, cd.top, 17);
      pending = lit_value_cd(w.asg, WIDX(w, (uint32_t)(ent >> 32), 2u * w.V, 18)) != LV_T;  // blocker
    }
    uint32_t g = NONE;
    uint64_t moved = 0;
    // both watches false: the clause may be on two lists of this batch, so
    // the lane locks it; a loser retries after the winner's pass
    while (__any_sync(FULL, pending)) {
      if (pending) {
        volatile uint32_t* C = cd.arena + c;
        const uint32_t other = C[CD_HDR] == jf ? C[CD_HDR + 1] : C[CD_HDR];
        bool go = true, locked = false;
        if (lit_value_cd(w.asg, other) == LV_F) {
          locked = atomicCAS((uint32_t*)&C[1], 0u, 1u) == 0u;
          go = locked;
        }
        if (go) {
          g = visit_learnt(w, cd, jf, at, c, moved);
          if (locked) {
            __threadfence_block();
            atomicExch((uint32_t*)&C[1], 0u);
          }
          pending = false;
        }
      }
      __syncwarp();
    }
    dirty |= __reduce_or_sync(FULL, g != NONE ? (1u << lo_j) : 0u);
    uint32_t movers = __ballot_sync(FULL, g != NONE);
    while (movers) {
      const int j = __ffs(movers) - 1;
      movers &= movers - 1u;
      const uint32_t gj = __shfl_sync(FULL, g, j);
      const uint64_t mj = __shfl_sync(FULL, moved, j);
      wl_append(w, cd, gj, mj);
    }
  }
  // compact the lists that lost entries (lane j owns frontier literal j)
  if (w.lane < nlit && ((dirty >> w.lane) & 1u) && !cd.full) {
    uint32_t keep = 0;
    for (uint32_t k = 0; k < cnt; k++) {
      const uint64_t ent = cd.pool[beg + k];
      if (ent != WATCH_GONE) cd.pool[beg + keep++] = ent;
    }
    cd.wl[f].len = keep;
  }
  __syncwarp();
  pf_add(*w.S, w, PF_LEARNED, t0);
}

// Static occurrence entries of one batch over the 32 lanes: lane j < nlit
// holds falsified literal f and its occurrence list ent[beg, beg + cnt). One
// evaluation site keeps the hot code small.
__device__ __forceinline__ void static_batch(Warp& w, CdWarp& cd, uint32_t nlit, uint32_t f,
                                             uint32_t beg, uint32_t cnt) {
  uint32_t inc = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, d);
    if (w.lane >= d) inc += y;
  }
  const uint32_t excl = inc - cnt;
  const uint32_t total = __shfl_sync(FULL, inc, 31);
  WCOUNT(w, visits, total);
  for (uint32_t e0 = 0; e0 < total; e0 += 32) {
    const uint32_t e = e0 + w.lane;
    int j = 0;  // owner: smallest lane j with inc_j > e (lane 0 alone when nlit == 1)
    if (nlit > 1) {
      int hi_j = 31;
#pragma unroll
      for (int s2 = 0; s2 < 5; s2++) {
        const int mid = (j + hi_j) >> 1;
        const uint32_t v = __shfl_sync(FULL, inc, mid);
        if (v > e) hi_j = mid; else j = mid + 1;
        if (j > hi_j) j = hi_j;
      }
    }
    const uint32_t jbeg = __shfl_sync(FULL, beg, j);
    const uint32_t jex = __shfl_sync(FULL, excl, j);
    const uint32_t jf = __shfl_sync(FULL, f, j);
    if (e < total) eval_entry_cd(w, cd, jf, __ldg(&w.ent[WIDX(w, jbeg + (e - jex), w.ent_end, 15)]));
  }
}

// Unit propagation to a fixpoint (true on conflict), in the frontier rounds
// of the DPLL search. Per batch of up to 32 frontier literals the lanes read
// their literal (from the ring when it is there), clear its fresh bit, and
// load both its occurrence-list bounds and its learned watch list before
// the static entries and then the learned watchers are evaluated.
__device__ bool bcp_cd(Warp& w, CdWarp& cd) {
  for (;;) {
    __syncwarp();
    const uint32_t hi = *(volatile uint32_t*)&w.ws->tail;
    if (w.head >= hi) return false;
    const uint32_t lo = w.head;
    w.head = hi;
    WCOUNT(w, props, hi - lo);
    for (uint32_t base = lo; base < hi; base += 32) {
      const uint32_t nlit = min(32u, hi - base);
      uint32_t f = 0, beg = 0, cnt = 0, lbeg = 0, lcnt = 0;
      if (w.lane < nlit) {
        const uint32_t t = trail_at(w, cd, base + w.lane);
        const uint32_t v = t >> 1;
        atomicAnd(&w.asg[v >> 3], ~(NB_FRESH << ((v & 7u) * 4u)));  // no longer fresh
        f = WIDX(w, t ^ 1u, 2u * w.V, 14);
        beg = __ldg(&w.occ[f]);
        cnt = __ldg(&w.occ[f + 1]) - beg;
        if (cd.top) {
          const WList L = cd.wl[f];
          lbeg = L.off;
          lcnt = L.len;
        }
      }
      __syncwarp();
      static_batch(w, cd, nlit, f, beg, cnt);
      learned_batch(w, cd, nlit, f, lbeg, lcnt);
      __syncwarp();
      if (*(volatile uint32_t*)&w.ws->conflict) return true;
    }
  }
}

// First-UIP analysis of the recorded conflict (all lanes). Leaves the learned
// clause in cd.learnt[0 .. n): the asserting literal first, then a literal of
// the backjump level; returns n, the backjump level in blev and the clause's
// LBD (distinct decision levels, counted per group of 32 literals) in lbd.
// Returns 0 if a consistency check fails (seen marks may then be left set).
__device__ uint32_t analyze_cd(Warp& w, CdWarp& cd, uint32_t& blev, uint32_t& lbd) {
  const uint32_t lvl = w.nd;
  uint32_t n = 1, path = 0, p = NONE;
  uint32_t r0 = w.ws->cl[0], r1 = w.ws->cl[1], r2 = w.ws->cl[2];
  int64_t idx = (int64_t)*(volatile uint32_t*)&w.ws->tail - 1;
  // Current-level literals not yet resolved wait in cd.cand with their trail
  // positions; the newest is the next to resolve. If more than CAND wait at
  // once, the rest of this analysis scans the trail for seen marks instead.
  uint32_t ncand = 0;
  bool overflow = false;
  bool big = false;
  for (;;) {
    // the literals of the clause: static entry (up to three codes), a long
    // clause of the caller's CSR, or a learned clause
    const uint32_t* src = nullptr;
    const int32_t* csr = nullptr;
    uint32_t cnt = 3;
    if (is_learnt_ref(r0)) {
      const uint32_t off = r0 & ~LEARNT_REF;
      cnt = cd.arena[off];
      src = cd.arena + off + CD_HDR;
    } else if (r0 & LONG_CLAUSE) {
      const int64_t cl = w.c0 + (r0 & ~LONG_CLAUSE);
      const int64_t b = w.cb[cl];
      csr = w.lits + b;
      cnt = (uint32_t)(w.cb[cl + 1] - b);
    }
    for (uint32_t k0 = 0; k0 < cnt; k0 += 32) {
      const uint32_t k = k0 + w.lane;
      uint32_t q = NONE;
      if (k < cnt) q = src ? src[k] : csr ? code_of(csr[k]) : (k == 0 ? r0 : k == 1 ? r1 : r2);
      const uint32_t v = q == NONE ? NONE >> 1 : WIDX(w, q >> 1, w.V, 21);
      bool take = false;
      uint32_t mk = 0, lv = 0, ps = 0;
      if (q != NONE && (p == NONE || v != (p >> 1))) {
        mk = cd.mark[v];  // three independent loads
        const uint2 pl = *reinterpret_cast<const uint2*>(&cd.var[v].pos);
        ps = pl.x;
        lv = pl.y;
        take = !(mk & MK_SEEN) && lv > 0;
      }
      // one lane per variable (a long clause may repeat a literal)
      const uint32_t grp = __match_any_sync(FULL, take ? v : NONE);
      if (take && __ffs(grp) - 1 != w.lane) take = false;
      if (take) {
        cd.mark[v] = mk | MK_SEEN;
        const float a = w.act[v] + w.inc;
        w.act[v] = a;
        big |= a > 1e20f;
      }
      const bool cur = take && lv >= lvl;
      const uint32_t curm = __ballot_sync(FULL, cur);
      path += __popc(curm);
      if (!overflow) {
        if (ncand + __popc(curm) <= CAND) {
          if (cur) cd.cand[ncand + __popc(curm & ((1u << w.lane) - 1u))] = make_uint2(ps, q ^ 1u);
          ncand += __popc(curm);
        } else {
          overflow = true;
        }
      }
      const uint32_t lowm = __ballot_sync(FULL, take && lv < lvl);
      if (take && lv < lvl) cd.learnt[WIDX(w, n + __popc(lowm & ((1u << w.lane) - 1u)), w.V, 20)] = q;
      n += __popc(lowm);
      __syncwarp();
    }
    // a conflict without a current-level literal, or a scan that runs off the
    // trail, means the search state is inconsistent: give up (n = 0)
    if (path == 0) return 0;
    if (!overflow) {
      // the newest waiting literal (trail positions are distinct)
      uint32_t key = 0, kk = 0;  // key = position + 1
      for (uint32_t k = w.lane; k < ncand; k += 32) {
        const uint32_t x = cd.cand[k].x + 1u;
        if (x > key) {
          key = x;
          kk = k;
        }
      }
      for (int d = 16; d > 0; d >>= 1) {
        const uint32_t ok = __shfl_xor_sync(FULL, key, d), oi = __shfl_xor_sync(FULL, kk, d);
        if (ok > key) {
          key = ok;
          kk = oi;
        }
      }
      if (key == 0) return 0;
      p = cd.cand[kk].y;
      idx = (int64_t)key - 2;  // where a trail scan would continue
      __syncwarp();
      if (w.lane == 0) cd.cand[kk] = cd.cand[ncand - 1];
      ncand--;
    } else {
      for (;;) {  // the newest seen literal on the trail
        if (idx < 0) return 0;
        const int64_t pos = idx - w.lane;
        bool sn = false;
        if (pos >= 0) sn = (cd.mark[w.trail[pos] >> 1] & MK_SEEN) != 0;
        const uint32_t m = __ballot_sync(FULL, sn);
        if (m) {
          idx -= __ffs(m) - 1;
          break;
        }
        idx -= 32;
      }
      p = w.trail[idx];
      idx--;
    }
    __syncwarp();
    if (w.lane == 0) cd.mark[p >> 1] &= (uint8_t)~MK_SEEN;
    __syncwarp();
    if (--path == 0) break;
    const uint2 rw = *reinterpret_cast<const uint2*>(&cd.var[p >> 1].reason_lo);
    const uint64_t why = (uint64_t)rw.x | ((uint64_t)rw.y << 32);
    r0 = (uint32_t)why;
    r1 = (uint32_t)(why >> 32);
    r2 = NONE;
  }
  if (w.lane == 0) cd.learnt[0] = p ^ 1u;
  // backjump level: the highest level among learnt[1..n), moved to position 1
  uint32_t best_l = 0, best_k = 1, levels = 1;  // learnt[0] is alone at level lvl
  for (uint32_t k0 = 1; k0 < n; k0 += 32) {
    const uint32_t k = k0 + w.lane;
    uint32_t lv = NONE;
    if (k < n) {
      const uint32_t q = cd.learnt[k];
      lv = cd.var[q >> 1].level;
      if (lv > best_l) {
        best_l = lv;
        best_k = k;
      }
      cd.mark[q >> 1] &= (uint8_t)~MK_SEEN;
    }
    const uint32_t grp = __match_any_sync(FULL, lv);
    levels += __popc(__ballot_sync(FULL, k < n && __ffs(grp) - 1 == w.lane));
  }
  lbd = levels;
  for (int d = 16; d > 0; d >>= 1) {
    const uint32_t ol = __shfl_xor_sync(FULL, best_l, d);
    const uint32_t ok = __shfl_xor_sync(FULL, best_k, d);
    if (ol > best_l || (ol == best_l && ok < best_k)) {
      best_l = ol;
      best_k = ok;
    }
  }
  __syncwarp();
  if (w.lane == 0 && n > 2 && best_k != 1) {
    const uint32_t t = cd.learnt[1];
    cd.learnt[1] = cd.learnt[best_k];
    cd.learnt[best_k] = t;
  }
  big = __any_sync(FULL, big);
  if (big) {
    for (uint32_t v = w.lane; v < w.V; v += 32) w.act[v] *= 1e-20f;
    w.inc *= 1e-20f;
  }
  __syncwarp();
  blev = best_l;
  return n;
}

// Undo every assignment above level lev, saving phases.
__device__ void backjump_cd(Warp& w, CdWarp& cd, uint32_t lev) {
  if (w.nd <= lev) return;
  const uint32_t pos = w.dstack[lev];
  const uint32_t tail = *(volatile uint32_t*)&w.ws->tail;
  WCOUNT(w, undone, tail - pos);
  for (uint32_t t = pos + w.lane; t < tail; t += 32) {
    const uint32_t l = w.trail[t], v = l >> 1;
    atomicAnd(&w.asg[v >> 3], ~(0xfu << ((v & 7u) * 4u)));
    cd.mark[v] = (l & 1u) ? 0 : MK_PHASE;
  }
  __syncwarp();
  if (w.lane == 0) w.ws->tail = pos;
  __syncwarp();
  w.nd = lev;
  w.head = pos;
}

// Arena words a learned clause of n literals takes.
__device__ __forceinline__ uint32_t clause_words(uint32_t n) {
  return CD_HDR + ((n + 3u) & ~3u);
}

// Store learnt[0..n) (n >= 2) at the arena top and watch its first two
// literals. The caller checked the arena has room; the pool may run out
// (cd.full).
__device__ uint32_t add_learnt(Warp& w, CdWarp& cd, uint32_t n, uint32_t lbd) {
  const uint32_t c = cd.top;
  for (uint32_t k = w.lane; k < ((n + 3u) & ~3u); k += 32)
    cd.arena[c + CD_HDR + k] = k < n ? cd.learnt[k] : NONE;
  if (w.lane == 0) {
    cd.arena[c] = n;
    cd.arena[c + 1] = 0u;
    cd.arena[c + 2] = lbd;
    cd.arena[c + 3] = 0u;
  }
  if (w.lane == 0) {
    cd.cl_off[cd.ncl] = c;
    if (w.S->prof) w.ws->cyc[PF_NLEARNT]++;
  }
  __syncwarp();
  cd.top = c + clause_words(n);
  cd.ncl++;
  const uint32_t l0 = cd.learnt[0], l1 = cd.learnt[1];
  wl_append(w, cd, l0, (uint64_t)c | ((uint64_t)l1 << 32));
  wl_append(w, cd, l1, (uint64_t)c | ((uint64_t)l0 << 32));
  return c;
}

__device__ void clear_learnts(Warp& w, CdWarp& cd) {
  for (uint32_t k = w.lane; k < 2u * w.V; k += 32) cd.wl[k] = WList{0u, 0u, 0u, 0u};
  cd.top = 0;
  cd.ncl = 0;
  cd.pool_top = 0;
  cd.full = 0;
  __syncwarp();
}

__device__ bool rebuild_watches(Warp& w, CdWarp& cd);

// Learned-clause database maintenance at the bottom level (no reason above it
// refers to a learned clause). With drop_half, keep the newer half of the
// clauses and every clause whose LBD is at most 3 (the "glue" clauses that
// tie few decision levels together); otherwise keep them all.
// Kept clauses move down the arena in order; then every watch list is built
// afresh from the clauses' first two literals (count, scan, fill), which
// also compacts the pool. Returns false when the lists would take more than
// half of the pool.
__device__ bool reduce_db(Warp& w, CdWarp& cd, bool drop_half) {
  const uint32_t n = cd.ncl;
  uint32_t run_words = 0, run_cl = 0;
  for (uint32_t k0 = 0; k0 < n; k0 += 32) {
    const uint32_t k = k0 + w.lane;
    uint32_t off = 0, words = 0;
    bool keep = false;
    if (k < n) {
      off = cd.cl_off[k];
      const uint32_t len = cd.arena[off];
      keep = !drop_half || k >= n / 2 || cd.arena[off + 2] <= 3u;
      if (keep) words = clause_words(len);
    }
    uint32_t inc = words;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (w.lane >= d) inc += y;
    }
    const uint32_t dst = run_words + inc - words;
    const uint32_t km = __ballot_sync(FULL, keep);
    __syncwarp();
    // move the kept clauses down one at a time, in order (dst <= src)
    for (uint32_t m = km; m; m &= m - 1u) {
      const int j = __ffs(m) - 1;
      const uint32_t src = __shfl_sync(FULL, off, j), to = __shfl_sync(FULL, dst, j);
      const uint32_t wd = __shfl_sync(FULL, words, j);
      if (src != to)
        for (uint32_t q0 = 0; q0 < wd; q0 += 32) {
          const uint32_t q = q0 + w.lane;
          const uint32_t x = q < wd ? cd.arena[src + q] : 0u;
          __syncwarp();
          if (q < wd) cd.arena[to + q] = x;
          __syncwarp();
        }
    }
    if (keep) cd.cl_off[run_cl + __popc(km & ((1u << w.lane) - 1u))] = dst;
    run_words += __shfl_sync(FULL, inc, 31);
    run_cl += __popc(km);
    __syncwarp();
  }
  cd.top = run_words;
  cd.ncl = run_cl;
  return rebuild_watches(w, cd);
}

// Every watch list built afresh from the learned clauses' first two literals
// (count, exclusive scan of capacities, fill); this also compacts the pool.
// Returns false when the lists would take more than half of the pool.
__device__ bool rebuild_watches(Warp& w, CdWarp& cd) {
  const uint32_t run_cl = cd.ncl;
  const uint32_t nl = 2u * w.V;
  for (uint32_t k = w.lane; k < nl; k += 32) cd.wl[k] = WList{0u, 0u, 0u, 0u};
  __syncwarp();
  for (uint32_t k = w.lane; k < run_cl; k += 32) {
    const uint32_t c = cd.cl_off[k];
    atomicAdd(&cd.wl[cd.arena[c + CD_HDR]].len, 1u);
    atomicAdd(&cd.wl[cd.arena[c + CD_HDR + 1]].len, 1u);
  }
  __syncwarp();
  uint32_t base = 0;
  for (uint32_t k0 = 0; k0 < nl; k0 += 32) {
    const uint32_t k = k0 + w.lane;
    const uint32_t len = k < nl ? cd.wl[k].len : 0u;
    const uint32_t cap = len ? len + max(4u, len / 2u) : 0u;
    uint32_t inc = cap;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (w.lane >= d) inc += y;
    }
    if (k < nl) cd.wl[k] = WList{base + inc - cap, 0u, cap, 0u};
    base += __shfl_sync(FULL, inc, 31);
  }
  __syncwarp();
  cd.pool_top = 0;
  cd.full = 0;
  if (base > cd.pool_cap / 2) return false;  // leave room for the lists to grow
  for (uint32_t k = w.lane; k < run_cl; k += 32) {
    const uint32_t c = cd.cl_off[k];
    const uint32_t l0 = cd.arena[c + CD_HDR], l1 = cd.arena[c + CD_HDR + 1];
    const uint32_t p0 = atomicAdd(&cd.wl[l0].len, 1u);
    cd.pool[cd.wl[l0].off + p0] = (uint64_t)c | ((uint64_t)l1 << 32);
    const uint32_t p1 = atomicAdd(&cd.wl[l1].len, 1u);
    cd.pool[cd.wl[l1].off + p1] = (uint64_t)c | ((uint64_t)l0 << 32);
  }
  cd.pool_top = base;
  __syncwarp();
  return true;
}

// Bring the database back within its limits at the bottom level: compact
// (drop_half false) or halve it, and if the lists still do not fit, drop it.
// Afterwards the bottom levels are propagated again from the first trail
// entry, over the rebuilt watch lists too.
__device__ void maintain_db(Warp& w, CdWarp& cd, bool drop_half) {
  const long long t0 = pf_now(*w.S);
  if (w.S->prof && w.lane == 0) w.ws->cyc[PF_NDB]++;
  backjump_cd(w, cd, w.nd_fixed);
  if (!reduce_db(w, cd, drop_half) && (drop_half || !reduce_db(w, cd, true)))
    clear_learnts(w, cd);
  if (w.lane == 0) w.ws->conflict = 0;
  __syncwarp();
  w.head = 0;
  pf_add(*w.S, w, PF_DB, t0);
}

// luby(i), i >= 1: 1 1 2 1 1 2 4 1 1 2 1 1 2 4 8 ...: luby(2^k - 1) = 2^(k-1);
// otherwise the sequence repeats itself, luby(i) = luby(i - 2^(k-1) + 1) for
// 2^(k-1) <= i < 2^k - 1 (Luby, Sinclair and Zuckerman).
__device__ uint32_t luby_cd(uint32_t i) {
  for (;;) {
    uint32_t k = 1;
    while (k < 31 && (1u << k) - 1u < i) k++;
    if (i == (1u << k) - 1u || k == 31) return 1u << (k - 1);
    i -= (1u << (k - 1)) - 1u;
  }
}

// Learned clauses handed to a cube with its assumptions (all lanes): the
// newest clauses of at most 12 literals and LBD at most 4, as many as fit
// dst[JOB_CLS_WORDS] = [count, words used, offsets[JOB_CLS_MAX], records
// {len, lbd, literals}]. Every learned clause is implied by the formula, so
// the cube may use them whatever its assumptions.
__device__ void export_clauses(Warp& w, CdWarp& cd, uint32_t* dst) {
  constexpr uint32_t base = 2 + JOB_CLS_MAX;
  uint32_t m = 0, used = base;
  for (int64_t k0 = (int64_t)cd.ncl - 1; k0 >= 0 && m < JOB_CLS_MAX; k0 -= 32) {
    const int64_t k = k0 - w.lane;
    uint32_t off = 0, len = 0, lbd = 0, words = 0;
    if (k >= 0) {
      off = cd.cl_off[k];
      len = cd.arena[off];
      lbd = cd.arena[off + 2];
      if (len <= 12u && lbd <= 4u) words = len + 2u;
    }
    uint32_t inc = words;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (w.lane >= d) inc += y;
    }
    const bool ok = words > 0 && used + inc <= JOB_CLS_WORDS;
    const uint32_t okm = __ballot_sync(FULL, ok);
    const uint32_t rank = __popc(okm & ((1u << w.lane) - 1u));
    if (ok && m + rank < JOB_CLS_MAX) {
      const uint32_t at = used + inc - words;
      dst[2 + m + rank] = at;
      dst[at] = len;
      dst[at + 1] = lbd;
      for (uint32_t q = 0; q < len; q++) dst[at + 2 + q] = cd.arena[off + CD_HDR + q];
    }
    const uint32_t taken = min((uint32_t)__popc(okm), JOB_CLS_MAX - m);
    // the prefix sums grow with the lane, so the clauses that fit are a prefix
    const int last = taken ? __fns(okm, 0, taken) : -1;
    if (taken) used += __shfl_sync(FULL, inc, last);
    m += taken;
    if (__popc(okm) < __popc(__ballot_sync(FULL, words > 0))) break;  // buffer full
  }
  if (w.lane == 0) {
    dst[0] = m;
    dst[1] = used;
  }
  __syncwarp();
}

// The clauses a donor attached to this cube (see export_clauses) into the
// empty database, then its watch lists. Returns false (the database is left
// empty) if they do not fit.
__device__ bool import_clauses(Warp& w, CdWarp& cd, const uint32_t* src) {
  const uint32_t m = min(src[0], JOB_CLS_MAX);
  uint32_t top = 0;
  for (uint32_t k0 = 0; k0 < m; k0 += 32) {
    const uint32_t k = k0 + w.lane;
    uint32_t at = 0, len = 0, words = 0;
    if (k < m) {
      at = src[2 + k];
      if (at >= 2 + JOB_CLS_MAX && at + 2 < JOB_CLS_WORDS) {
        len = src[at];
        if (at + 2 + len <= JOB_CLS_WORDS && len >= 2u && len <= 12u) words = clause_words(len);
      }
    }
    uint32_t inc = words;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (w.lane >= d) inc += y;
    }
    const uint32_t c = top + inc - words;
    const uint32_t okm = __ballot_sync(FULL, words > 0);
    if (!__all_sync(FULL, !words || c + words <= cd.arena_words)) {  // no room
      clear_learnts(w, cd);
      return false;
    }
    if (words) {
      cd.arena[c] = len;
      cd.arena[c + 1] = 0u;
      cd.arena[c + 2] = src[at + 1];
      cd.arena[c + 3] = 0u;
      for (uint32_t q = 0; q < words - CD_HDR; q++)
        cd.arena[c + CD_HDR + q] = q < len ? src[at + 2 + q] : NONE;
      cd.cl_off[cd.ncl + __popc(okm & ((1u << w.lane) - 1u))] = c;
    }
    top += __shfl_sync(FULL, inc, 31);
    cd.ncl += __popc(okm);
    __syncwarp();
  }
  cd.top = top;
  if (!rebuild_watches(w, cd)) {
    clear_learnts(w, cd);
    return false;
  }
  return true;
}

// Highest-activity unassigned variable (ties: lowest id) over the 4-bit
// assignment; NONE if all are assigned.
__device__ uint32_t pick_cd(Warp& w) {
  float best_a = -1.0f;
  uint32_t best_v = NONE;
  const uint32_t nwords = (w.V + 7u) >> 3;
  for (uint32_t k = w.lane; k < nwords; k += 32) {
    const uint32_t word = w.asg[k];
    uint32_t un = ~(word | (word >> 1)) & 0x11111111u;  // value bits 00
    const uint32_t lim = w.V - 8u * k;
    if (lim < 8u) un &= (1u << (4u * lim)) - 1u;
    while (un) {
      const uint32_t bitpos = __ffs(un) - 1;
      un &= un - 1u;
      const uint32_t v = 8u * k + (bitpos >> 2);
      const float a = w.act[v];
      if (a > best_a || (a == best_a && v < best_v)) {
        best_a = a;
        best_v = v;
      }
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    const float oa = __shfl_xor_sync(FULL, best_a, d);
    const uint32_t ov = __shfl_xor_sync(FULL, best_v, d);
    if (oa > best_a || (oa == best_a && ov < best_v)) {
      best_a = oa;
      best_v = ov;
    }
  }
  return best_v;
}

// ---- clauses shared between the jobs of one instance ----------------------
//
// Every learned clause is implied by the formula alone (assumption literals
// enter it as decisions, level-0 literals are dropped only when false at
// level 0), so any job of the same instance may use it, whatever its own
// assumptions. Jobs that run beside others of their instance publish their
// short, low-LBD learned clauses to a per-instance pool and read the others'
// at each restart. A pool is a ring of fixed-size records in global memory:
// a writer reserves record r with one atomicAdd on the pool's cursor, writes
// the body, fences, then writes the header r + 1. A reader takes record r only
// if its header reads r + 1 before the body and the cursor shows, after the
// body, that no writer can have reserved the record's slot again (cursor <=
// r + cap). Records that fail either check are skipped, never guessed.

// Publish learnt[0..n) (1 <= n <= SHARE_MAXLEN) with its LBD (all lanes).
__device__ void share_publish(const Solve& S, Warp& w, CdWarp& cd, uint32_t n, uint32_t lbd,
                              int64_t slot) {
  const uint32_t p = (uint32_t)w.inst & S.share_mask;
  unsigned long long r = 0;
  if (w.lane == 0) r = atomicAdd(&S.share_cur[p], 1ull);
  r = __shfl_sync(FULL, r, 0);
  uint32_t* rec =
      S.share + ((size_t)p * S.share_cap + (uint32_t)(r & (S.share_cap - 1u))) * SHARE_REC;
  if (w.lane >= 1 && w.lane < (int)SHARE_REC) {
    uint32_t x;
    if (w.lane == 1) x = (uint32_t)w.inst;
    else if (w.lane == 2) x = n | (min(lbd, 255u) << 8);
    else if (w.lane == 3) x = (uint32_t)slot;
    else x = (uint32_t)(w.lane - 4) < n ? cd.learnt[w.lane - 4] : NONE;
    *(volatile uint32_t*)&rec[w.lane] = x;
  }
  __threadfence();
  __syncwarp();
  if (w.lane == 0) *(volatile uint32_t*)&rec[0] = (uint32_t)(r + 1ull);
  __syncwarp();
}

// Read the pool's records published since *rd by other jobs of this
// instance, at most 256 per call, into the learned-clause database (all
// lanes, at the bottom level after a restart). Each clause is watched on two
// literals that are not false if it has them, else on its one such literal
// and the false literal of highest level; a clause with one open literal
// left implies it, one with none refutes the job. Returns false in that
// case (the job's assumptions contradict the formula), true otherwise.
__device__ bool share_import(const Solve& S, Warp& w, CdWarp& cd, int64_t slot,
                             unsigned long long& rd) {
  const uint32_t p = (uint32_t)w.inst & S.share_mask;
  const unsigned long long cap = S.share_cap;
  unsigned long long cur = 0;
  if (w.lane == 0) cur = *(volatile unsigned long long*)&S.share_cur[p];
  cur = __shfl_sync(FULL, cur, 0);
  unsigned long long from = rd;
  if (cur > cap / 2 && from < cur - cap / 2) from = cur - cap / 2;  // skip what may be overwritten
  const unsigned long long to = min(cur, from + 256ull);
  const uint64_t no_reason = ~0ull;
  bool ok_all = true;
  for (unsigned long long base = from; base < to && ok_all; base += 32) {
    const unsigned long long r = base + (unsigned long long)w.lane;
    bool ok = r < to;
    uint32_t n = 0, lbd = 0, lit[SHARE_MAXLEN];
    const uint32_t* rec = S.share + ((size_t)p * S.share_cap + (uint32_t)(r & (cap - 1u))) * SHARE_REC;
    if (ok) ok = *(const volatile uint32_t*)&rec[0] == (uint32_t)(r + 1ull);
    if (ok) {
      __threadfence();
      const uint32_t ins = *(const volatile uint32_t*)&rec[1];
      const uint32_t nl = *(const volatile uint32_t*)&rec[2];
      const uint32_t prod = *(const volatile uint32_t*)&rec[3];
      n = nl & 255u;
      lbd = nl >> 8;
      ok = ins == (uint32_t)w.inst && prod != (uint32_t)slot && n >= 1 && n <= SHARE_MAXLEN;
#pragma unroll
      for (uint32_t k = 0; k < SHARE_MAXLEN; k++) {
        lit[k] = *(const volatile uint32_t*)&rec[4 + k];
        if (k < n && lit[k] >= 2u * w.V) ok = false;
      }
      __threadfence();
      const unsigned long long now = *(volatile unsigned long long*)&S.share_cur[p];
      if (now > r + cap) ok = false;  // the slot may hold a newer record by now
    }
    for (uint32_t todo = __ballot_sync(FULL, ok); todo && ok_all; todo &= todo - 1u) {
      const int j = __ffs(todo) - 1;
      const uint32_t nj = __shfl_sync(FULL, n, j), lbdj = __shfl_sync(FULL, lbd, j);
      uint32_t my = NONE;
#pragma unroll
      for (uint32_t k = 0; k < SHARE_MAXLEN; k++) {
        const uint32_t x = __shfl_sync(FULL, lit[k], j);
        if ((uint32_t)w.lane == k) my = x;
      }
      const bool have = (uint32_t)w.lane < nj;
      const uint32_t val = have ? lit_value_cd(w.asg, my) : LV_F;
      const uint32_t lvl = have && val == LV_F ? cd.var[my >> 1].level : 0u;
      const uint32_t nf = __ballot_sync(FULL, have && val != LV_F);
      if (nf == 0u) {  // every literal false: the job's assumptions are refuted
        ok_all = false;
        break;
      }
      const int w0 = __ffs(nf) - 1;
      int w1 = -1;
      if (__popc(nf) >= 2) {
        w1 = __fns(nf, 0, 2);
      } else if (nj >= 2) {  // the false literal of the highest level (lowest lane on ties)
        const bool cand = have && w.lane != w0;
        uint32_t best = cand ? lvl : 0u;
        for (int d = 16; d > 0; d >>= 1) best = max(best, __shfl_xor_sync(FULL, best, d));
        w1 = __ffs(__ballot_sync(FULL, cand && lvl == best)) - 1;
      }
      const bool unit = __popc(nf) == 1 && __shfl_sync(FULL, val, w0) == LV_U;
      const uint32_t first = __shfl_sync(FULL, my, w0);
      if (nj == 1) {  // a unit clause: its literal holds in every model
        if (unit && w.lane == 0) imply_cd(w, cd, first, no_reason, 0u);
        __syncwarp();
        continue;
      }
      if ((uint64_t)cd.top + clause_words(nj) > cd.arena_words || cd.full) break;
      // the two watches first, then the rest in record order
      const uint32_t rest = __ballot_sync(FULL, have) & ~(1u << w0) & ~(1u << w1);
      if (have) {
        uint32_t at;
        if (w.lane == w0) at = 0;
        else if (w.lane == w1) at = 1;
        else at = 2u + __popc(rest & ((1u << w.lane) - 1u));
        cd.learnt[at] = my;
      }
      __syncwarp();
      const uint32_t c = add_learnt(w, cd, nj, lbdj);
      if (unit) {
        if (w.lane == 0) imply_cd(w, cd, cd.learnt[0], (uint64_t)(LEARNT_REF | c), 0u);
        __syncwarp();
      }
    }
  }
  rd = to;
  __syncwarp();
  return ok_all;
}

// One job: an instance, or a cube of it (the job's literals as assumptions,
// from the subtree-sharing ring), start to verdict. Returns SAT, UNSAT (for a
// cube: no model extends it) or UNKNOWN.
__device__ int run_cdcl(const Solve& S, Warp& w, int64_t slot, int unit, int inst,
                        const TakenJob* job, uint2* ring, int& abort_code) {
  CdWarp cd;
  cd.ring = ring;
  cd.cand = ring + RING;
  cd.var = reinterpret_cast<VarInfo*>(S.cd_var) + slot * S.vmax;
  for (uint32_t k = w.lane; k < RING; k += 32) ring[k] = make_uint2(NONE, NONE);
  cd.mark = S.cd_mark + slot * S.vmax;
  cd.wl = S.cd_wl + slot * 2 * S.vmax;
  cd.pool = S.cd_pool + slot * S.cd_pool_cap;
  cd.arena = S.cd_arena + slot * S.cd_arena_words;
  cd.learnt = S.cd_learnt + slot * S.vmax;
  cd.cl_off = S.cd_clidx + slot * (S.cd_arena_words / 8);
  cd.arena_words = (uint32_t)S.cd_arena_words;
  cd.ncl = 0;
  cd.pool_cap = (uint32_t)S.cd_pool_cap;
  cd.top = 0;
  cd.pool_top = 0;
  cd.full = 0;
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
  w.inc = job ? job->inc : 1.0f;  // a cube starts from its donor's activities
  const uint32_t nwords = (w.V + 7u) >> 3;
  for (uint32_t k = w.lane; k < nwords; k += 32) w.asg[k] = 0u;
  for (uint32_t v = w.lane; v < w.V; v += 32) {
    if (!job) w.act[v] = 0.0f;
    cd.mark[v] = 0;
  }
  clear_learnts(w, cd);
  if (job && job->cls) import_clauses(w, cd, job->cls);  // the donor's clauses
  if (w.lane == 0) {
    w.ws->tail = 0;
    w.ws->conflict = 0;
  }
  __syncwarp();
  if (S.flags[inst] & F_EMPTY) return SCUBA_UNSAT;
  const uint64_t no_reason = ~0ull;
  const uint32_t nu = S.nunits[inst];
  const uint32_t* un = S.units + w.c0;
  for (uint32_t k = w.lane; k < nu; k += 32)
    if (!imply_cd(w, cd, un[k], no_reason, 0u)) record_conflict(w, un[k], NONE, NONE);
  __syncwarp();
  if (w.ws->conflict) return SCUBA_UNSAT;
  if (job) {  // the cube's literals as decisions of levels 1, 2, ...
    for (int k = 0; k < job->len; k++) {
      if (bcp_cd(w, cd)) return SCUBA_UNSAT;
      const uint32_t l = job->lit[k];
      const uint32_t val = lit_value_cd(w.asg, l);
      if (val == LV_F) return SCUBA_UNSAT;
      if (val == LV_T) continue;
      if (w.lane == 0) w.dstack[WIDX(w, w.nd, (uint32_t)S.vmax, 19)] = *(volatile uint32_t*)&w.ws->tail;
      w.nd++;
      if (w.lane == 0) imply_cd(w, cd, l, no_reason, 0u);
      __syncwarp();
    }
    w.nd_fixed = w.nd;
  }

  // fixed levels that are the unit's own assumptions, not cube literals
  const uint32_t asm_levels =
      S.unit_asm_begin ? (uint32_t)min(S.unit_asm_begin[unit + 1] - S.unit_asm_begin[unit],
                                       (int64_t)MAX_PREFIX)
                       : 0u;
  uint32_t iter = 0, conflicts = 0, since_restart = 0, restart_no = 1;
  uint32_t next_reduce = 2000u, reductions = 0;  // periodic database reduction
  uint32_t restart_at = (uint32_t)S.restart_unit * luby_cd(1);
  // clause sharing with the other jobs of this instance: on for a cube and
  // once this job has given one away or sees others running
  bool shared = S.share_lbd > 0 && job != nullptr;
  unsigned long long share_rd = 0;
  for (;;) {
    if ((++iter & 63u) == 0u) {
      int stop = 0;
      if (w.lane == 0) {
        if (S.abort_flag && *S.abort_flag) stop = 1;
        else if (globaltimer() - S.ctrl->t0 > S.time_ns) stop = 2;
        else if (*(volatile uint32_t*)&S.done[unit] & 1u) stop = 3;
#ifdef SCUBA_CHECKED
        else if (batch_failed(S.ctrl)) stop = 4;  // a bounds check failed: stop
#endif
      }
      stop = __shfl_sync(FULL, stop, 0);
      if (stop == 4) { abort_code = SCUBA_ERR_INTERNAL; return SCUBA_UNKNOWN; }
      if (stop == 1) { abort_code = SCUBA_ERR_ABORTED; return SCUBA_UNKNOWN; }
      if (stop == 2) { abort_code = SCUBA_ERR_TIMEOUT; return SCUBA_UNKNOWN; }
      if (stop == 3) return SCUBA_UNSAT;  // the instance is SAT already; this cube is moot
    }
    long long t0 = pf_now(S);
    const bool confl = bcp_cd(w, cd);
    pf_add(S, w, PF_BCP, t0);
    if (cd.full) {  // the watch pool ran out: compact it (or halve the clauses)
      maintain_db(w, cd, false);
      continue;
    }
    if (confl) {
      WCOUNT(w, conflicts, 1);
      if (w.nd <= w.nd_fixed) return SCUBA_UNSAT;
      conflicts++;
      since_restart++;
      t0 = pf_now(S);
      uint32_t blev, lbd;
      const uint32_t n = analyze_cd(w, cd, blev, lbd);
      if (n == 0) {
        abort_code = SCUBA_ERR_INTERNAL;
        return SCUBA_UNKNOWN;
      }
      if (shared && n <= SHARE_MAXLEN && (n == 1 || lbd <= S.share_lbd))
        share_publish(S, w, cd, n, lbd, slot);
      w.inc *= (1.0f / 0.95f);
      if (w.lane == 0) w.ws->conflict = 0;
      const uint32_t target = max(blev, w.nd_fixed);
      if (n >= 2 && (uint64_t)cd.top + clause_words(n) > cd.arena_words) {
        maintain_db(w, cd, true);  // arena full: restart with half the clauses
        if ((uint64_t)cd.top + clause_words(n) > cd.arena_words) clear_learnts(w, cd);
        since_restart = 0;
      } else {
        backjump_cd(w, cd, target);
      }
      uint64_t why = no_reason;
      if (n >= 2) {
        uint32_t c = add_learnt(w, cd, n, lbd);
        if (cd.full) {  // the pool ran out: compact it, the new clause included
          maintain_db(w, cd, false);
          // the newest clause survives a compaction or a halving; after a
          // full drop it is added again to the empty database
          c = cd.ncl > 0 ? cd.cl_off[cd.ncl - 1] : add_learnt(w, cd, n, lbd);
        }
        why = (uint64_t)(LEARNT_REF | c);
      }
      // the clause is unit once every literal but the first is false
      if (n == 1 || blev <= w.nd) {
        if (w.lane == 0) imply_cd(w, cd, cd.learnt[0], why, 0u);
        __syncwarp();
      }
      pf_add(S, w, PF_ANALYZE, t0);
      if (S.budget > 0) {  // conflicts of the instance, all of its cubes together
        unsigned long long tot = 0;
        if (w.lane == 0) tot = atomicAdd(&S.inst_dec[unit], 1ull) + 1ull;
        tot = __shfl_sync(FULL, tot, 0);
        if ((int64_t)tot >= S.budget) return SCUBA_UNKNOWN;
      }
      continue;
    }
    if (since_restart >= restart_at) {
      since_restart = 0;
      restart_no++;
      restart_at = (uint32_t)S.restart_unit * luby_cd(restart_no);
      if (conflicts >= next_reduce) {  // a restart that also halves the database
        reductions++;
        next_reduce = conflicts + 2000u + 300u * reductions;
        maintain_db(w, cd, true);
      } else {
        backjump_cd(w, cd, w.nd_fixed);
      }
      if (S.share_lbd > 0 && !shared) {
        uint32_t others = 0;
        if (w.lane == 0) others = *(volatile uint32_t*)&S.pending[unit] > 1u;
        shared = __shfl_sync(FULL, others, 0) != 0u;
      }
      if (shared && !share_import(S, w, cd, slot, share_rd)) return SCUBA_UNSAT;
      continue;
    }
    WCOUNT(w, act_reads, w.V - *(volatile uint32_t*)&w.ws->tail);
    t0 = pf_now(S);
    const uint32_t v = pick_cd(w);
    pf_add(S, w, PF_DECIDE, t0);
    if (v == NONE) {
      // the first cube of the instance to reach a model writes it
      uint32_t won = 0;
      if (w.lane == 0) won = !(atomicOr(&S.done[unit], 8u) & 8u);
      won = __shfl_sync(FULL, won, 0);
      if (won && S.model)
        for (uint32_t x = w.lane; x < w.V; x += 32) {
          S.model[(S.unit_vb ? S.unit_vb[unit] : S.vb[inst]) + x] =
              (nib(w.asg, x) & 3u) == NB_T ? 1 : 0;
        }
      __syncwarp();
      return SCUBA_SAT;
    }
    // cube-and-conquer: hand the other side of the first free decision to an
    // idle warp and keep this side as an assumption, up to split_depth cube
    // levels below the instance. A cube relearns almost from scratch, so a
    // job should share only once it has shown itself hard (split_min
    // decisions): splitting easy jobs whenever warps are idle can cost an
    // instance that needs a few hundred conflicts alone millions of them
    if (S.split && w.decisions >= (uint32_t)S.split_min &&
        (w.decisions % (uint32_t)S.split_interval) == 0 && w.nd > w.nd_fixed &&
        w.nd_fixed + 1 <= (uint32_t)MAX_PREFIX &&
        w.nd_fixed < asm_levels + (uint32_t)S.split_depth) {
      uint32_t idle = 0;
      if (w.lane == 0) idle = *(volatile uint32_t*)&S.ctrl->idle;
      idle = __shfl_sync(FULL, idle, 0);
      if (idle > 0) {
        const uint32_t k = w.nd_fixed;
        if (w.lane == 0) atomicAdd(&S.pending[unit], 1u);
        __syncwarp();
        if (ring_push(S, w, unit, k + 1, w.trail, w.dstack, k, [&](uint32_t cell) {
              export_clauses(w, cd, S.job_cls + (size_t)cell * JOB_CLS_WORDS);
            })) {
          w.nd_fixed = k + 1;
          shared = S.share_lbd > 0;
          if (w.lane == 0) {
            atomicAdd(&S.ctrl->jobs_split, 1u);
            if (S.prof) {
              atomicAdd(&S.prof[0], 1ull);
              atomicAdd(&S.prof[2], (unsigned long long)(k + 1));
              atomicAdd(&S.prof[3], (unsigned long long)(w.nd - k));
            }
          }
        } else if (w.lane == 0) {
          atomicSub(&S.pending[unit], 1u);
          if (S.prof) atomicAdd(&S.prof[4], 1ull);
        }
        __syncwarp();
      }
    }
    w.decisions++;
    WCOUNT(w, decisions, 1);
    const uint32_t lit = 2u * v + ((cd.mark[v] & MK_PHASE) ? 0u : 1u);
    if (w.lane == 0) w.dstack[WIDX(w, w.nd, (uint32_t)S.vmax, 19)] = *(volatile uint32_t*)&w.ws->tail;
    w.nd++;
    if (w.lane == 0) imply_cd(w, cd, lit, no_reason, 0u);
    __syncwarp();
  }
}
