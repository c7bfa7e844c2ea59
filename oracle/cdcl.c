/*
 * cdcl.c -- plain conflict-driven clause learning for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY: the product library never links or loads it.
 *
 * What it computes: the same verdict as oracle_dpll, i.e. whether the CNF
 * (and so the query, Sec. V-B, step 10) is satisfiable. The paper hands the
 * constraints to OR-Tools' SAT solver, which learns clauses internally but
 * is not described further; this file is the textbook loop that such
 * solvers share:
 *
 *   - unit propagation over two watched literals per clause;
 *   - on a conflict, the first-UIP clause: resolve the conflicting clause
 *     with the reasons of current-level literals, newest first on the trail,
 *     until exactly one current-level literal is left;
 *   - a non-chronological backjump to the second-highest level of that
 *     clause, where it is unit, and assert its UIP literal;
 *   - decisions on the unassigned variable of highest activity (ties: lowest
 *     id); every variable met during an analysis is bumped, the increment
 *     grows by 1/0.95 per conflict; the value is the variable's last value
 *     (false at first);
 *   - restarts after 100 * luby(k) conflicts; no clause deletion and no
 *     clause minimisation.
 *
 * Every learned clause is appended (DIMACS, 0-terminated) to the trace, and
 * a refutation ends with the empty clause, so rup.c can check an UNSAT
 * verdict; a SAT verdict comes with a model that satisfies every clause.
 * The budget counts conflicts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_UNSAT = 0, K_SAT = 1, K_UNKNOWN = 2, K_ERROR = 3 };

typedef struct {
  int64_t *a;
  int64_t n, cap;
} ivec_t;

static int ivec_push(ivec_t *v, int64_t x) {
  if (v->n == v->cap) {
    int64_t cap = v->cap ? 2 * v->cap : 4;
    int64_t *a = (int64_t *)realloc(v->a, sizeof(int64_t) * (size_t)cap);
    if (!a) return -1;
    v->a = a;
    v->cap = cap;
  }
  v->a[v->n++] = x;
  return 0;
}

typedef struct {
  int nv;
  /* clauses: literals L[cstart[c] .. cstart[c]+clen[c]) (DIMACS) */
  int32_t *L;
  int64_t nL, capL;
  int64_t *cstart;
  int32_t *clen;
  int64_t ncl, capC;
  ivec_t *watch;       /* [2 nv + 2]: clauses watching literal l, at wi(l) */
  int8_t *val;         /* [nv+1] -1 open, 0 false, 1 true */
  int32_t *level;      /* [nv+1] */
  int64_t *reason;     /* [nv+1] clause that implied the variable, -1 none */
  int8_t *phase;       /* [nv+1] last value */
  uint8_t *seen;       /* [nv+1] */
  int32_t *trail;      /* [nv] true literals in assignment order */
  int64_t tlen, qhead;
  int32_t *lim;        /* [nv+1] trail length at the start of each level */
  int nlev;
  double *act, inc;
  int32_t *heap, *hpos; /* max-heap of variables by activity; hpos -1 = absent */
  int hn;
  int32_t *learnt;     /* [nv+1] scratch */
  int64_t decisions, conflicts, propagations;
  int32_t *tr;         /* trace */
  int64_t trcap, trlen;
  int troverflow;
} S_t;

static inline int avar(int l) { return l > 0 ? l : -l; }
static inline int64_t wi(int l) { return 2 * (int64_t)avar(l) + (l < 0); }
static inline int lval(const S_t *s, int l) {
  int v = s->val[avar(l)];
  if (v < 0) return -1;
  return l > 0 ? v : 1 - v;
}

static void trace_add(S_t *s, const int32_t *c, int n) {
  if (!s->tr) return;
  if (s->trlen + n + 1 > s->trcap) { s->troverflow = 1; return; }
  for (int i = 0; i < n; i++) s->tr[s->trlen++] = c[i];
  s->tr[s->trlen++] = 0;
}

/* ---- activity heap ------------------------------------------------------ */

static inline int better(const S_t *s, int a, int b) {
  return s->act[a] > s->act[b] || (s->act[a] == s->act[b] && a < b);
}

static void heap_up(S_t *s, int i) {
  int x = s->heap[i];
  while (i > 0) {
    int p = (i - 1) / 2;
    if (!better(s, x, s->heap[p])) break;
    s->heap[i] = s->heap[p];
    s->hpos[s->heap[i]] = i;
    i = p;
  }
  s->heap[i] = x;
  s->hpos[x] = i;
}

static void heap_down(S_t *s, int i) {
  int x = s->heap[i];
  for (;;) {
    int c = 2 * i + 1;
    if (c >= s->hn) break;
    if (c + 1 < s->hn && better(s, s->heap[c + 1], s->heap[c])) c++;
    if (!better(s, s->heap[c], x)) break;
    s->heap[i] = s->heap[c];
    s->hpos[s->heap[i]] = i;
    i = c;
  }
  s->heap[i] = x;
  s->hpos[x] = i;
}

static void heap_insert(S_t *s, int v) {
  if (s->hpos[v] >= 0) return;
  s->heap[s->hn] = v;
  s->hpos[v] = s->hn;
  s->hn++;
  heap_up(s, s->hn - 1);
}

static int heap_pop(S_t *s) {
  int top = s->heap[0];
  s->hpos[top] = -1;
  s->hn--;
  if (s->hn > 0) {
    s->heap[0] = s->heap[s->hn];
    s->hpos[s->heap[0]] = 0;
    heap_down(s, 0);
  }
  return top;
}

static void bump(S_t *s, int v) {
  s->act[v] += s->inc;
  if (s->act[v] > 1e100) {
    for (int u = 1; u <= s->nv; u++) s->act[u] *= 1e-100;
    s->inc *= 1e-100;
  }
  if (s->hpos[v] >= 0) heap_up(s, s->hpos[v]);
}

/* ---- clauses, assignment ------------------------------------------------ */

static int64_t add_clause(S_t *s, const int32_t *c, int n) {
  if (s->nL + n > s->capL) {
    int64_t cap = s->capL ? 2 * s->capL : 64;
    while (cap < s->nL + n) cap *= 2;
    int32_t *L = (int32_t *)realloc(s->L, sizeof(int32_t) * (size_t)cap);
    if (!L) return -1;
    s->L = L;
    s->capL = cap;
  }
  if (s->ncl == s->capC) {
    int64_t cap = s->capC ? 2 * s->capC : 64;
    int64_t *cs = (int64_t *)realloc(s->cstart, sizeof(int64_t) * (size_t)cap);
    if (!cs) return -1;
    s->cstart = cs;
    int32_t *cl = (int32_t *)realloc(s->clen, sizeof(int32_t) * (size_t)cap);
    if (!cl) return -1;
    s->clen = cl;
    s->capC = cap;
  }
  int64_t id = s->ncl++;
  s->cstart[id] = s->nL;
  s->clen[id] = n;
  memcpy(s->L + s->nL, c, sizeof(int32_t) * (size_t)n);
  s->nL += n;
  if (ivec_push(&s->watch[wi(c[0])], id) || ivec_push(&s->watch[wi(c[1])], id)) return -1;
  return id;
}

static void assign(S_t *s, int l, int64_t why) {
  int v = avar(l);
  s->val[v] = l > 0;
  s->level[v] = s->nlev;
  s->reason[v] = why;
  s->trail[s->tlen++] = l;
}

static void backjump(S_t *s, int lev) {
  if (s->nlev <= lev) return;
  for (int64_t t = s->tlen - 1; t >= s->lim[lev]; t--) {
    int v = avar(s->trail[t]);
    s->phase[v] = s->val[v];
    s->val[v] = -1;
    s->reason[v] = -1;
    heap_insert(s, v);
  }
  s->tlen = s->lim[lev];
  s->qhead = s->tlen;
  s->nlev = lev;
}

/* Two-watched-literal propagation. Returns a falsified clause or -1. */
static int64_t propagate(S_t *s) {
  while (s->qhead < s->tlen) {
    int f = -s->trail[s->qhead++];  /* literal that just became false */
    s->propagations++;
    ivec_t *ws = &s->watch[wi(f)];
    int64_t i = 0, j = 0;
    while (i < ws->n) {
      int64_t c = ws->a[i++];
      int32_t *C = s->L + s->cstart[c];
      int n = s->clen[c];
      if (C[0] == f) { C[0] = C[1]; C[1] = f; }
      if (lval(s, C[0]) == 1) { ws->a[j++] = c; continue; }
      int moved = 0;
      for (int k = 2; k < n; k++) {
        if (lval(s, C[k]) != 0) {
          C[1] = C[k];
          C[k] = f;
          if (ivec_push(&s->watch[wi(C[1])], c)) return -2;
          moved = 1;
          break;
        }
      }
      if (moved) continue;
      ws->a[j++] = c;
      if (lval(s, C[0]) == 0) {
        while (i < ws->n) ws->a[j++] = ws->a[i++];
        ws->n = j;
        return c;
      }
      assign(s, C[0], c);
    }
    ws->n = j;
  }
  return -1;
}

/* First-UIP analysis of conflict clause c. Writes the learned clause to
   s->learnt (the UIP literal first, then a literal of the backjump level)
   and returns its length; *blev receives the backjump level. */
static int analyze(S_t *s, int64_t c, int *blev) {
  int n = 1, path = 0, p = 0;
  int64_t idx = s->tlen - 1;
  for (;;) {
    const int32_t *C = s->L + s->cstart[c];
    for (int k = 0; k < s->clen[c]; k++) {
      int q = C[k];
      int v = avar(q);
      if (p != 0 && v == avar(p)) continue;
      if (s->seen[v] || s->level[v] == 0) continue;
      s->seen[v] = 1;
      bump(s, v);
      if (s->level[v] >= s->nlev) path++;
      else s->learnt[n++] = q;
    }
    while (!s->seen[avar(s->trail[idx])]) idx--;
    p = s->trail[idx--];
    s->seen[avar(p)] = 0;
    path--;
    if (path == 0) break;
    c = s->reason[avar(p)];
  }
  s->learnt[0] = -p;
  int best = 1;
  *blev = 0;
  for (int k = 1; k < n; k++) {
    int lv = s->level[avar(s->learnt[k])];
    if (lv > *blev) { *blev = lv; best = k; }
  }
  if (n > 1) {
    int t = s->learnt[1]; s->learnt[1] = s->learnt[best]; s->learnt[best] = t;
  }
  for (int k = 1; k < n; k++) s->seen[avar(s->learnt[k])] = 0;
  return n;
}

/* luby(i), i >= 1: 1 1 2 1 1 2 4 1 1 2 1 1 2 4 8 ... (Luby, Sinclair and
   Zuckerman): luby(2^k - 1) = 2^(k-1), and otherwise the sequence repeats
   its first 2^(k-1) - 1 terms, so luby(i) = luby(i - 2^(k-1) + 1) for
   2^(k-1) <= i < 2^k - 1. */
static int64_t luby(int64_t i) {
  for (;;) {
    int k = 1;
    while (((int64_t)1 << k) - 1 < i) k++;
    if (i == ((int64_t)1 << k) - 1) return (int64_t)1 << (k - 1);
    i -= ((int64_t)1 << (k - 1)) - 1;
  }
}

static void s_free(S_t *s) {
  if (s->watch)
    for (int64_t i = 0; i < 2 * (int64_t)s->nv + 2; i++) free(s->watch[i].a);
  free(s->watch); free(s->L); free(s->cstart); free(s->clen); free(s->val); free(s->level);
  free(s->reason); free(s->phase); free(s->seen); free(s->trail); free(s->lim);
  free(s->act); free(s->heap); free(s->hpos); free(s->learnt);
}

int oracle_cdcl(int nv, int64_t nc, const int64_t *cb, const int32_t *lits,
                int64_t budget, uint8_t *model, int64_t *stats3, int32_t *trace_buf,
                int64_t trace_cap, int64_t *trace_len) {
  S_t s;
  memset(&s, 0, sizeof(s));
  s.nv = nv;
  s.tr = trace_buf;
  s.trcap = trace_cap;
  s.inc = 1.0;
  int verdict = K_UNKNOWN;
  size_t n1 = (size_t)nv + 1;
  s.watch = (ivec_t *)calloc(2 * n1, sizeof(ivec_t));
  s.val = (int8_t *)malloc(n1);
  s.level = (int32_t *)calloc(n1, sizeof(int32_t));
  s.reason = (int64_t *)malloc(n1 * sizeof(int64_t));
  s.phase = (int8_t *)calloc(n1, 1);
  s.seen = (uint8_t *)calloc(n1, 1);
  s.trail = (int32_t *)malloc(n1 * sizeof(int32_t));
  s.lim = (int32_t *)malloc(n1 * sizeof(int32_t));
  s.act = (double *)calloc(n1, sizeof(double));
  s.heap = (int32_t *)malloc(n1 * sizeof(int32_t));
  s.hpos = (int32_t *)malloc(n1 * sizeof(int32_t));
  s.learnt = (int32_t *)malloc(n1 * sizeof(int32_t));
  int32_t *tmp = (int32_t *)malloc(n1 * sizeof(int32_t));
  if (!s.watch || !s.val || !s.level || !s.reason || !s.phase || !s.seen || !s.trail ||
      !s.lim || !s.act || !s.heap || !s.hpos || !s.learnt || !tmp) {
    verdict = K_ERROR;
    goto done;
  }
  for (int v = 0; v <= nv; v++) { s.val[v] = -1; s.reason[v] = -1; s.hpos[v] = -1; }
  for (int v = 1; v <= nv; v++) heap_insert(&s, v);

  /* original clauses: duplicates removed, tautologies dropped; empty clause
     -> UNSAT, unit clauses are assigned at level 0 */
  for (int64_t c = 0; c < nc; c++) {
    int n = 0, taut = 0;
    for (int64_t q = cb[c]; q < cb[c + 1]; q++) {
      int l = lits[q];
      if (l == 0 || avar(l) > nv) { verdict = K_ERROR; goto done; }
      int dup = 0;
      for (int k = 0; k < n; k++) {
        if (tmp[k] == l) dup = 1;
        if (tmp[k] == -l) taut = 1;
      }
      if (!dup) tmp[n++] = l;
    }
    if (taut) continue;
    if (n == 0) { trace_add(&s, tmp, 0); verdict = K_UNSAT; goto done; }
    if (n == 1) {
      int lv = lval(&s, tmp[0]);
      if (lv == 0) { trace_add(&s, tmp, 0); verdict = K_UNSAT; goto done; }
      if (lv < 0) assign(&s, tmp[0], -1);
      continue;
    }
    if (add_clause(&s, tmp, n) < 0) { verdict = K_ERROR; goto done; }
  }

  int64_t restart_no = 1, since_restart = 0;
  for (;;) {
    int64_t confl = propagate(&s);
    if (confl == -2) { verdict = K_ERROR; break; }
    if (confl >= 0) {
      s.conflicts++;
      since_restart++;
      if (s.nlev == 0) { trace_add(&s, tmp, 0); verdict = K_UNSAT; break; }
      int blev;
      int n = analyze(&s, confl, &blev);
      s.inc /= 0.95;
      trace_add(&s, s.learnt, n);
      backjump(&s, blev);
      if (n == 1) {
        assign(&s, s.learnt[0], -1);
      } else {
        int64_t id = add_clause(&s, s.learnt, n);
        if (id < 0) { verdict = K_ERROR; break; }
        assign(&s, s.learnt[0], id);
      }
      continue;
    }
    if (budget > 0 && s.conflicts >= budget) break;
    if (since_restart >= 100 * luby(restart_no)) {
      since_restart = 0;
      restart_no++;
      backjump(&s, 0);
      continue;
    }
    int v = 0;
    while (s.hn > 0) {
      int u = heap_pop(&s);
      if (s.val[u] < 0) { v = u; break; }
    }
    if (v == 0) { verdict = K_SAT; break; }
    s.decisions++;
    s.lim[s.nlev++] = (int32_t)s.tlen;
    assign(&s, s.phase[v] ? v : -v, -1);
  }
  if (verdict == K_SAT && model)
    for (int v = 1; v <= nv; v++) model[v - 1] = (uint8_t)s.val[v];
done:
  if (stats3) { stats3[0] = s.decisions; stats3[1] = s.conflicts; stats3[2] = s.propagations; }
  if (trace_len) *trace_len = s.troverflow ? -1 : s.trlen;
  free(tmp);
  s_free(&s);
  return verdict;
}
