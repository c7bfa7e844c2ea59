/*
 * oracle.c -- plain CPU reference for the out-of-bounds satisfiability check.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this code. It shares no source with the product
 * library (paper_2601_21552_gb300/csrc) and never includes its headers.
 *
 * What it computes (Sec. IV-A and Sec. V-B of the paper): for one memory
 * access, the constraint set (kind 1: ids below dimensions; kind 2: offset
 * >= size or offset outside its partition; kind 3: equalities defining the
 * offset/size expression trees and the asserts) is satisfiable iff some input
 * makes the access go out of bounds. Verdict SAT = an OOB is possible.
 *
 * Pieces, each written for obviousness rather than speed:
 *   1. ir_*      : parse the serialized query IR (format in workloads/ir.py).
 *   2. enc_*     : bit-blast the IR to CNF with plain Tseitin gates (AND/XOR/OR
 *                  with full equivalences), ripple-carry adders, shift-and-add
 *                  multipliers, LSB-to-MSB comparator chains, division by a
 *                  constant through q,r with x = k*q + r, r < k, and C's
 *                  unsigned k-bit wrap-around as bit selection (truncation)
 *                  and negated bits (complement).
 *   3. dpll_*    : complete DPLL -- occurrence-list unit propagation to a
 *                  fixpoint, decide the unassigned variable of highest
 *                  activity (ties: lowest id), false polarity first, on
 *                  conflict bump the activity of the falsified clause's
 *                  variables and backtrack chronologically to the deepest
 *                  decision not yet flipped. Optionally emits a RUP trace of
 *                  the refuted DPLL tree for the independent checker (rup.c).
 *   4. brute_*   : the plain definition: enumerate every input assignment
 *                  and evaluate the integer constraints exactly.
 *   5. batch     : a pthread pool solving many queries / CNFs.
 *
 * Parity pins live in tests/: brute force, closed forms, the paper's worked
 * examples, model re-verification and RUP checking of UNSAT verdicts.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define IR_MAGIC 0x53435542LL
#define IR_VERSION 1

enum {
  OP_FREE = 1, OP_CONST = 2, OP_ADD = 3, OP_MUL = 4, OP_ULT = 5, OP_ULE = 6,
  OP_EQ = 7, OP_OR = 8, OP_AND = 9, OP_NOT = 10, OP_UDIV = 11, OP_UREM = 12,
  OP_TRUNC = 13, OP_NOTW = 14 /* y: a bit count, not a node */
};

enum { V_UNSAT = 0, V_SAT = 1, V_UNKNOWN = 2, V_ERROR = 3 };

/* ------------------------------------------------------------------------ */
/* 1. IR                                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n, r;
  const int64_t *node; /* n x 4 */
  const int64_t *root; /* r */
} ir_t;

static int ir_open(const int64_t *a, int64_t len, ir_t *ir) {
  if (len < 4 || a[0] != IR_MAGIC || a[1] != IR_VERSION) return -1;
  ir->n = a[2];
  ir->r = a[3];
  if (ir->n < 0 || ir->r < 0 || len != 4 + 4 * ir->n + ir->r) return -1;
  ir->node = a + 4;
  ir->root = a + 4 + 4 * ir->n;
  for (int64_t i = 0; i < ir->n; i++) {
    int64_t op = ir->node[4 * i], x = ir->node[4 * i + 1], y = ir->node[4 * i + 2];
    if (op == OP_FREE) {
      if (x < 1 || x > 64) return -1;
    } else if (op == OP_CONST) {
      if (x < 0) return -1;
    } else if (op == OP_TRUNC || op == OP_NOTW) {
      if (x < 0 || x >= i || y < 1 || y > 64) return -1;
    } else if (op >= OP_ADD && op <= OP_UREM) {
      if (x < 0 || x >= i) return -1;
      if (op != OP_NOT && (y < 0 || y >= i)) return -1;
      if ((op == OP_UDIV || op == OP_UREM) &&
          (ir->node[4 * y] != OP_CONST || ir->node[4 * y + 1] < 1))
        return -1;
    } else {
      return -1;
    }
  }
  for (int64_t i = 0; i < ir->r; i++)
    if (ir->root[i] < 0 || ir->root[i] >= ir->n) return -1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 2. Tseitin encoder                                                        */
/* ------------------------------------------------------------------------ */

/* A "bit" is a DIMACS literal (+-v) or one of the two constants below. */
#define BT 0x7fffffff
#define BF (-0x7fffffff)

typedef struct {
  int nvars;
  int64_t ncl, cap_cl;
  int64_t *cb; /* clause_begin, ncl+1 */
  int64_t nl, cap_l;
  int32_t *lits;
  int failed;
} enc_t;

typedef struct {
  int w;
  int *b; /* LSB first */
} word_t;

static void enc_init(enc_t *e) {
  memset(e, 0, sizeof(*e));
  e->cap_cl = 1024;
  e->cap_l = 4096;
  e->cb = (int64_t *)malloc(sizeof(int64_t) * (e->cap_cl + 1));
  e->lits = (int32_t *)malloc(sizeof(int32_t) * e->cap_l);
  if (!e->cb || !e->lits) e->failed = 1;
  else e->cb[0] = 0;
}

static void enc_free(enc_t *e) {
  free(e->cb);
  free(e->lits);
  e->cb = NULL;
  e->lits = NULL;
}

static int new_var(enc_t *e) { return ++e->nvars; }

static void clause(enc_t *e, int k, const int *l) {
  if (e->failed) return;
  if (e->ncl + 1 > e->cap_cl) {
    e->cap_cl *= 2;
    int64_t *p = (int64_t *)realloc(e->cb, sizeof(int64_t) * (e->cap_cl + 1));
    if (!p) { e->failed = 1; return; }
    e->cb = p;
  }
  if (e->nl + k > e->cap_l) {
    while (e->nl + k > e->cap_l) e->cap_l *= 2;
    int32_t *p = (int32_t *)realloc(e->lits, sizeof(int32_t) * e->cap_l);
    if (!p) { e->failed = 1; return; }
    e->lits = p;
  }
  for (int i = 0; i < k; i++) e->lits[e->nl++] = l[i];
  e->ncl++;
  e->cb[e->ncl] = e->nl;
}

static void cl1(enc_t *e, int a) { int l[1] = {a}; clause(e, 1, l); }
static void cl2(enc_t *e, int a, int b) { int l[2] = {a, b}; clause(e, 2, l); }
static void cl3(enc_t *e, int a, int b, int c) { int l[3] = {a, b, c}; clause(e, 3, l); }

/* z <-> a AND b */
static int g_and(enc_t *e, int a, int b) {
  if (a == BF || b == BF) return BF;
  if (a == BT) return b;
  if (b == BT) return a;
  if (a == b) return a;
  if (a == -b) return BF;
  int z = new_var(e);
  cl2(e, -z, a);
  cl2(e, -z, b);
  cl3(e, z, -a, -b);
  return z;
}

/* z <-> a OR b, by De Morgan */
static int g_or(enc_t *e, int a, int b) { return -g_and(e, -a, -b); }

/* z <-> a XOR b */
static int g_xor(enc_t *e, int a, int b) {
  if (a == BF) return b;
  if (b == BF) return a;
  if (a == BT) return -b;
  if (b == BT) return -a;
  if (a == b) return BF;
  if (a == -b) return BT;
  int z = new_var(e);
  cl3(e, -z, a, b);
  cl3(e, -z, -a, -b);
  cl3(e, z, -a, b);
  cl3(e, z, a, -b);
  return z;
}

static word_t w_new(int w) {
  word_t r;
  r.w = w;
  r.b = (int *)malloc(sizeof(int) * (w > 0 ? w : 1));
  for (int i = 0; i < w; i++) r.b[i] = BF;
  return r;
}

static int w_bit(const word_t *x, int i) { return i < x->w ? x->b[i] : BF; }

/* exact sum: width max(wa, wb) + 1, ripple carry */
static word_t w_add(enc_t *e, const word_t *a, const word_t *b) {
  int W = (a->w > b->w ? a->w : b->w) + 1;
  word_t s = w_new(W);
  int carry = BF;
  for (int i = 0; i < W; i++) {
    int x = w_bit(a, i), y = w_bit(b, i);
    int xy = g_xor(e, x, y);
    s.b[i] = g_xor(e, xy, carry);
    carry = g_or(e, g_and(e, x, y), g_and(e, carry, xy));
  }
  return s;
}

/* exact product: width wa + wb, shift-and-add over the bits of b */
static word_t w_mul(enc_t *e, const word_t *a, const word_t *b) {
  int W = a->w + b->w;
  word_t acc = w_new(W);
  for (int j = 0; j < b->w; j++) {
    word_t pp = w_new(W);
    for (int i = 0; i < a->w && i + j < W; i++) pp.b[i + j] = g_and(e, a->b[i], b->b[j]);
    word_t t = w_add(e, &acc, &pp);
    for (int i = 0; i < W; i++) acc.b[i] = t.b[i]; /* product < 2^W: top carry is 0 */
    free(t.b);
    free(pp.b);
  }
  return acc;
}

/* x < y over the zero-extended common width, LSB to MSB:
   lt_i = (!x_i & y_i) | ((x_i == y_i) & lt_{i-1}) */
static int w_ult(enc_t *e, const word_t *x, const word_t *y) {
  int W = x->w > y->w ? x->w : y->w;
  int lt = BF;
  for (int i = 0; i < W; i++) {
    int xi = w_bit(x, i), yi = w_bit(y, i);
    int here = g_and(e, -xi, yi);
    int same = -g_xor(e, xi, yi);
    lt = g_or(e, here, g_and(e, same, lt));
  }
  return lt;
}

static int w_eq(enc_t *e, const word_t *x, const word_t *y) {
  int W = x->w > y->w ? x->w : y->w;
  int all = BT;
  for (int i = 0; i < W; i++) all = g_and(e, all, -g_xor(e, w_bit(x, i), w_bit(y, i)));
  return all;
}

static word_t w_const(uint64_t v) {
  int w = 1;
  while (w < 64 && (v >> w)) w++;
  word_t r = w_new(w);
  for (int i = 0; i < w; i++) r.b[i] = ((v >> i) & 1) ? BT : BF;
  return r;
}

static void assert_bit(enc_t *e, int b) {
  if (b == BT) return;
  if (b == BF) { clause(e, 0, NULL); return; }
  cl1(e, b);
}

typedef struct {
  int nvars;
  int64_t ncl, nl;
  int64_t *cb;
  int32_t *lits;
  int n_free;
  int *free_width;  /* per FREE node */
  int32_t *in_map;  /* concatenated FREE bits, LSB first */
} ocnf_t;

ocnf_t *oracle_encode(const int64_t *a, int64_t len) {
  ir_t ir;
  if (ir_open(a, len, &ir)) return NULL;
  enc_t e;
  enc_init(&e);
  word_t *wd = (word_t *)calloc((size_t)(ir.n ? ir.n : 1), sizeof(word_t));
  int *bl = (int *)calloc((size_t)(ir.n ? ir.n : 1), sizeof(int));
  /* division results: q and r per (x, k) node pair; stored on the UDIV/UREM node */
  word_t *q_of = (word_t *)calloc((size_t)(ir.n ? ir.n : 1), sizeof(word_t));
  word_t *r_of = (word_t *)calloc((size_t)(ir.n ? ir.n : 1), sizeof(word_t));
  ocnf_t *out = (ocnf_t *)calloc(1, sizeof(ocnf_t));

  /* input words first, MSB with the lowest variable id */
  int n_free = 0, free_bits = 0;
  for (int64_t i = 0; i < ir.n; i++)
    if (ir.node[4 * i] == OP_FREE) { n_free++; free_bits += (int)ir.node[4 * i + 1]; }
  out->n_free = n_free;
  out->free_width = (int *)malloc(sizeof(int) * (n_free ? n_free : 1));
  out->in_map = (int32_t *)malloc(sizeof(int32_t) * (free_bits ? free_bits : 1));
  int fi = 0, fb = 0;
  for (int64_t i = 0; i < ir.n; i++) {
    if (ir.node[4 * i] != OP_FREE) continue;
    int w = (int)ir.node[4 * i + 1];
    wd[i] = w_new(w);
    int base = e.nvars;
    e.nvars += w;
    for (int k = 0; k < w; k++) wd[i].b[k] = base + (w - k);
    out->free_width[fi++] = w;
    for (int k = 0; k < w; k++) out->in_map[fb++] = wd[i].b[k];
  }

  for (int64_t i = 0; i < ir.n; i++) {
    int64_t op = ir.node[4 * i], x = ir.node[4 * i + 1], y = ir.node[4 * i + 2];
    switch (op) {
      case OP_FREE: break;
      case OP_CONST: wd[i] = w_const((uint64_t)x); break;
      case OP_ADD: wd[i] = w_add(&e, &wd[x], &wd[y]); break;
      case OP_MUL: wd[i] = w_mul(&e, &wd[x], &wd[y]); break;
      case OP_TRUNC: { /* C unsigned conversion to y bits: keep the low y bits */
        int w = wd[x].w < y ? wd[x].w : (int)y;
        wd[i] = w_new(w);
        for (int k = 0; k < w; k++) wd[i].b[k] = wd[x].b[k];
        break;
      }
      case OP_NOTW: /* bitwise complement of the low y bits (missing bits are 0) */
        wd[i] = w_new((int)y);
        for (int k = 0; k < y; k++) wd[i].b[k] = -w_bit(&wd[x], k);
        break;
      case OP_UDIV:
      case OP_UREM: {
        /* look for an earlier division of the same operand by the same constant */
        int64_t twin = -1;
        for (int64_t j = 0; j < i; j++) {
          int64_t oj = ir.node[4 * j];
          if ((oj == OP_UDIV || oj == OP_UREM) && ir.node[4 * j + 1] == x &&
              ir.node[4 * j + 2] == y) { twin = j; break; }
        }
        word_t q, r;
        if (twin >= 0) {
          q = q_of[twin];
          r = r_of[twin];
        } else {
          uint64_t k = (uint64_t)ir.node[4 * y + 1];
          int wq = wd[x].w;
          q = w_new(wq);
          for (int t = 0; t < wq; t++) q.b[t] = new_var(&e);
          int wr = 1;
          while (wr < 64 && ((k - 1) >> wr)) wr++;
          r = w_new(wr);
          if (k > 1) for (int t = 0; t < wr; t++) r.b[t] = new_var(&e);
          word_t kw = w_const(k);
          word_t kq = w_mul(&e, &kw, &q);
          word_t sum = w_add(&e, &kq, &r);
          assert_bit(&e, w_eq(&e, &sum, &wd[x])); /* x = k*q + r */
          assert_bit(&e, w_ult(&e, &r, &kw));     /* r < k */
          free(kw.b); free(kq.b); free(sum.b);
        }
        q_of[i] = q;
        r_of[i] = r;
        word_t *src = op == OP_UDIV ? &q : &r;
        wd[i] = w_new(src->w);
        memcpy(wd[i].b, src->b, sizeof(int) * src->w);
        break;
      }
      case OP_ULT: bl[i] = w_ult(&e, &wd[x], &wd[y]); break;
      case OP_ULE: bl[i] = -w_ult(&e, &wd[y], &wd[x]); break;
      case OP_EQ: bl[i] = w_eq(&e, &wd[x], &wd[y]); break;
      case OP_OR: bl[i] = g_or(&e, bl[x], bl[y]); break;
      case OP_AND: bl[i] = g_and(&e, bl[x], bl[y]); break;
      case OP_NOT: bl[i] = -bl[x]; break;
    }
  }
  for (int64_t i = 0; i < ir.r; i++) assert_bit(&e, bl[ir.root[i]]);

  for (int64_t i = 0; i < ir.n; i++) {
    int64_t op = ir.node[4 * i];
    free(wd[i].b);
    if ((op == OP_UDIV || op == OP_UREM)) {
      /* q/r arrays are shared between twins: free only at the first owner */
      int64_t x = ir.node[4 * i + 1], y = ir.node[4 * i + 2];
      int owner = 1;
      for (int64_t j = 0; j < i; j++) {
        int64_t oj = ir.node[4 * j];
        if ((oj == OP_UDIV || oj == OP_UREM) && ir.node[4 * j + 1] == x &&
            ir.node[4 * j + 2] == y) { owner = 0; break; }
      }
      if (owner) { free(q_of[i].b); free(r_of[i].b); }
    }
  }
  free(wd); free(bl); free(q_of); free(r_of);
  if (e.failed) {
    enc_free(&e);
    free(out->free_width); free(out->in_map); free(out);
    return NULL;
  }
  out->nvars = e.nvars;
  out->ncl = e.ncl;
  out->nl = e.nl;
  out->cb = e.cb;
  out->lits = e.lits;
  return out;
}

int64_t oracle_cnf_info(const ocnf_t *c, int64_t *out4) {
  out4[0] = c->nvars; out4[1] = c->ncl; out4[2] = c->nl; out4[3] = c->n_free;
  int64_t bits = 0;
  for (int i = 0; i < c->n_free; i++) bits += c->free_width[i];
  return bits;
}

void oracle_cnf_copy(const ocnf_t *c, int64_t *cb, int32_t *lits, int32_t *in_map,
                     int32_t *free_width) {
  memcpy(cb, c->cb, sizeof(int64_t) * (c->ncl + 1));
  memcpy(lits, c->lits, sizeof(int32_t) * c->nl);
  int64_t bits = 0;
  for (int i = 0; i < c->n_free; i++) bits += c->free_width[i];
  memcpy(in_map, c->in_map, sizeof(int32_t) * bits);
  memcpy(free_width, c->free_width, sizeof(int32_t) * c->n_free);
}

void oracle_cnf_free(ocnf_t *c) {
  if (!c) return;
  free(c->cb); free(c->lits); free(c->free_width); free(c->in_map); free(c);
}

/* ------------------------------------------------------------------------ */
/* 3. DPLL                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t decisions, conflicts, propagations;
} dstats_t;

typedef struct {
  int32_t *buf;
  int64_t cap, len;
  int overflow;
} trace_t;

static void trace_clause(trace_t *t, const int *dec_lits, int nd) {
  if (!t) return;
  if (t->len + nd + 1 > t->cap) { t->overflow = 1; return; }
  /* clause = NOT(d1 & ... & dk) = (-d1 | ... | -dk) */
  for (int i = 0; i < nd; i++) t->buf[t->len++] = -dec_lits[i];
  t->buf[t->len++] = 0;
}

/* value of DIMACS literal l under val[] (1 true, 0 false, -1 unassigned) */
static inline int lval(const int8_t *val, int l) {
  int v = val[l > 0 ? l : -l];
  if (v < 0) return -1;
  return l > 0 ? v : 1 - v;
}

static inline int lcode(int l) { return 2 * ((l > 0 ? l : -l) - 1) + (l < 0); }

int oracle_dpll(int nv, int64_t nc, const int64_t *cb, const int32_t *lits,
                int64_t budget, uint8_t *model, int64_t *stats3, int32_t *trace_buf,
                int64_t trace_cap, int64_t *trace_len) {
  dstats_t st = {0, 0, 0};
  trace_t tr = {trace_buf, trace_cap, 0, 0};
  trace_t *T = trace_buf ? &tr : NULL;
  int verdict = V_UNKNOWN;

  /* occurrence lists per literal code */
  int64_t nlc = 2 * (int64_t)nv;
  int64_t *ob = (int64_t *)calloc((size_t)nlc + 1, sizeof(int64_t));
  int64_t nlit = cb[nc];
  int64_t *occ = (int64_t *)malloc(sizeof(int64_t) * (nlit ? nlit : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nlc ? nlc : 1));
  int8_t *val = (int8_t *)malloc((size_t)nv + 1);
  int *trail = (int *)malloc(sizeof(int) * ((size_t)nv + 1));
  int *dpos = (int *)malloc(sizeof(int) * ((size_t)nv + 1));
  uint8_t *dflip = (uint8_t *)malloc((size_t)nv + 1);
  int *dlits = (int *)malloc(sizeof(int) * ((size_t)nv + 1));
  double *act = (double *)calloc((size_t)nv + 1, sizeof(double));
  if (!ob || !occ || !fill || !val || !trail || !dpos || !dflip || !dlits || !act) {
    verdict = V_ERROR;
    goto done;
  }
  for (int64_t i = 0; i < nlit; i++) {
    int l = lits[i];
    if (l == 0 || (l > 0 ? l : -l) > nv) { verdict = V_ERROR; goto done; }
    ob[lcode(l) + 1]++;
  }
  for (int64_t i = 0; i < nlc; i++) ob[i + 1] += ob[i];
  for (int64_t i = 0; i < nlc; i++) fill[i] = ob[i];
  for (int64_t c = 0; c < nc; c++)
    for (int64_t k = cb[c]; k < cb[c + 1]; k++) occ[fill[lcode(lits[k])]++] = c;

  for (int v = 0; v <= nv; v++) val[v] = -1;
  int tlen = 0, qhead = 0, nd = 0;
  double inc = 1.0;

  /* level 0: empty clauses and unit clauses */
  for (int64_t c = 0; c < nc; c++) {
    int64_t len = cb[c + 1] - cb[c];
    if (len == 0) { trace_clause(T, dlits, 0); verdict = V_UNSAT; goto done; }
  }
  for (int64_t c = 0; c < nc; c++) {
    if (cb[c + 1] - cb[c] != 1) continue;
    int l = lits[cb[c]];
    int lv = lval(val, l);
    if (lv == 0) { trace_clause(T, dlits, 0); verdict = V_UNSAT; goto done; }
    if (lv < 0) { val[l > 0 ? l : -l] = l > 0; trail[tlen++] = l; }
  }

  for (;;) {
    /* unit propagation to a fixpoint over occurrence lists */
    int64_t confl = -1;
    while (qhead < tlen && confl < 0) {
      int p = trail[qhead++];
      st.propagations++;
      int f = -p; /* literal that just became false */
      int64_t fc = lcode(f);
      for (int64_t k = ob[fc]; k < ob[fc + 1] && confl < 0; k++) {
        int64_t c = occ[k];
        int sat = 0, nun = 0, unit = 0;
        for (int64_t q = cb[c]; q < cb[c + 1]; q++) {
          int l = lits[q];
          int lv = lval(val, l);
          if (lv == 1) { sat = 1; break; }
          if (lv < 0 && l != unit) { nun++; unit = l; }
        }
        if (sat) continue;
        if (nun == 0) { confl = c; break; }
        if (nun == 1) {
          int v = unit > 0 ? unit : -unit;
          val[v] = unit > 0;
          trail[tlen++] = unit;
        }
      }
    }
    if (confl >= 0) {
      st.conflicts++;
      for (int64_t q = cb[confl]; q < cb[confl + 1]; q++) {
        int v = lits[q] > 0 ? lits[q] : -lits[q];
        act[v] += inc;
      }
      inc /= 0.95;
      int big = inc > 1e20;
      for (int64_t q = cb[confl]; q < cb[confl + 1]; q++) {
        int v = lits[q] > 0 ? lits[q] : -lits[q];
        if (act[v] > 1e20) big = 1;
      }
      if (big) {
        for (int v = 1; v <= nv; v++) act[v] *= 1e-20;
        inc *= 1e-20;
      }
      /* refuted under the current decisions */
      for (int i = 0; i < nd; i++) dlits[i] = trail[dpos[i]];
      trace_clause(T, dlits, nd);
      while (nd > 0 && dflip[nd - 1]) {
        nd--;
        trace_clause(T, dlits, nd);
      }
      if (nd == 0) { verdict = V_UNSAT; goto done; }
      int pos = dpos[nd - 1];
      int d = trail[pos];
      for (int t = tlen - 1; t >= pos; t--) {
        int l = trail[t];
        val[l > 0 ? l : -l] = -1;
      }
      tlen = pos;
      dflip[nd - 1] = 1;
      val[d > 0 ? d : -d] = d < 0; /* assign -d */
      trail[tlen++] = -d;
      qhead = pos;
      continue;
    }
    if (tlen == nv) { verdict = V_SAT; break; }
    if (st.decisions >= budget) { verdict = V_UNKNOWN; break; }
    int best = 0;
    double ba = -1.0;
    for (int v = 1; v <= nv; v++)
      if (val[v] < 0 && act[v] > ba) { ba = act[v]; best = v; }
    st.decisions++;
    dpos[nd] = tlen;
    dflip[nd] = 0;
    nd++;
    val[best] = 0;
    trail[tlen++] = -best;
  }
  if (verdict == V_SAT && model)
    for (int v = 1; v <= nv; v++) model[v - 1] = (uint8_t)val[v];
done:
  if (stats3) { stats3[0] = st.decisions; stats3[1] = st.conflicts; stats3[2] = st.propagations; }
  if (trace_len) *trace_len = tr.overflow ? -1 : tr.len;
  free(ob); free(occ); free(fill); free(val); free(trail); free(dpos); free(dflip);
  free(dlits); free(act);
  return verdict;
}

/* ------------------------------------------------------------------------ */
/* 4. Brute force over every input assignment (the plain definition)        */
/* ------------------------------------------------------------------------ */

typedef unsigned __int128 u128;

/* Evaluates the IR on one assignment of the FREE words. Returns 1 if every
   root holds, 0 if not, -1 if an intermediate value overflowed 128 bits. */
static int eval_ir(const ir_t *ir, const uint64_t *inputs, u128 *wv, uint8_t *bv) {
  int fi = 0;
  for (int64_t i = 0; i < ir->n; i++) {
    int64_t op = ir->node[4 * i], x = ir->node[4 * i + 1], y = ir->node[4 * i + 2];
    switch (op) {
      case OP_FREE: wv[i] = inputs[fi++]; break;
      case OP_CONST: wv[i] = (u128)(uint64_t)x; break;
      case OP_ADD:
        wv[i] = wv[x] + wv[y];
        if (wv[i] < wv[x]) return -1;
        break;
      case OP_MUL:
        if (wv[x] != 0 && wv[y] > ((~(u128)0) / wv[x])) return -1;
        wv[i] = wv[x] * wv[y];
        break;
      case OP_UDIV: wv[i] = wv[x] / wv[y]; break;
      case OP_UREM: wv[i] = wv[x] % wv[y]; break;
      case OP_TRUNC:
      case OP_NOTW: {
        u128 m = (((u128)1) << y) - 1; /* y <= 64 */
        wv[i] = op == OP_TRUNC ? (wv[x] & m) : (m - (wv[x] & m));
        break;
      }
      case OP_ULT: bv[i] = wv[x] < wv[y]; break;
      case OP_ULE: bv[i] = wv[x] <= wv[y]; break;
      case OP_EQ: bv[i] = wv[x] == wv[y]; break;
      case OP_OR: bv[i] = bv[x] | bv[y]; break;
      case OP_AND: bv[i] = bv[x] & bv[y]; break;
      case OP_NOT: bv[i] = !bv[x]; break;
    }
  }
  for (int64_t i = 0; i < ir->r; i++)
    if (!bv[ir->root[i]]) return 0;
  return 1;
}

/* Returns V_SAT (witness written), V_UNSAT, or V_ERROR (too many points or
   overflow). max_bits bounds the total number of input bits enumerated. */
int oracle_brute_force(const int64_t *a, int64_t len, int max_bits, uint64_t *witness) {
  ir_t ir;
  if (ir_open(a, len, &ir)) return V_ERROR;
  int nf = 0, bits = 0;
  int widths[64];
  for (int64_t i = 0; i < ir.n; i++)
    if (ir.node[4 * i] == OP_FREE) {
      if (nf >= 64) return V_ERROR;
      widths[nf] = (int)ir.node[4 * i + 1];
      bits += widths[nf];
      nf++;
    }
  if (bits > max_bits || bits > 40) return V_ERROR;
  u128 *wv = (u128 *)calloc((size_t)(ir.n ? ir.n : 1), sizeof(u128));
  uint8_t *bv = (uint8_t *)calloc((size_t)(ir.n ? ir.n : 1), 1);
  uint64_t in[64];
  int verdict = V_UNSAT;
  uint64_t total = 1ULL << bits;
  for (uint64_t code = 0; code < total; code++) {
    uint64_t rest = code;
    for (int f = 0; f < nf; f++) {
      in[f] = rest & ((1ULL << widths[f]) - 1);
      rest >>= widths[f];
    }
    int r = eval_ir(&ir, in, wv, bv);
    if (r < 0) { verdict = V_ERROR; break; }
    if (r == 1) {
      verdict = V_SAT;
      if (witness) memcpy(witness, in, sizeof(uint64_t) * nf);
      break;
    }
  }
  free(wv);
  free(bv);
  return verdict;
}

/* ------------------------------------------------------------------------ */
/* 5. Batch solving with a pthread pool                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  /* query mode (irs != NULL) or CNF mode */
  const int64_t *irs, *ir_off;
  int nvars_fixed;
  const int32_t *cnf_nv;
  const int64_t *cnf_cb_off, *cnf_cb, *cnf_lit_off;
  const int32_t *cnf_lits;
  int n;
  int64_t budget;
  uint8_t *verdict;
  int64_t *stats;      /* n x 3 */
  uint64_t *words;     /* query mode: per query, up to words_stride input words */
  int words_stride;
  int64_t *cnf_size;   /* query mode: n x 2 (vars, clauses) */
  int algo;            /* 0 DPLL, 1 CDCL (cdcl.c; the budget then counts conflicts) */
  int next;
  pthread_mutex_t mu;
} batch_t;

int oracle_cdcl(int nv, int64_t nc, const int64_t *cb, const int32_t *lits,
                int64_t budget, uint8_t *model, int64_t *stats3, int32_t *trace_buf,
                int64_t trace_cap, int64_t *trace_len);

static int solve_cnf(const batch_t *b, int nv, int64_t nc, const int64_t *cb,
                     const int32_t *lits, uint8_t *model, int64_t *st) {
  if (b->algo == 1) return oracle_cdcl(nv, nc, cb, lits, b->budget, model, st, NULL, 0, NULL);
  return oracle_dpll(nv, nc, cb, lits, b->budget, model, st, NULL, 0, NULL);
}

static void solve_one(batch_t *b, int i) {
  int64_t st[3] = {0, 0, 0};
  if (b->irs) {
    const int64_t *a = b->irs + b->ir_off[i];
    int64_t len = b->ir_off[i + 1] - b->ir_off[i];
    ocnf_t *c = oracle_encode(a, len);
    if (!c) { b->verdict[i] = V_ERROR; return; }
    uint8_t *model = (uint8_t *)malloc((size_t)c->nvars + 1);
    int v = solve_cnf(b, c->nvars, c->ncl, c->cb, c->lits, model, st);
    b->verdict[i] = (uint8_t)v;
    if (b->cnf_size) { b->cnf_size[2 * i] = c->nvars; b->cnf_size[2 * i + 1] = c->ncl; }
    if (v == V_SAT && b->words) {
      int off = 0;
      for (int f = 0; f < c->n_free && f < b->words_stride; f++) {
        uint64_t word = 0;
        for (int k = 0; k < c->free_width[f]; k++) {
          int lit = c->in_map[off + k];
          int bit = lit > 0 ? model[lit - 1] : 1 - model[-lit - 1];
          word |= (uint64_t)bit << k;
        }
        b->words[(int64_t)i * b->words_stride + f] = word;
        off += c->free_width[f];
      }
    }
    free(model);
    oracle_cnf_free(c);
  } else {
    int nv = b->cnf_nv[i];
    const int64_t *cb = b->cnf_cb + b->cnf_cb_off[i];
    int64_t nc = b->cnf_cb_off[i + 1] - b->cnf_cb_off[i] - 1;
    const int32_t *lits = b->cnf_lits + b->cnf_lit_off[i];
    b->verdict[i] = (uint8_t)solve_cnf(b, nv, nc, cb, lits, NULL, st);
  }
  if (b->stats) { b->stats[3 * i] = st[0]; b->stats[3 * i + 1] = st[1]; b->stats[3 * i + 2] = st[2]; }
}

static void *worker(void *arg) {
  batch_t *b = (batch_t *)arg;
  for (;;) {
    pthread_mutex_lock(&b->mu);
    int i = b->next++;
    pthread_mutex_unlock(&b->mu);
    if (i >= b->n) break;
    solve_one(b, i);
  }
  return NULL;
}

static void run_pool(batch_t *b, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  pthread_t th[512];
  pthread_mutex_init(&b->mu, NULL);
  b->next = 0;
  for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, worker, b);
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&b->mu);
}

/* Encode + solve n queries. words: n x words_stride input words of each SAT
   model (may be NULL). cnf_size: n x 2 (may be NULL). algo: 0 DPLL, 1 CDCL. */
void oracle_solve_queries(int n, const int64_t *irs, const int64_t *ir_off, int nthreads,
                          int64_t budget, uint8_t *verdict, int64_t *stats,
                          uint64_t *words, int words_stride, int64_t *cnf_size, int algo) {
  batch_t b;
  memset(&b, 0, sizeof(b));
  b.algo = algo;
  b.irs = irs; b.ir_off = ir_off; b.n = n; b.budget = budget; b.verdict = verdict;
  b.stats = stats; b.words = words; b.words_stride = words_stride; b.cnf_size = cnf_size;
  run_pool(&b, nthreads);
}

/* Solve n CNFs. cb_off[n+1] indexes cb (each instance has nc+1 entries,
   relative to its own lits); lit_off[n] indexes lits. */
void oracle_solve_cnfs(int n, const int32_t *nv, const int64_t *cb_off, const int64_t *cb,
                       const int64_t *lit_off, const int32_t *lits, int nthreads,
                       int64_t budget, uint8_t *verdict, int64_t *stats, int algo) {
  batch_t b;
  memset(&b, 0, sizeof(b));
  b.algo = algo;
  b.cnf_nv = nv; b.cnf_cb_off = cb_off; b.cnf_cb = cb; b.cnf_lit_off = lit_off;
  b.cnf_lits = lits; b.n = n; b.budget = budget; b.verdict = verdict; b.stats = stats;
  run_pool(&b, nthreads);
}
