/*
 * rup.c -- independent reverse-unit-propagation (RUP) checker.
 *
 * TEST INFRASTRUCTURE ONLY. Pins the oracle's UNSAT verdicts where no closed
 * form or brute force applies: the oracle's DPLL emits, for every refuted
 * node of its search tree (in post-order), the clause NOT(d1 & ... & dk) over
 * that node's decision literals, ending with the empty clause. This checker
 * accepts a clause C iff asserting the negation of every literal of C and
 * running unit propagation over the original clauses plus the clauses
 * accepted so far reaches a conflict. The formula is UNSAT iff every clause
 * is accepted and the last one is empty.
 *
 * Written separately from oracle.c (no shared code). Propagation here is the
 * naive fixpoint: sweep every stored clause, assign the single open literal of
 * each unit clause, repeat until a sweep changes nothing or a clause is false.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { C_SAT, C_FALSE, C_UNIT, C_OPEN };

/* status of clause L[b..e) under val (1 true, 0 false, -1 open per var) */
static int clause_status(const int32_t *L, int64_t b, int64_t e, const int8_t *val, int *unit) {
  int open_lit = 0, n_open = 0;
  for (int64_t k = b; k < e; k++) {
    int l = L[k];
    int v = l > 0 ? l : -l;
    if (val[v] < 0) {
      if (n_open == 0 || l != open_lit) { n_open++; open_lit = l; }
      continue;
    }
    if ((l > 0) == (val[v] == 1)) return C_SAT;
  }
  if (n_open == 0) return C_FALSE;
  if (n_open == 1) { *unit = open_lit; return C_UNIT; }
  return C_OPEN;
}

/* Returns 1 = valid refutation, 0 = some clause is not RUP (or the last
   clause is not empty), -1 = malformed input / out of memory. */
int rup_check(int nv, int64_t nc, const int64_t *cb, const int32_t *lits,
              int64_t tlen, const int32_t *trace) {
  int64_t ntrace = 0;
  for (int64_t i = 0; i < tlen; i++) if (trace[i] == 0) ntrace++;
  if (ntrace == 0 || trace[tlen - 1] != 0) return 0;
  int64_t total = nc + ntrace;
  int64_t *beg = (int64_t *)malloc(sizeof(int64_t) * (total + 1));
  int64_t nl = cb[nc] + tlen;
  int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (nl ? nl : 1));
  int8_t *val = (int8_t *)malloc((size_t)nv + 1);
  int result = -1;
  if (!beg || !L || !val) goto out;

  int64_t m = 0, pos = 0;
  beg[0] = 0;
  for (int64_t c = 0; c < nc; c++) {
    for (int64_t k = cb[c]; k < cb[c + 1]; k++) {
      int l = lits[k];
      if (l == 0 || (l > 0 ? l : -l) > nv) goto out;
      L[pos++] = l;
    }
    beg[++m] = pos;
  }

  int last_empty = 0;
  int64_t t = 0;
  while (t < tlen) {
    int64_t s = t;
    while (trace[t] != 0) t++;
    int64_t e = t++; /* clause = trace[s..e) */

    for (int v = 0; v <= nv; v++) val[v] = -1;
    int conflict = 0;
    for (int64_t k = s; k < e; k++) {
      int l = trace[k];
      int v = l > 0 ? l : -l;
      if (l == 0 || v > nv) goto out;
      int8_t want = (int8_t)(l < 0); /* make l false */
      if (val[v] < 0) val[v] = want;
      else if (val[v] != want) conflict = 1; /* tautology: trivially implied */
    }
    while (!conflict) {
      int changed = 0;
      for (int64_t c = 0; c < m; c++) {
        int u = 0;
        int st = clause_status(L, beg[c], beg[c + 1], val, &u);
        if (st == C_FALSE) { conflict = 1; break; }
        if (st == C_UNIT) {
          val[u > 0 ? u : -u] = (int8_t)(u > 0);
          changed = 1;
        }
      }
      if (!changed) break;
    }
    if (!conflict) { result = 0; goto out; }
    for (int64_t k = s; k < e; k++) L[pos++] = trace[k];
    beg[++m] = pos;
    last_empty = (e == s);
  }
  result = last_empty ? 1 : 0;
out:
  free(beg); free(L); free(val);
  return result;
}
