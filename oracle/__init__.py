"""CPU oracle for the out-of-bounds satisfiability check.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` leg (and its ``--impl reference`` arm) may import
this package. It shares no code with the product library and does not import
it. Everything here is plain and slow on purpose.

What each function follows in the paper:

* ``encode`` -- Sec. V-B: the three kinds of constraints over solver
  variables, bit-blasted to CNF with plain Tseitin gates (oracle.c).
* ``dpll`` / ``solve_queries`` / ``solve_cnfs`` -- Sec. V-B, step (10): decide
  whether all constraints are simultaneously satisfiable; a plain complete
  DPLL (unit propagation, activity decisions, chronological backtracking).
* ``brute_force`` -- the definition itself (Sec. IV-A: "under any possible
  input"): enumerate every input and evaluate the constraints exactly.
* ``cdcl`` -- the same decision by plain conflict-driven clause learning
  (first-UIP clauses, backjumping, restarts; cdcl.c). The paper's solver
  learns internally without further detail; this is the textbook loop.
* ``rup_check`` -- independent checker for the refutation traces of both.

Parity status: encode+dpll are pinned by brute force (widths <= 6), by
closed forms (bounds and partition families at 8 and 16 bits), by the
paper's worked examples (tests/golden), by model re-verification and by the
RUP checker; cdcl by the RUP check of its learned clauses, model checks,
brute force and the same corpora. No function here is unpinned.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build as _build

UNSAT, SAT, UNKNOWN, ERROR = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        L.oracle_encode.restype = P
        L.oracle_encode.argtypes = [P, i64]
        L.oracle_cnf_info.restype = i64
        L.oracle_cnf_info.argtypes = [P, P]
        L.oracle_cnf_copy.restype = None
        L.oracle_cnf_copy.argtypes = [P, P, P, P, P]
        L.oracle_cnf_free.restype = None
        L.oracle_cnf_free.argtypes = [P]
        L.oracle_dpll.restype = i32
        L.oracle_dpll.argtypes = [i32, i64, P, P, i64, P, P, P, i64, P]
        L.oracle_brute_force.restype = i32
        L.oracle_brute_force.argtypes = [P, i64, i32, P]
        L.oracle_solve_queries.restype = None
        L.oracle_solve_queries.argtypes = [i32, P, P, i32, i64, P, P, P, i32, P, i32]
        L.oracle_solve_cnfs.restype = None
        L.oracle_solve_cnfs.argtypes = [i32, P, P, P, P, P, i32, i64, P, P, i32]
        L.oracle_cdcl.restype = i32
        L.oracle_cdcl.argtypes = [i32, i64, P, P, i64, P, P, P, i64, P]
        L.rup_check.restype = i32
        L.rup_check.argtypes = [i32, i64, P, P, i64, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class CNF:
    """A CNF in DIMACS numbering: clause_begin[nc+1] (int64), lits (int32)."""

    def __init__(self, nvars, clause_begin, lits, in_map=None, free_width=None):
        self.nvars = int(nvars)
        self.clause_begin = np.ascontiguousarray(clause_begin, dtype=np.int64)
        self.lits = np.ascontiguousarray(lits, dtype=np.int32)
        self.in_map = in_map
        self.free_width = free_width

    @property
    def nclauses(self) -> int:
        return len(self.clause_begin) - 1

    def clauses(self):
        cb, L = self.clause_begin, self.lits
        return [L[cb[i]:cb[i + 1]].tolist() for i in range(self.nclauses)]


def encode(ir_array: np.ndarray) -> CNF:
    a = np.ascontiguousarray(ir_array, dtype=np.int64)
    h = lib().oracle_encode(_p(a), len(a))
    if not h:
        raise ValueError("oracle: malformed IR")
    try:
        info = np.zeros(4, dtype=np.int64)
        bits = lib().oracle_cnf_info(h, _p(info))
        nv, nc, nl, nf = (int(x) for x in info)
        cb = np.zeros(nc + 1, dtype=np.int64)
        lits = np.zeros(max(nl, 1), dtype=np.int32)
        in_map = np.zeros(max(bits, 1), dtype=np.int32)
        fw = np.zeros(max(nf, 1), dtype=np.int32)
        lib().oracle_cnf_copy(h, _p(cb), _p(lits), _p(in_map), _p(fw))
        return CNF(nv, cb, lits[:nl], in_map[:bits], fw[:nf])
    finally:
        lib().oracle_cnf_free(h)


def _solve_one(fn, cnf: CNF, budget: int, want_trace: bool, trace_cap: int):
    model = np.zeros(max(cnf.nvars, 1), dtype=np.uint8)
    stats = np.zeros(3, dtype=np.int64)
    tl = np.zeros(1, dtype=np.int64)
    tbuf = np.zeros(trace_cap if want_trace else 1, dtype=np.int32)
    v = fn(cnf.nvars, cnf.nclauses, _p(cnf.clause_begin), _p(cnf.lits), int(budget),
           _p(model), _p(stats), _p(tbuf) if want_trace else None,
           trace_cap if want_trace else 0, _p(tl))
    trace = None
    if want_trace:
        if tl[0] < 0:
            raise RuntimeError("oracle: trace buffer overflow")
        trace = tbuf[:tl[0]].copy()
    return dict(verdict=int(v), model=model[:cnf.nvars].copy(), decisions=int(stats[0]),
                conflicts=int(stats[1]), propagations=int(stats[2]), trace=trace)


def dpll(cnf: CNF, budget: int = 1 << 40, want_trace: bool = False, trace_cap: int = 1 << 24):
    """Solve one CNF by plain DPLL. Returns dict(verdict, model, decisions,
    conflicts, propagations, trace); the budget counts decisions and the trace
    holds NOT(decisions) of every refuted node, then the empty clause."""
    return _solve_one(lib().oracle_dpll, cnf, budget, want_trace, trace_cap)


def cdcl(cnf: CNF, budget: int = 1 << 40, want_trace: bool = False, trace_cap: int = 1 << 24):
    """Solve one CNF by plain CDCL (first-UIP learning, backjumping, restarts).
    Same result dict as dpll; the budget counts conflicts and the trace holds
    every learned clause, then the empty clause on UNSAT."""
    return _solve_one(lib().oracle_cdcl, cnf, budget, want_trace, trace_cap)


def rup_check(cnf: CNF, trace: np.ndarray) -> int:
    t = np.ascontiguousarray(trace, dtype=np.int32)
    return int(lib().rup_check(cnf.nvars, cnf.nclauses, _p(cnf.clause_begin), _p(cnf.lits),
                               len(t), _p(t)))


def brute_force(ir_array: np.ndarray, max_bits: int = 28):
    """Exhaustive check. Returns (verdict, witness words or None)."""
    a = np.ascontiguousarray(ir_array, dtype=np.int64)
    wit = np.zeros(64, dtype=np.uint64)
    v = int(lib().oracle_brute_force(_p(a), len(a), int(max_bits), _p(wit)))
    if v == ERROR:
        raise ValueError("brute force not applicable (too many input bits or overflow)")
    return v, (wit if v == SAT else None)


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1


ALGOS = {"dpll": 0, "cdcl": 1}


def solve_queries(irs: list[np.ndarray], threads: int | None = None, budget: int = 1 << 40,
                  max_words: int = 64, algo: str = "dpll"):
    """Encode and solve many queries on a thread pool (algo "dpll" or "cdcl";
    the budget counts decisions, resp. conflicts). Returns dict with
    verdict[n], stats[n,3] (decisions, conflicts, propagations), words[n,
    max_words] (input words of each SAT model, FREE-node order) and
    size[n,2] (vars, clauses of the oracle's own CNF)."""
    n = len(irs)
    offs = np.zeros(n + 1, dtype=np.int64)
    for i, a in enumerate(irs):
        offs[i + 1] = offs[i] + len(a)
    buf = np.ascontiguousarray(np.concatenate(irs) if n else np.zeros(1, np.int64), dtype=np.int64)
    verdict = np.zeros(max(n, 1), dtype=np.uint8)
    stats = np.zeros((max(n, 1), 3), dtype=np.int64)
    words = np.zeros((max(n, 1), max_words), dtype=np.uint64)
    size = np.zeros((max(n, 1), 2), dtype=np.int64)
    lib().oracle_solve_queries(n, _p(buf), _p(offs), int(threads or default_threads()),
                               int(budget), _p(verdict), _p(stats), _p(words), max_words,
                               _p(size), ALGOS[algo])
    return dict(verdict=verdict[:n], stats=stats[:n], words=words[:n], size=size[:n])


def solve_cnfs(cnfs: list[CNF], threads: int | None = None, budget: int = 1 << 40,
               algo: str = "dpll"):
    n = len(cnfs)
    nv = np.array([c.nvars for c in cnfs] or [0], dtype=np.int32)
    cb_off = np.zeros(n + 1, dtype=np.int64)
    lit_off = np.zeros(max(n, 1), dtype=np.int64)
    for i, c in enumerate(cnfs):
        cb_off[i + 1] = cb_off[i] + len(c.clause_begin)
        if i + 1 < n:
            lit_off[i + 1] = lit_off[i] + len(c.lits)
    cb = np.concatenate([c.clause_begin for c in cnfs]) if n else np.zeros(1, np.int64)
    lits = np.concatenate([c.lits for c in cnfs]) if n else np.zeros(1, np.int32)
    cb = np.ascontiguousarray(cb, dtype=np.int64)
    lits = np.ascontiguousarray(lits, dtype=np.int32)
    verdict = np.zeros(max(n, 1), dtype=np.uint8)
    stats = np.zeros((max(n, 1), 3), dtype=np.int64)
    lib().oracle_solve_cnfs(n, _p(nv), _p(cb_off), _p(cb), _p(lit_off), _p(lits),
                            int(threads or default_threads()), int(budget), _p(verdict),
                            _p(stats), ALGOS[algo])
    return dict(verdict=verdict[:n], stats=stats[:n])
