"""Pins of the oracle's clause-learning solver (oracle/cdcl.c), none of them
the solver itself: brute force over every assignment, the RUP check of its
learned clauses (rup.c, written separately), model checks, the closed forms
of both query families, the paper's worked examples -- and planted mistakes
in text copies of cdcl.c that those pins must catch."""
import ctypes
import glob
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from closed_forms import bounds_algebra, partition_algebra
from ir_eval import cnf_satisfied, evaluate
from workloads import queries
from workloads.ir import parse_text

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
ODIR = os.path.join(ROOT, "oracle")


def _cnf_from_3sat(nv, lits):
    return oracle.CNF(nv, np.arange(0, 3 * len(lits) + 1, 3), lits.reshape(-1))


def _bf_3sat(nv, lits):
    a = np.arange(1 << nv, dtype=np.uint32)
    ok = np.ones(1 << nv, dtype=bool)
    for cl in lits:
        sat = np.zeros(1 << nv, dtype=bool)
        for l in cl:
            bit = (a >> (abs(int(l)) - 1)) & 1
            sat |= (bit == 1) if l > 0 else (bit == 0)
        ok &= sat
    return bool(ok.any())


def test_random_3sat_bruteforce_and_rup():
    seen = set()
    for s in range(80):
        nv, lits = queries.random_3sat(5100 + s, 10, 14)
        cnf = _cnf_from_3sat(nv, lits)
        res = oracle.cdcl(cnf, want_trace=True)
        want = _bf_3sat(nv, lits)
        assert res["verdict"] == (oracle.SAT if want else oracle.UNSAT)
        if want:
            assert cnf_satisfied(cnf.clause_begin, cnf.lits, res["model"])
        else:
            assert oracle.rup_check(cnf, res["trace"]) == 1
        seen.add(want)
    assert seen == {True, False}


def test_rup_refutations_larger_3sat():
    """Past brute force: every learned clause is RUP, the last one empty."""
    n_unsat = 0
    for s in range(30):
        nv, lits = queries.random_3sat(5300 + s, 50, 70, ratio=5.0)
        cnf = _cnf_from_3sat(nv, lits)
        res = oracle.cdcl(cnf, want_trace=True)
        assert res["verdict"] == oracle.dpll(cnf)["verdict"]
        if res["verdict"] == oracle.UNSAT:
            n_unsat += 1
            t = res["trace"]
            assert t[-1] == 0 and (len(t) == 1 or t[-2] == 0)   # ends with the empty clause
            assert oracle.rup_check(cnf, t) == 1
            assert res["conflicts"] > 0
        else:
            assert cnf_satisfied(cnf.clause_begin, cnf.lits, res["model"])
    assert n_unsat >= 10


def test_closed_forms():
    b_params = [queries.config1_params(6100 + i, w=8) for i in range(128)]
    irs = [queries.bounds_query(**q).to_array() for q in b_params]
    v = oracle.solve_queries(irs, algo="cdcl")["verdict"]
    assert [int(x) for x in v] == [int(bounds_algebra(**q)) for q in b_params]
    p_params = [queries.config2_params(6200 + i, w=10) for i in range(128)]
    irs = [queries.partition_query(**q).to_array() for q in p_params]
    r = oracle.solve_queries(irs, algo="cdcl", max_words=8)
    assert [int(x) for x in r["verdict"]] == [int(partition_algebra(**q)) for q in p_params]
    # SAT models decode to inputs that satisfy the integer constraints
    for i in np.flatnonzero(r["verdict"] == oracle.SAT)[:20]:
        nfree = int((irs[i][4:4 + 4 * irs[i][2]].reshape(-1, 4)[:, 0] == 1).sum())
        assert evaluate(irs[i], [int(x) for x in r["words"][i][:nfree]])


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.sq"))),
                         ids=os.path.basename)
def test_worked_examples(path):
    ir, meta = parse_text(open(path).read())
    cnf = oracle.encode(ir.to_array())
    res = oracle.cdcl(cnf, want_trace=True, trace_cap=1 << 26)
    assert res["verdict"] == (oracle.SAT if meta["expect"] == "SAT" else oracle.UNSAT)
    if res["verdict"] == oracle.SAT:
        assert cnf_satisfied(cnf.clause_begin, cnf.lits, res["model"])
    elif cnf.nclauses * max(res["conflicts"], 1) < 5e7:
        assert oracle.rup_check(cnf, res["trace"]) == 1


def test_degenerate_and_budget():
    assert oracle.cdcl(oracle.CNF(3, [0], []))["verdict"] == oracle.SAT
    assert oracle.cdcl(oracle.CNF(2, [0, 1, 1], [1]))["verdict"] == oracle.UNSAT
    assert oracle.cdcl(oracle.CNF(1, [0, 1, 2], [1, -1]))["verdict"] == oracle.UNSAT
    r = oracle.cdcl(oracle.CNF(2, [0, 3, 4], [1, 1, 2, -2]))
    assert r["verdict"] == oracle.SAT and r["model"].tolist() == [1, 0]
    taut = oracle.CNF(2, [0, 2, 5], [1, -1, 2, -2, 1])
    assert oracle.cdcl(taut)["verdict"] == oracle.SAT
    nv, lits = queries.random_3sat(4242, 150, 150)
    r = oracle.cdcl(_cnf_from_3sat(nv, lits), budget=5)
    assert r["verdict"] == oracle.UNKNOWN and r["conflicts"] == 5


# ---------------------------------------------------------------------------
# Planted mistakes
# ---------------------------------------------------------------------------

MUTANTS = {
    "asserts_the_uip_itself": (
        "s->learnt[0] = -p;",
        "s->learnt[0] = p;"),
    "learned_clause_drops_a_literal": (
        "int n = analyze(&s, confl, &blev);",
        "int n = analyze(&s, confl, &blev); if (n > 2) n--;"),
    "moved_watch_not_registered": (
        "if (ivec_push(&s->watch[wi(C[1])], c)) return -2;",
        "(void)0;"),
    "unit_assigned_with_wrong_sign": (
        "assign(s, C[0], c);",
        "assign(s, -C[0], c);"),
    "level_zero_conflict_ignored": (
        "if (s.nlev == 0) { trace_add(&s, tmp, 0); verdict = K_UNSAT; break; }",
        "if (s.nlev == 0) { continue; }"),
}


def _build(cdcl_src: str, tag: str) -> ctypes.CDLL:
    d = tempfile.mkdtemp(prefix=f"cdcl_{tag}_")
    c = os.path.join(d, "cdcl.c")
    with open(c, "w") as f:
        f.write(cdcl_src)
    so = os.path.join(d, "lib.so")
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-w",
                           "-o", so, c, os.path.join(ODIR, "rup.c"), "-lm"])
    L = ctypes.CDLL(so)
    P = ctypes.c_void_p
    L.oracle_cdcl.restype = ctypes.c_int
    L.oracle_cdcl.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, ctypes.c_int64, P, P, P,
                              ctypes.c_int64, P]
    L.rup_check.restype = ctypes.c_int
    L.rup_check.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, ctypes.c_int64, P]
    return L


def _pins_failed(L) -> int:
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    fails = 0
    for s in range(40):
        nv, lits = queries.random_3sat(5500 + s, 10, 14)
        cnf = _cnf_from_3sat(nv, lits)
        model = np.zeros(nv, np.uint8)
        st = np.zeros(3, np.int64)
        tl = np.zeros(1, np.int64)
        tbuf = np.zeros(1 << 20, np.int32)
        v = L.oracle_cdcl(nv, cnf.nclauses, p(cnf.clause_begin), p(cnf.lits), 20000, p(model),
                          p(st), p(tbuf), len(tbuf), p(tl))
        want = _bf_3sat(nv, lits)
        if v != (oracle.SAT if want else oracle.UNSAT):
            fails += 1
        elif want and not cnf_satisfied(cnf.clause_begin, cnf.lits, model):
            fails += 1
        elif not want and (tl[0] < 0 or L.rup_check(nv, cnf.nclauses, p(cnf.clause_begin),
                                                     p(cnf.lits), int(tl[0]), p(tbuf)) != 1):
            fails += 1
    return fails


def test_unmodified_cdcl_passes_the_pins():
    assert _pins_failed(_build(open(os.path.join(ODIR, "cdcl.c")).read(), "orig")) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_cdcl_mistake_is_caught(name):
    old, new = MUTANTS[name]
    src = open(os.path.join(ODIR, "cdcl.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    assert _pins_failed(_build(src.replace(old, new), name)) > 0, f"pins missed {name}"
