"""The front end on the GPU: the worked examples written as programs and the
two query families written as programs, decided through analyze_programs
(one batch, through the C ABI), verdicts against the cited expectations and
the closed forms, every witness satisfying its query."""
import os

import pytest

torch = pytest.importorskip("torch")

from closed_forms import bounds_algebra, bounds_wrap, partition_algebra, partition_wrap
from ir_eval import evaluate
from test_frontend import PROGRAMS, bounds_program, partition_program
from workloads import queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frontend():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_21552_gb300 import build
    build.build()
    from paper_2601_21552_gb300 import frontend as F
    return F


@pytest.mark.parametrize("search", ["dpll", "cdcl"])
def test_worked_examples_as_programs(frontend, search):
    texts = [open(p).read() for p in PROGRAMS]
    reports = frontend.analyze_programs(texts, search=search, time_budget_ms=60000)
    for path, rep in zip(PROGRAMS, reports):
        for a in rep.accesses:
            assert a.verdict == (1 if a.meta["expect"] == "SAT" else 0), (path, a.line)
            if a.verdict == 1:
                assert evaluate(a.ir, [a.witness[k] for k in a.inputs]), (path, a.line)
    uaf = [(os.path.basename(p), u.what, u.name) for p, r in zip(PROGRAMS, reports)
           for u in r.uaf]
    assert sorted(uaf) == [("uaf_host_and_kernel.kp", "access", "p"),
                           ("uaf_host_and_kernel.kp", "launch", "a")]


def test_families_as_programs(frontend):
    bp = [queries.config1_params(8400 + i, w=8) for i in range(64)]
    pp = [queries.config2_params(8500 + i, w=8) for i in range(64)]
    texts = [bounds_program(**p) for p in bp] + [partition_program(**p) for p in pp]
    reports = frontend.analyze_programs(texts, bid_width=8, search="cdcl")
    got = [r.accesses[0].verdict for r in reports]
    want = [int(bounds_algebra(**p)) for p in bp] + [int(partition_algebra(**p)) for p in pp]
    assert got == want


@pytest.mark.parametrize("search", ["dpll", "cdcl"])
def test_incremental_form(frontend, search):
    """One query per kernel, one unit per memory instruction (scuba_solve_units):
    the same verdicts as the per-access queries, models verified by the host."""
    from test_frontend import stencil_program
    texts = [open(p).read() for p in PROGRAMS] + [stencil_program(), stencil_program(w=10, radius=5)]
    inc = frontend.analyze_incremental(texts, search=search, time_budget_ms=60000)
    per = frontend.analyze_programs(texts, search=search, time_budget_ms=60000)
    for ri, rp in zip(inc, per):
        assert [a.verdict for a in ri.accesses] == [a.verdict for a in rp.accesses]
        assert [(u.what, u.name) for u in ri.uaf] == [(u.what, u.name) for u in rp.uaf]
        for a in ri.accesses:
            assert (a.witness is not None) == (a.verdict == 1)
    flat = [a.verdict for r in inc for a in r.accesses]
    assert 0 in flat and 1 in flat


@pytest.mark.parametrize("search", ["dpll", "cdcl"])
def test_wrap_families_as_programs(frontend, search):
    """The C wrap-around variant on the GPU: the two families under 'wrap W'
    against brute force with explicit modulo-2^W arithmetic (5-bit inputs)
    and against the oracle (8-bit inputs, W = 9 and 10)."""
    import oracle
    texts, want = [], []
    for d in (1, 2):
        for i in range(16):
            p = queries.config1_params(8600 + i, w=5)
            texts.append(f"wrap {5 + d}\n" + bounds_program(**p))
            want.append(int(bounds_wrap(**p, W=5 + d)))
            q = queries.config2_params(8700 + i, w=5)
            texts.append(f"wrap {5 + d}\n" + partition_program(**q))
            want.append(int(partition_wrap(**q, W=5 + d)))
    reports = frontend.analyze_programs(texts, bid_width=5, search=search)
    assert [r.accesses[0].verdict for r in reports] == want
    assert set(want) == {0, 1}
    t8 = []
    for d in (1, 2):
        t8 += [f"wrap {8 + d}\n" + bounds_program(**queries.config1_params(8800 + i, w=8))
               for i in range(32)]
        t8 += [f"wrap {8 + d}\n" + partition_program(**queries.config2_params(8900 + i, w=8))
               for i in range(32)]
    r8 = frontend.analyze_programs(t8, bid_width=8, search=search)
    irs = [frontend.queries(frontend.parse(t), bid_width=8)[0].ir for t in t8]
    ref = oracle.solve_queries(irs, max_words=16)["verdict"]
    assert [r.accesses[0].verdict for r in r8] == [int(v) for v in ref]
    for r in r8:
        a = r.accesses[0]
        if a.verdict == 1:
            assert evaluate(a.ir, [a.witness[k] for k in a.inputs])
