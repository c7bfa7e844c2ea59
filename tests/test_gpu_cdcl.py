"""GPU parity of the clause-learning search (scuba_options.search = CDCL)
through the C ABI: verdicts bit-exact against the CPU oracles on the same
seeded inputs, every SAT model re-verified (integer constraints or clauses),
plus the paths that only this mode has -- a full learned-clause arena,
restarts after every conflict, the conflict budget -- and its option checks."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from closed_forms import bounds_algebra, partition_algebra
from raw_cnf import model_ok, solve_raw
from workloads import queries

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_21552_gb300 import build
    build.build()
    from paper_2601_21552_gb300 import api as A
    return A


def _check_queries(api, irs, **opts):
    res = api.solve_queries(irs, time_budget_ms=120000, search="cdcl", **opts)
    assert res["status"] == 0
    assert res["fails"] == 0, "a SAT model violates the original constraints"
    assert ((res["verdict"] == 1) == (res["verified"] == 1)).all()
    return res


def test_config1_full(api):
    irs, params = queries.config1(256)
    res = _check_queries(api, irs)
    want = np.array([1 if bounds_algebra(**p) else 0 for p in params], np.uint8)
    assert (res["verdict"] == want).all()
    assert (res["verdict"] == oracle.solve_queries(irs, algo="cdcl")["verdict"]).all()


def test_config2_full_size(api):
    """4,096 partition queries at 16 bits against the stored oracle verdicts
    (pinned by the closed form)."""
    stored = np.array([int(x) for x in open(os.path.join(
        GOLDEN, "config2_w16_oracle_verdicts.txt")).read().split()], np.uint8)
    irs, params = queries.config2(4096)
    res = _check_queries(api, irs)
    assert (res["verdict"] == stored).all()
    for i in range(0, 4096, 97):
        assert res["verdict"][i] == (1 if partition_algebra(**params[i]) else 0)


def _random_cnfs(seed0, count, lo, hi):
    out = []
    for s in range(count):
        n, l = queries.random_3sat(seed0 + s, lo, hi)
        out.append((n, l.tolist()))
    return out


def _oracle_verdicts(cnfs, algo="cdcl"):
    ocnfs = [oracle.CNF(n, np.cumsum([0] + [len(c) for c in cls]),
                        np.array([x for c in cls for x in c] or [1], np.int32)
                        [:sum(len(c) for c in cls)]) for n, cls in cnfs]
    return oracle.solve_cnfs(ocnfs, algo=algo)["verdict"]


@pytest.mark.parametrize("split", [True, False])
def test_random_3sat_vs_oracle(api, split):
    """With split, hard instances are shared as cubes among idle warps."""
    cnfs = _random_cnfs(71000, 400, 60, 200)
    st, v, m, vb, stats = solve_raw(api, cnfs, search="cdcl", split=split,
                                    time_budget_ms=180000)
    assert st == 0
    ref = _oracle_verdicts(cnfs)
    assert (v == ref).all()
    assert set(ref.tolist()) == {0, 1}
    for i, (n, c) in enumerate(cnfs):
        if v[i] == 1:
            assert model_ok(c, m, vb[i])
    assert (stats[:, 1] > 0).any() and (stats[:, 2] > 0).all()


def test_long_clauses_and_duplicates(api):
    rng = np.random.default_rng(5)
    cnfs = []
    for _ in range(300):
        n = int(rng.integers(8, 30))
        cls = []
        for _ in range(int(rng.integers(n, 5 * n))):
            k = int(rng.integers(1, 9))
            cls.append([int(rng.integers(1, n + 1)) * (1 if rng.random() < 0.5 else -1)
                        for _ in range(k)])
        cnfs.append((n, cls))
    st, v, m, vb, _ = solve_raw(api, cnfs, search="cdcl")
    assert st == 0
    assert (v == _oracle_verdicts(cnfs, algo="dpll")).all()
    for i, (n, cls) in enumerate(cnfs):
        if v[i] == 1:
            assert model_ok(cls, m, vb[i])


def test_degenerate_instances(api):
    cnfs = [
        (3, []),
        (2, [[1, 2], []]),
        (1, [[1], [-1]]),
        (2, [[1, 1, 2], [-2]]),
        (2, [[1, -1], [2, -2, 1]]),
        (0, []),
        (4, [[1, 2, 3, 4], [-1], [-2], [-3]]),
        (2, [[1, 2], [1, -2], [-1, 2], [-1, -2]]),  # UNSAT after one conflict at level 1
    ]
    st, v, m, vb, _ = solve_raw(api, cnfs, search="cdcl")
    assert st == 0
    assert v.tolist() == [1, 0, 0, 1, 1, 1, 1, 0]
    assert m[vb[3]] == 1 and m[vb[6] + 3] == 1


@pytest.mark.parametrize("learnt_words,restart_unit", [(0, 1), (4096, 0), (2048, 1)])
def test_arena_full_and_restarts(api, learnt_words, restart_unit):
    """A small arena (full and dropped every few dozen conflicts, the watch
    pool with it) and restarts after every Luby unit of one conflict: verdicts
    unchanged."""
    cnfs = _random_cnfs(72000, 120, 30, 70)
    st, v, m, vb, _ = solve_raw(api, cnfs, search="cdcl", learnt_words=learnt_words,
                                restart_unit=restart_unit)
    assert st == 0
    assert (v == _oracle_verdicts(cnfs)).all()
    for i, (n, c) in enumerate(cnfs):
        if v[i] == 1:
            assert model_ok(c, m, vb[i])


def test_conflict_budget_gives_unknown(api):
    n, l = queries.random_3sat(4243, 250, 250)
    st, v, m, vb, stats = solve_raw(api, [(n, l.tolist())], search="cdcl", decision_budget=5)
    assert st == 0 and v[0] == 2 and stats[0, 1] <= 6


def test_options_rejected(api):
    from paper_2601_21552_gb300 import binding as B
    cnfs = [(3, [[1, 2, 3]])]
    for bad in (dict(search="cdcl", heuristic=B.SCUBA_HEUR_LEARNED),
                dict(search="cdcl", learnt_words=40),  # below 64
                dict(search="cdcl", learnt_words=1 << 30),
                dict(search=7)):
        with pytest.raises(RuntimeError, match=f"status {B.SCUBA_ERR_ARG}"):
            solve_raw(api, cnfs, **bad)
    assert solve_raw(api, cnfs, search="cdcl")[1].tolist() == [1]


def test_bounds_w32(api):
    """The 32-bit bounds queries of the stress batch against the closed form."""
    irs, params = queries.config5_bounds(300)
    res = _check_queries(api, irs)
    want = np.array([1 if bounds_algebra(**p) else 0 for p in params], np.uint8)
    assert (res["verdict"] == want).all()
