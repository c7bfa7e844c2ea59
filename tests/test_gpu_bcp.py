"""BCP exactness and failure handling on the GPU.

The unit-propagation closure of a CNF under assumptions is unique, whatever
order the literals are propagated in, so the GPU closure (the search's own BCP
through scuba_propagate_batch) must equal a plain CPU closure exactly, and
report a conflict exactly when the CPU closure does.

Failure handling is tested without any fault: an abort flag raised before
the launch and a time budget that expires make the persistent kernel return a
status, with every unfinished instance UNKNOWN."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_21552_gb300 import build
    build.build()
    from paper_2601_21552_gb300 import api, binding
    return api, binding


def cpu_closure(nv, clauses, assumptions):
    """Plain fixpoint of unit propagation (test-side): returns (conflict,
    values[nv] with 0 open / 1 true / 2 false)."""
    val = np.zeros(nv + 1, np.int8)   # 1 true, -1 false
    k = max([len(c) for c in clauses] + [1])
    C = np.zeros((max(len(clauses), 1), k), np.int64)
    for i, c in enumerate(clauses):
        C[i, :len(c)] = c
    pad = C == 0
    if any(len(c) == 0 for c in clauses):
        return True, None
    for l in list(assumptions) + [c[0] for c in clauses if len(set(c)) == 1]:
        want = 1 if l > 0 else -1
        if val[abs(l)] == -want:
            return True, None
        val[abs(l)] = want
    while True:
        lv = np.where(pad, -1, val[np.abs(C)] * np.sign(C))
        sat = (lv == 1).any(axis=1)
        opn = (lv == 0)
        # distinct open literals per clause
        first = np.where(opn, C, np.iinfo(np.int64).min).max(axis=1)
        lo = np.where(opn, C, np.iinfo(np.int64).max).min(axis=1)
        nopen = opn.sum(axis=1)
        single = (nopen >= 1) & (first == lo)
        if ((nopen == 0) & ~sat).any():
            return True, None
        unit = single & ~sat
        if not unit.any():
            break
        lits = first[unit]
        for l in np.unique(lits):
            want = 1 if l > 0 else -1
            if val[abs(l)] == -want or (-l in set(lits.tolist())):
                return True, None
            val[abs(l)] = want
    out = np.where(val[1:] == 1, 1, np.where(val[1:] == -1, 2, 0)).astype(np.uint8)
    return False, out


def _cases():
    rng = np.random.default_rng(11)
    cases = []
    for s in range(60):
        n, l = queries.random_3sat(9000 + s, 40, 90)
        cases.append((n, [list(map(int, c)) for c in l]))
    for s in range(30):   # generic: clauses of length 1..6, duplicates allowed
        n = int(rng.integers(10, 40))
        cls = [[int(rng.integers(1, n + 1)) * (1 if rng.random() < 0.5 else -1)
                for _ in range(int(rng.integers(1, 7)))] for _ in range(int(rng.integers(n, 3 * n)))]
        cases.append((n, cls))
    return cases


def _csr(cases):
    icb, cb, lits, nv, vb = [0], [0], [], [], [0]
    for n, cls in cases:
        for c in cls:
            lits.extend(c)
            cb.append(len(lits))
        icb.append(len(cb) - 1)
        nv.append(n)
        vb.append(vb[-1] + n)
    return (np.array(icb, np.int64), np.array(cb, np.int64), np.array(lits, np.int32),
            np.array(nv, np.int32), np.array(vb, np.int64))


def test_gpu_closure_equals_cpu_closure(libs):
    api, B = libs
    rng = np.random.default_rng(5)
    cases = _cases()
    # encoded bounds queries too (the solver's real CNFs)
    irs, _ = queries.config1(40, w=6)
    enc = B.scuba_encode_batch(irs)
    for i in range(enc.n):
        c0, c1 = enc.inst_clause_begin[i], enc.inst_clause_begin[i + 1]
        cls = [enc.lits[enc.clause_begin[c]:enc.clause_begin[c + 1]].tolist() for c in range(c0, c1)]
        cases.append((int(enc.inst_num_vars[i]), cls))
    asm_b, asm_l = [0], []
    for n, _ in cases:
        k = int(rng.integers(0, min(8, n) + 1))
        vs = rng.choice(np.arange(1, n + 1), size=k, replace=False)
        asm_l.extend(int(v) if rng.random() < 0.5 else -int(v) for v in vs)
        asm_b.append(len(asm_l))
    icb, cb, lits, nv, vb = _csr(cases)
    db = api.DeviceBatch.from_csr(icb, cb, lits, nv, vb)
    d_ab = torch.tensor(asm_b, dtype=torch.int64, device="cuda")
    d_al = torch.tensor(asm_l or [0], dtype=torch.int32, device="cuda")
    values = torch.zeros(int(vb[-1]), dtype=torch.uint8, device="cuda")
    confl = torch.zeros(len(cases), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert B._lib.scuba_propagate_batch(db.struct(), d_ab.data_ptr(), d_al.data_ptr(),
                                        values.data_ptr(), confl.data_ptr(), s) == 0
    assert B.scuba_sync_status(s) == 0
    vals, cf = values.cpu().numpy(), confl.cpu().numpy()
    n_conf = 0
    for i, (n, cls) in enumerate(cases):
        want_c, want_v = cpu_closure(n, cls, asm_l[asm_b[i]:asm_b[i + 1]])
        assert bool(cf[i]) == want_c, i
        if not want_c:
            assert (vals[vb[i]:vb[i] + n] == want_v).all(), i
        n_conf += want_c
    assert 0 < n_conf < len(cases)


def _hard_batch(api, count=64):
    cases = []
    for s in range(count):
        n, l = queries.random_3sat(31000 + s, 300, 300)
        cases.append((n, [list(map(int, c)) for c in l]))
    icb, cb, lits, nv, vb = _csr(cases)
    return api.DeviceBatch.from_csr(icb, cb, lits, nv, vb)


def test_abort_flag_stops_the_search(libs):
    api, B = libs
    db = _hard_batch(api)
    flag = torch.ones(1, dtype=torch.int32, device="cuda")
    v, _, _ = api.solve(db, abort_flag_ptr=flag.data_ptr(), time_budget_ms=60000)
    assert api.status() == B.SCUBA_ERR_ABORTED
    assert (v.cpu().numpy() != 1).sum() > 0  # hard instances stay UNKNOWN
    assert set(v.cpu().numpy().tolist()) <= {0, 1, 2}


def test_time_budget_ends_the_search(libs):
    api, B = libs
    db = _hard_batch(api)
    v, _, _ = api.solve(db, time_budget_ms=50)
    assert api.status() == B.SCUBA_ERR_TIMEOUT
    vh = v.cpu().numpy()
    assert (vh == 2).sum() > 0
    # the context is still usable afterwards
    irs, _ = queries.config1(16, w=6)
    res = api.solve_queries(irs, time_budget_ms=60000)
    assert res["status"] == 0 and res["fails"] == 0
