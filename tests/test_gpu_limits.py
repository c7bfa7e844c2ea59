"""Size limits and malformed units through the C ABI: each is refused by a
host-side check (before any launch) or by the kernels' own validation (the
unit then comes back UNKNOWN with a status), never by a fault."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from raw_cnf import pack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_21552_gb300 import build
    build.build()
    from paper_2601_21552_gb300 import api, binding
    return api, binding


def _batch(B, cnfs, max_vars=None):
    icb, cb, lits, nv, vb, L = pack(cnfs)
    t = lambda a: torch.from_numpy(a).cuda()
    keep = [t(icb), t(cb), t(lits), t(nv), t(vb)]
    b = B.make_batch(len(cnfs), int(nv.max()) if max_vars is None else max_vars, len(cb) - 1, L,
                     int(vb[-1]), *(x.data_ptr() for x in keep))
    return b, keep


def _status(B, fn):
    try:
        fn()
    except RuntimeError as e:  # the binding raises on a synchronous error
        return int(str(e).split("status ")[1].split(":")[0])
    return B.scuba_sync_status(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("search,max_vars", [("dpll", 1 << 29), ("cdcl", 1 << 29),
                                             ("dpll", 1_000_000), ("cdcl", 500_000)])
def test_declared_sizes_over_the_limits(libs, search, max_vars):
    """max_vars >= 2^29, or an assignment (2 bits per variable for DPLL, 4 for
    clause learning) larger than a warp's share of shared memory."""
    api, B = libs
    b, keep = _batch(B, [(3, [[1, 2, 3]])], max_vars=max_vars)
    v = torch.zeros(1, dtype=torch.uint8, device="cuda")
    o = api.options(search=search, learnt_words=max_vars + 64 if search == "cdcl" else 0)
    st = _status(B, lambda: B.scuba_solve_batch_ex(b, v.data_ptr(), None,
                                                   torch.cuda.current_stream().cuda_stream, o))
    assert st == B.SCUBA_ERR_TOO_LARGE


def test_instance_over_declared_max_vars(libs):
    api, B = libs
    b, keep = _batch(B, [(10, [[1, 10]]), (2, [[1, 2]])], max_vars=4)
    v = torch.full((2,), 9, dtype=torch.uint8, device="cuda")
    st = _status(B, lambda: B.scuba_solve_batch_ex(b, v.data_ptr(), None,
                                                   torch.cuda.current_stream().cuda_stream,
                                                   api.options()))
    assert st == B.SCUBA_ERR_MALFORMED
    assert v.cpu().tolist()[0] == 2  # UNKNOWN


@pytest.mark.parametrize("search", ["dpll", "cdcl"])
def test_malformed_units(libs, search):
    """Units whose assumptions are too many or out of range, or whose
    instance index is out of range, come back UNKNOWN with
    SCUBA_ERR_MALFORMED; the other units are still decided."""
    api, B = libs
    from paper_2601_21552_gb300.api import DeviceBatch
    cnfs = [(300, [[1, 2], [-1, 2], [3, 300]])]
    icb, cb, lits, nv, vb, L = pack(cnfs)
    db = DeviceBatch.from_csr(icb, cb, lits, nv, vb)
    asm = [[1], list(range(1, 300)), [301], [-2]]   # ok, 299 > 248, out of range, UNSAT
    begin = np.concatenate([[0], np.cumsum([len(a) for a in asm])]).astype(np.int64)
    flat = np.array([x for a in asm for x in a], np.int32)
    v, m, mb = api.solve_units(db, [0, 0, 0, 0], begin, flat, search=search)
    st = api.status()
    assert st == B.SCUBA_ERR_MALFORMED
    assert v.cpu().tolist() == [1, 2, 2, 0]
    v, m, mb = api.solve_units(db, [0, 1], np.array([0, 1, 2], np.int64),
                               np.array([1, 1], np.int32), search=search)
    assert api.status() == B.SCUBA_ERR_MALFORMED
    assert v.cpu().tolist() == [1, 2]


@pytest.mark.parametrize("search", ["dpll", "cdcl"])
def test_units_without_assumptions_and_models(libs, search):
    """Units with no assumptions are whole instances; every unit's model is
    written at its own offset and satisfies its instance and assumptions."""
    api, B = libs
    from paper_2601_21552_gb300.api import DeviceBatch
    cnfs = [(4, [[1, 2], [-1, 3], [-3, 4]]), (2, [[1], [-1, 2]])]
    icb, cb, lits, nv, vb, L = pack(cnfs)
    db = DeviceBatch.from_csr(icb, cb, lits, nv, vb)
    units = [0, 0, 1, 1, 0]
    asm = [[], [1], [], [-2], [1, -4]]  # SAT, SAT, SAT, UNSAT (unit 2 forced), UNSAT
    begin = np.concatenate([[0], np.cumsum([len(a) for a in asm])]).astype(np.int64)
    flat = np.array([x for a in asm for x in a] or [0], np.int32)
    v, m, mb = api.solve_units(db, units, begin, flat, search=search)
    assert api.status() == 0
    assert v.cpu().tolist() == [1, 1, 1, 0, 0]
    mh, mbh = m.cpu().numpy(), mb.cpu().numpy()
    for u in range(3):
        n, cls = cnfs[units[u]]
        val = mh[mbh[u]:mbh[u] + n]
        assert all(any((val[abs(l) - 1] == 1) == (l > 0) for l in c) for c in cls)
        assert all((val[abs(l) - 1] == 1) == (l > 0) for l in asm[u])
