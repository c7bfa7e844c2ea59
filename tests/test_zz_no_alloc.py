"""The allocation-free entry point, for callers that cannot call cudaMalloc
(for example code running under another framework's allocator, or a plugin
whose host forbids device allocation). It must give exactly the verdicts of
the regular entry point, on two calls in a row (its scratch array keeps the
previous call's contents), and refuse batches larger than its fixed scratch.

Kept in its own file, named to be collected last."""
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


def _batch(api, B, irs):
    enc = B.scuba_encode_batch(irs)
    return enc, api.DeviceBatch(enc, "cuda")


def test_noalloc_matches_regular_entry_point_twice(libs):
    api, B = libs
    enc, db = _batch(api, B, queries.config1(256)[0])
    stream = torch.cuda.current_stream().cuda_stream
    # regular entry point
    v_ref = torch.empty(db.n, dtype=torch.uint8, device="cuda")
    B.scuba_solve_batch_ex(db.struct(), v_ref.data_ptr(), None, stream,
                           api.options(time_budget_ms=60000))
    assert B.scuba_sync_status(stream) == 0
    ref = v_ref.cpu().numpy()
    assert set(ref.tolist()) == {0, 1}
    for call in range(2):
        v = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
        m = torch.zeros(db.total_vars, dtype=torch.uint8, device="cuda")
        rc = B.scuba_solve_batch_noalloc(db.struct(), v.data_ptr(), m.data_ptr(), stream,
                                         api.options(time_budget_ms=60000))
        assert rc == 0, B.last_error()
        got = v.cpu().numpy()
        assert (got == ref).all(), f"call {call}: verdicts differ"
        fails, ok = B.scuba_verify_batch(enc, got, m.cpu().numpy())
        assert fails == 0
    # a regular call after the allocation-free ones still launches: the
    # allocation-free call never lowers the search kernel's shared-memory grant
    v_after = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
    B.scuba_solve_batch_ex(db.struct(), v_after.data_ptr(), None, stream,
                           api.options(time_budget_ms=60000))
    assert B.scuba_sync_status(stream) == 0, B.last_error()
    assert (v_after.cpu().numpy() == ref).all()


def _raw_noalloc(B, db, v, opt, stream):
    """The C-ABI call itself (the binding raises on a negative status)."""
    import ctypes
    return B._lib.scuba_solve_batch_noalloc(ctypes.byref(db.struct()), v.data_ptr(), None,
                                            stream, ctypes.byref(opt))


def test_noalloc_reports_abort_like_the_regular_entry_point(libs):
    api, B = libs
    # 16-bit partition queries: the guarded ones need thousands of decisions,
    # so their searches reach the abort poll (every 64 search steps)
    enc, db = _batch(api, B, queries.config2(64)[0])
    stream = torch.cuda.current_stream().cuda_stream
    clean = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
    B.scuba_solve_batch_ex(db.struct(), clean.data_ptr(), None, stream,
                           api.options(time_budget_ms=60000))
    assert B.scuba_sync_status(stream) == 0
    clean = clean.cpu().numpy()
    flag = torch.ones(1, dtype=torch.int32, device="cuda")  # raised before the call
    v_ref = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
    B.scuba_solve_batch_ex(db.struct(), v_ref.data_ptr(), None, stream,
                           api.options(abort_flag_ptr=flag.data_ptr(), time_budget_ms=60000))
    st_ref = B.scuba_sync_status(stream)
    assert st_ref == B.SCUBA_ERR_ABORTED
    v = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
    rc = _raw_noalloc(B, db, v, api.options(abort_flag_ptr=flag.data_ptr(),
                                            time_budget_ms=60000), stream)
    assert rc == st_ref, B.last_error()
    # instances finished before their first poll keep their verdict; every
    # other one is UNKNOWN, never a wrong verdict
    for got in (v.cpu().numpy(), v_ref.cpu().numpy()):
        assert (got == 2).any()
        decided = got != 2
        assert (got[decided] == clean[decided]).all()
    # the next call with the flag down starts from a clean status
    flag.zero_()
    rc = _raw_noalloc(B, db, v, api.options(abort_flag_ptr=flag.data_ptr(),
                                            time_budget_ms=60000), stream)
    assert rc == 0, B.last_error()
    assert (v.cpu().numpy() == clean).all()


def test_noalloc_decision_budget_leaves_unknown_with_status_ok(libs):
    api, B = libs
    # guarded 16-bit partition queries need far more than 2 decisions each
    enc, db = _batch(api, B, queries.config2(64)[0])
    stream = torch.cuda.current_stream().cuda_stream
    opt = api.options(decision_budget=2, split=False, time_budget_ms=60000)
    v_ref = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
    B.scuba_solve_batch_ex(db.struct(), v_ref.data_ptr(), None, stream, opt)
    st_ref = B.scuba_sync_status(stream)
    v = torch.full((db.n,), 9, dtype=torch.uint8, device="cuda")
    rc = _raw_noalloc(B, db, v, api.options(decision_budget=2, split=False,
                                            time_budget_ms=60000), stream)
    assert rc == st_ref == 0, B.last_error()
    got, ref = v.cpu().numpy(), v_ref.cpu().numpy()
    assert set(got.tolist()) <= {0, 1, 2} and (got == 2).any()
    both = (got != 2) & (ref != 2)
    assert (got[both] == ref[both]).all()


def test_noalloc_refuses_batches_above_its_fixed_scratch(libs):
    api, B = libs
    enc, db = _batch(api, B, queries.config2(512)[0])  # ~100 MB of scratch
    v = torch.empty(db.n, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="more than the fixed"):
        B.scuba_solve_batch_noalloc(db.struct(), v.data_ptr(), None,
                                    torch.cuda.current_stream().cuda_stream, api.options())
