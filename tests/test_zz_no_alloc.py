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


def test_noalloc_refuses_batches_above_its_fixed_scratch(libs):
    api, B = libs
    enc, db = _batch(api, B, queries.config2(512)[0])  # ~100 MB of scratch
    v = torch.empty(db.n, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="more than the fixed"):
        B.scuba_solve_batch_noalloc(db.struct(), v.data_ptr(), None,
                                    torch.cuda.current_stream().cuda_stream, api.options())
