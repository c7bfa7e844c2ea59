"""Learned branching on the GPU: the network's forward pass and gradients
(project kernels, tensor cores) against the FP64 reference on the same
BF16-rounded weights; decision traces; and the trained network inside the
search -- verdicts identical to the plain search and to the oracle, with the
decision counts of both reported."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp_ref as R
from workloads import queries

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_21552_gb300 import build
    build.build()
    from paper_2601_21552_gb300 import api, binding
    return api, binding


def _bf16_bits(a: np.ndarray) -> np.ndarray:
    """float -> BF16 bits, round to nearest even (test-side helper)."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16).astype(np.uint16)
    return r


def _synthetic_trace(api, rows=700, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(rows, 16)).astype(np.float32)
    xb = _bf16_bits(x)
    target = rng.integers(0, 6, size=rows).astype(np.float32)
    bounds = [0, 120, 121, 300, 450, 451, 700]
    tr = api.Trace(4, len(bounds) - 1, rows)
    tr.x.copy_(torch.from_numpy(xb.view(np.int16).reshape(-1)))
    tr.target.copy_(torch.from_numpy(target))
    nodes = [(bounds[i], bounds[i + 1] - bounds[i]) for i in range(len(bounds) - 1)]
    tr.node_row.copy_(torch.tensor([b for b, _ in nodes], dtype=torch.int64))
    tr.node_nrows.copy_(torch.tensor([n for _, n in nodes], dtype=torch.int32))
    tr.node_closed.fill_(1)
    tr.counts.copy_(torch.tensor([len(nodes), rows]))
    return tr, R.bf16_to_f64(xb), nodes, target.astype(np.float64)


def test_forward_and_gradient_match_fp64(libs):
    api, B = libs
    tr, X, nodes, target = _synthetic_trace(api)
    net = api.Mlp(seed=7)
    W1, b1, w2, b2 = R.unpack_weights(net.weights.cpu().numpy())
    p = R.flat(W1, b1, w2, b2)
    # forward
    scores = torch.zeros(X.shape[0], dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert B._lib.scuba_mlp_forward(tr.x.data_ptr(), X.shape[0], net.weights.data_ptr(),
                                    scores.data_ptr(), s) == 0
    ref_s = R.scores(X, W1, b1, w2, b2)
    assert np.allclose(scores.cpu().numpy(), ref_s, rtol=2e-3, atol=2e-3)
    # gradient
    grad = torch.zeros(R.NPARAM + 2, dtype=torch.float32, device="cuda")
    dS = torch.zeros(X.shape[0], dtype=torch.float32, device="cuda")
    t = tr.struct()
    import ctypes
    assert B._lib.scuba_mlp_grad(ctypes.byref(t), 0, len(nodes), net.weights.data_ptr(),
                                 grad.data_ptr(), dS.data_ptr(), s) == 0
    g = grad.cpu().numpy().astype(np.float64)
    ref = R.grad(p, X, nodes, target)
    assert abs(g[R.NPARAM] - R.loss(p, X, nodes, target)) < 1e-3 * max(1.0, abs(g[R.NPARAM]))
    assert g[R.NPARAM + 1] == 4  # nodes with >1 row and nonzero targets
    parts = {"W1": slice(0, 1024), "b1": slice(1024, 1088), "w2": slice(1088, 1152),
             "b2": slice(1152, 1153)}
    for name, sl in parts.items():
        a, b = g[:R.NPARAM][sl], ref[sl]
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert cos > 0.999, (name, cos)
        scale = np.abs(b).max() + 1e-12
        assert np.abs(a - b).max() <= 1e-2 * scale + 1e-6, (name, np.abs(a - b).max(), scale)


def test_trace_records_closed_nodes(libs):
    api, B = libs
    irs, _ = queries.config2(64, w=10)
    enc = B.scuba_encode_batch(irs)
    db = api.DeviceBatch(enc, "cuda")
    tr, v, st = api.record_trace(db, depth=4, time_budget_ms=60000)
    nodes, rows = tr.used()
    assert nodes > 0 and rows > 0
    closed = tr.node_closed.cpu().numpy()[:nodes]
    assert closed.all()
    nr = tr.node_nrows.cpu().numpy()[:nodes]
    depth = tr.node_depth.cpu().numpy()[:nodes]
    assert (depth < 4).all() and (nr > 0).all()
    assert rows == int(nr.sum())
    ref = oracle.solve_queries(irs)["verdict"]
    assert (v.cpu().numpy() == ref).all()
    x = tr.x.cpu().numpy()[:rows * 16].view(np.uint16).reshape(rows, 16)
    assert (R.bf16_to_f64(x[:, 15]) == 1.0).all()      # constant feature
    assert (tr.target.cpu().numpy()[:rows] >= 0).all()


def test_learned_branching_gain_and_identical_verdicts(libs):
    """Train on decision traces of even-seed queries, test on odd seeds: the
    learned search returns exactly the plain search's (and the oracle's)
    verdicts; the decision counts of both are reported."""
    api, B = libs
    tr_irs, _, te_irs, _ = queries.config4_split(512, 512, w=12)
    enc = B.scuba_encode_batch(tr_irs)
    db = api.DeviceBatch(enc, "cuda")
    trace, _, _ = api.record_trace(db, depth=6, time_budget_ms=120000)
    net = api.Mlp(seed=3)
    losses = net.train(trace, epochs=12, batch_nodes=64, lr=3e-3)
    assert losses[-1] < losses[0]
    te_enc = B.scuba_encode_batch(te_irs)
    te = api.DeviceBatch(te_enc, "cuda")
    v0, _, s0 = api.solve(te, want_model=False, time_budget_ms=120000)
    assert api.status() == 0
    v1, m1, s1 = api.solve(te, heuristic=B.SCUBA_HEUR_LEARNED, mlp_weights=net.weights,
                           learned_depth=6, time_budget_ms=120000)
    assert api.status() == 0
    v0, v1 = v0.cpu().numpy(), v1.cpu().numpy()
    ref = oracle.solve_queries(te_irs)["verdict"]
    assert (v0 == ref).all() and (v1 == ref).all()
    fails, _ = B.scuba_verify_batch(te_enc, v1, m1.cpu().numpy())
    assert fails == 0
    d0, d1 = int(s0[:, 0].sum().item()), int(s1[:, 0].sum().item())
    unsat = ref == 0
    report = {"train_queries": 512, "test_queries": 512, "input_bits": 12,
              "loss_first": losses[0], "loss_last": losses[-1],
              "decisions_plain": d0, "decisions_learned": d1,
              "decisions_plain_unsat": int(s0.cpu().numpy()[unsat, 0].sum()),
              "decisions_learned_unsat": int(s1.cpu().numpy()[unsat, 0].sum())}
    print("learned-vs-plain", json.dumps(report))
    out = os.environ.get("SCUBA_REPORT_DIR")
    if out:
        with open(os.path.join(out, "learned_vs_plain_w12.json"), "w") as f:
            json.dump(report, f)
