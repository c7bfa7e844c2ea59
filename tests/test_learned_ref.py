"""CPU pins for the FP64 reference of the branching network: its analytic
gradient against central finite differences, and the softmax cross-entropy
against a direct evaluation."""
import numpy as np

from oracle import mlp_ref as R


def _problem(seed=0, rows=90):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(rows, R.NFEAT))
    target = rng.integers(0, 5, size=rows).astype(np.float64)
    nodes = [(0, 30), (30, 1), (31, 40), (71, 19)]
    target[31:71] = 0.0   # a node with zero targets is skipped
    p = rng.normal(scale=0.3, size=R.NPARAM)
    return p, X, nodes, target


def test_gradient_matches_finite_differences():
    p, X, nodes, target = _problem()
    g = R.grad(p, X, nodes, target)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(R.NPARAM, 60, replace=False), [R.NPARAM - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (R.loss(p + e, X, nodes, target) - R.loss(p - e, X, nodes, target)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_loss_is_cross_entropy_of_softmax():
    p, X, nodes, target = _problem(3)
    W1, b1, w2, b2 = R.unflat(p)
    s = np.maximum(X @ W1 + b1, 0) @ w2 + b2
    want = 0.0
    for r0, n in nodes:
        t = target[r0:r0 + n]
        if n < 2 or t.sum() == 0:
            continue
        q = np.exp(s[r0:r0 + n]) / np.exp(s[r0:r0 + n]).sum()
        want += -(t / t.sum() * np.log(q)).sum()
    assert abs(R.loss(p, X, nodes, target) - want) < 1e-9


def test_bf16_decode():
    u = np.array([0x3F80, 0xC000, 0x0000, 0x4049], np.uint16)
    assert R.bf16_to_f64(u).tolist() == [1.0, -2.0, 0.0, 3.140625]
