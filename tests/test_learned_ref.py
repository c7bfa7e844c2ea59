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


def test_adam_two_steps_hand_derived():
    """Algorithm 1 of Kingma and Ba worked by hand for gradients 1 then 3
    (beta1 0.9, beta2 0.999, eps 1e-8): step 1 moves by lr / (1 + eps) (m_hat = g, v_hat =
    g^2); step 2 has m_hat = (0.09 + 0.3) / 0.19 and v_hat = (0.000999 +
    0.009) / 0.001999, so it moves by lr * 2.052631... / sqrt(5.002001...)."""
    lr = 0.01
    p0, z = np.zeros(1), np.zeros(1)
    p1, m1, v1 = R.adam_step(p0, z, z, np.array([1.0]), 1, lr)
    assert abs(p1[0] - (-lr / (1.0 + 1e-8))) < 1e-15
    assert abs(m1[0] - 0.1) < 1e-15 and abs(v1[0] - 0.001) < 1e-15
    p2, m2, v2 = R.adam_step(p1, m1, v1, np.array([3.0]), 2, lr)
    m_hat = (0.09 + 0.3) / 0.19
    v_hat = (0.000999 + 0.009) / 0.001999
    assert abs(m_hat - 2.0526315789473686) < 1e-12
    assert abs(v_hat - 5.0020010005002) < 1e-9
    assert abs((p1[0] - p2[0]) - lr * m_hat / (np.sqrt(v_hat) + 1e-8)) < 1e-14
    assert abs((p1[0] - p2[0]) / lr - 0.917781) < 1e-6


def test_adam_scale_invariance_and_convergence():
    """Adam's step does not depend on the gradient's scale (eps aside), and it
    takes a separable convex quadratic to its minimum."""
    rng = np.random.default_rng(3)
    gs = rng.normal(size=(5, 40))
    pa = pb = np.zeros(40)
    ma = va = mb = vb = np.zeros(40)
    for t, g in enumerate(gs, start=1):
        pa, ma, va = R.adam_step(pa, ma, va, g, t, 1e-2)
        pb, mb, vb = R.adam_step(pb, mb, vb, 1000.0 * g, t, 1e-2)
    assert np.allclose(pa, pb, rtol=1e-6, atol=1e-12)
    a = rng.uniform(0.5, 5.0, size=40)
    x_star = rng.normal(size=40)
    x, m, v = np.zeros(40), np.zeros(40), np.zeros(40)
    for t in range(1, 4001):
        x, m, v = R.adam_step(x, m, v, a * (x - x_star), t, 1e-2)
    assert np.abs(x - x_star).max() < 1e-2
