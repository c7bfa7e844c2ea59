"""FP64 reference of the branching network's forward pass, loss and gradients.

TEST INFRASTRUCTURE ONLY (imported by tests/). The network is not in the
paper: it orders decisions of the search and never changes a verdict. This
module restates its plain definition so that the GPU gradients can be checked
against it; the definition itself is pinned by central finite differences in
tests/test_learned_ref.py.

Model: z = X W1 + b1, h = relu(z), s = h w2 + b2 (16 -> 64 -> 1).
Loss per node (a set of rows): cross-entropy between t / sum(t) and
softmax(s) over the node's rows; the total is the sum over nodes.
Training: Adam (Kingma and Ba, 2015, Algorithm 1) on the mean loss of each
minibatch of nodes, restated by adam_step; pinned in tests/test_learned_ref.py
by hand-derived values, scale invariance and convergence on a quadratic.
"""
from __future__ import annotations

import numpy as np

NFEAT, NHID = 16, 64
NPARAM = NFEAT * NHID + NHID + NHID + 1


def bf16_to_f64(u16: np.ndarray) -> np.ndarray:
    """BF16 bit patterns (uint16) -> float64."""
    return (np.asarray(u16, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def unpack_weights(blob: np.ndarray):
    """Packed device weights (bytes) -> W1[16,64], b1[64], w2[64], b2 (fp64)."""
    b = np.asarray(blob, dtype=np.uint8)
    w1t = bf16_to_f64(b[0:2048].view(np.uint16)).reshape(NHID, NFEAT)
    w2 = bf16_to_f64(b[2048:2176].view(np.uint16))
    b1 = b[2176:2432].view(np.float32).astype(np.float64)
    b2 = float(b[2432:2436].view(np.float32)[0])
    return w1t.T.copy(), b1, w2, b2


def flat(W1, b1, w2, b2) -> np.ndarray:
    return np.concatenate([W1.reshape(-1), b1, w2, [b2]])


def unflat(p: np.ndarray):
    W1 = p[:NFEAT * NHID].reshape(NFEAT, NHID)
    b1 = p[NFEAT * NHID:NFEAT * NHID + NHID]
    w2 = p[NFEAT * NHID + NHID:NFEAT * NHID + 2 * NHID]
    return W1, b1, w2, float(p[-1])


def scores(X, W1, b1, w2, b2):
    return np.maximum(X @ W1 + b1, 0.0) @ w2 + b2


def loss(p: np.ndarray, X, nodes, target) -> float:
    """Summed cross-entropy over nodes; nodes = list of (row_begin, rows)."""
    W1, b1, w2, b2 = unflat(p)
    s = scores(X, W1, b1, w2, b2)
    total = 0.0
    for r0, n in nodes:
        t = target[r0:r0 + n]
        if n < 2 or t.sum() <= 0:
            continue
        t = t / t.sum()
        ss = s[r0:r0 + n]
        lse = ss.max() + np.log(np.exp(ss - ss.max()).sum())
        total -= float((t * (ss - lse)).sum())
    return total


def grad(p: np.ndarray, X, nodes, target) -> np.ndarray:
    """Analytic gradient of loss() with respect to the flat parameters."""
    W1, b1, w2, b2 = unflat(p)
    z = X @ W1 + b1
    h = np.maximum(z, 0.0)
    s = h @ w2 + b2
    dS = np.zeros_like(s)
    for r0, n in nodes:
        t = target[r0:r0 + n]
        if n < 2 or t.sum() <= 0:
            continue
        t = t / t.sum()
        ss = s[r0:r0 + n]
        e = np.exp(ss - ss.max())
        dS[r0:r0 + n] = e / e.sum() - t
    gw2 = h.T @ dS
    gb2 = dS.sum()
    dh = np.outer(dS, w2) * (z > 0)
    gW1 = X.T @ dh
    gb1 = dh.sum(axis=0)
    return flat(gW1, gb1, gw2, gb2)


def adam_step(p: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, t: int,
              lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) in FP64: the biased
    first and second moment estimates, their bias corrections at step t >= 1,
    and the parameter step. Returns new (p, m, v); the inputs are unchanged."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
