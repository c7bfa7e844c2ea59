"""Seeded query families shaped like the paper's examples.

Each family mirrors the constraint kinds of Sec. V-B: kind 1 (thread id below
block dimension), kind 3 (equalities defining the offset and size expression
trees, plus asserts/guards), kind 2 (the offset leaves its allocation or its
logical partition). Inputs are w-bit unsigned words; arithmetic is exact.

* ``bounds_query``: the 1-D access of Fig. 5 (saxpy) and Fig. 1 (fluid):
  idx = bid*bdim + tid, offset = a*idx + c, size = k1*n + k0, optional guard
  idx < n (the path condition of Fig. 2's ``if (i < numv)``).
* ``partition_query``: the intra-allocation case of Fig. 3 (sosfilt) and the
  partition-size rule of Fig. 7b: one allocation of size k1*n + k0 split at
  p_i = i*m with m = n / k; partition j ends at p_{j+1}, the last one at the
  allocation size; the query is offset outside [p_j, end_j).
* ``grown_query``: bounds/partition queries grown with the paper's
  multiplicative structure (2-D/3-D ids as in Fig. 1's ``threadIdx.y*16 +
  threadIdx.x``, cubic sizes like Fig. 1's ``(cubN+1)^3*Nelements*3``) until
  a structural size proxy reaches a log-uniform target.
* ``random_3sat``: uniform random 3-SAT (no IR; a DIMACS-style clause list).

The generator is deliberately free of the method's arithmetic: it only emits
IR. Every random draw comes from ``SplitMix64`` so workloads are identical on
every machine.
"""
from __future__ import annotations

import math

import numpy as np

from .ir import IR
from .rng import SplitMix64

# Seeds follow a fixed convention: config c, query i uses seed base(c) + i.
SEED_BASE = {1: 1000, 2: 200000, 3: 3000000, 4: 4000000, 5: 5000000}


def bounds_query(w: int, k1: int, k0: int, a: int, c: int, guard: bool) -> IR:
    """Config-1 template (1-D bounds check of one global-memory access)."""
    ir = IR()
    n = ir.free(w, "n")
    tid = ir.free(w, "tid")
    bid = ir.free(w, "bid")
    bdim = ir.free(w, "bdim")
    idx = ir.add(ir.mul(bid, bdim), tid)
    offset = ir.add(ir.mul(ir.const(a), idx), ir.const(c))
    size = ir.add(ir.mul(ir.const(k1), n), ir.const(k0))
    ir.assert_(ir.ult(tid, bdim))            # kind 1
    if guard:
        ir.assert_(ir.ult(idx, n))           # path condition / assert
    ir.assert_(ir.ule(size, offset))         # kind 2: offset >= size
    return ir


def partition_query(w: int, k1: int, k0: int, a: int, c: int, k: int, j: int,
                    guard: bool) -> IR:
    """Config-2 template (intra-allocation partition check)."""
    ir = IR()
    n = ir.free(w, "n")
    tid = ir.free(w, "tid")
    bid = ir.free(w, "bid")
    bdim = ir.free(w, "bdim")
    idx = ir.add(ir.mul(bid, bdim), tid)
    size = ir.add(ir.mul(ir.const(k1), n), ir.const(k0))
    m = ir.udiv(n, k)
    p_j = ir.mul(ir.const(j), m)
    end_j = ir.mul(ir.const(j + 1), m) if j < k - 1 else size
    local = ir.add(ir.mul(ir.const(a), idx), ir.const(c))
    offset = ir.add(p_j, local)
    ir.assert_(ir.ult(tid, bdim))
    if guard:
        ir.assert_(ir.ult(idx, m))
    ir.assert_(ir.or_(ir.ult(offset, p_j), ir.ule(end_j, offset)))
    return ir


def config1_params(seed: int, w: int = 8) -> dict:
    r = SplitMix64(seed)
    return dict(w=w, k1=r.randint(1, 4), k0=r.randint(0, 7), a=r.randint(1, 4),
                c=r.randint(0, 7), guard=r.bernoulli(0.5))


def config2_params(seed: int, w: int = 16) -> dict:
    r = SplitMix64(seed)
    p = dict(w=w, k1=r.randint(1, 4), k0=r.randint(0, 7), a=r.randint(1, 4),
             c=r.randint(0, 7))
    p["k"] = r.randint(2, 8)
    p["j"] = r.randint(0, p["k"] - 1)
    p["guard"] = r.bernoulli(0.5)
    return p


def config1(count: int = 256, w: int = 8, seed0: int | None = None):
    """Return (irs, params) for the config-1 family."""
    seed0 = SEED_BASE[1] if seed0 is None else seed0
    params = [config1_params(seed0 + i, w) for i in range(count)]
    return [bounds_query(**p).to_array() for p in params], params


def config2(count: int = 4096, w: int = 16, seed0: int | None = None):
    seed0 = SEED_BASE[2] if seed0 is None else seed0
    params = [config2_params(seed0 + i, w) for i in range(count)]
    return [partition_query(**p).to_array() for p in params], params


# --------------------------------------------------------------------------
# Grown (uneven) queries.
# --------------------------------------------------------------------------

CELLS_PER_CLAUSE = 1.0 / 14.0   # size proxy calibration (cells per encoded clause)


def grown_query(seed: int, target_clauses: float | None = None) -> tuple[IR, dict]:
    """One config-3 query: width from {8,16,32} (p = .4/.4/.2), a clause-count
    target log-uniform in [500, 200k], grown from a bounds or partition base by
    adding thread-block dimensions (idx*bd + t), row-major scalings (idx*R +
    col) and cubic size factors ((N+1)^3*E*3, Fig. 1) while a size proxy stays
    within the target.

    The proxy counts bit-cells: a product of words of widths p and q costs
    p*q cells, a p-bit sum or comparison p cells; widths follow exact
    arithmetic (p*q has p+q bits). It only steers growth; the encoded size is
    whatever the encoder produces and is reported as such."""
    r = SplitMix64(seed)
    u = r.uniform()
    w = 8 if u < 0.4 else (16 if u < 0.8 else 32)
    if target_clauses is None:
        target_clauses = math.exp(math.log(500) + r.uniform() * (math.log(200000) - math.log(500)))
    budget = target_clauses * CELLS_PER_CLAUSE
    k1, k0, a, c = r.randint(1, 4), r.randint(0, 7), r.randint(1, 4), r.randint(0, 7)
    guard = r.bernoulli(0.5)
    use_part = r.bernoulli(0.3)
    k = r.randint(2, 8)
    j = r.randint(0, k - 1)

    ir = IR()
    n = ir.free(w, "n")
    tid = ir.free(w, "tid")
    bid = ir.free(w, "bid")
    bdim = ir.free(w, "bdim")
    ir.assert_(ir.ult(tid, bdim))
    idx = ir.add(ir.mul(bid, bdim), tid)
    limit = n                      # what the guard bounds idx by
    size = ir.add(ir.mul(ir.const(k1), n), ir.const(k0))
    w_idx, w_lim, w_size = 2 * w + 1, w, w + 3
    cells = w * w + 6 * w
    structs = []

    def cost(kind):
        if kind in ("dim", "rows"):    # idx*x + t, limit*x, size*x, t < x
            return w_idx * w + w_lim * w + w_size * w + 4 * w
        wf = 3 * (w + 1) + w + 2       # width of (N+1)^3 * E * 3
        return ((w + 1) ** 2 + 2 * (w + 1) ** 2 + (3 * w + 3) * w + 2 * (4 * w + 3)
                + w_size * wf + w_lim * wf)

    for _ in range(64):
        kinds = ["dim", "cube", "rows"]
        first = r.randint(0, 2)
        choice = None
        for t in range(3):
            kd = kinds[(first + t) % 3]
            if cells + cost(kd) <= budget * 1.15:
                choice = kd
                break
        if choice is None or cells >= budget * 0.85:
            break
        cells += cost(choice)
        if choice == "dim":
            bd = ir.free(w, "bd")
            t_ = ir.free(w, "t")
            ir.assert_(ir.ult(t_, bd))
            idx = ir.add(ir.mul(idx, bd), t_)
            limit = ir.mul(limit, bd)
            size = ir.mul(size, bd)
            w_idx, w_lim, w_size = w_idx + w + 1, w_lim + w, w_size + w
        elif choice == "cube":
            big_n = ir.free(w, "N")
            e = ir.free(w, "E")
            n1 = ir.add(big_n, ir.const(1))
            f = ir.mul(ir.mul(ir.mul(ir.mul(n1, n1), n1), e), ir.const(3))
            size = ir.mul(size, f)
            limit = ir.mul(limit, f)
            wf = 3 * (w + 1) + w + 2
            w_lim, w_size = w_lim + wf, w_size + wf
        else:
            rows = ir.free(w, "R")
            col = ir.free(w, "col")
            ir.assert_(ir.ult(col, rows))
            idx = ir.add(ir.mul(idx, rows), col)
            limit = ir.mul(limit, rows)
            size = ir.mul(size, rows)
            w_idx, w_lim, w_size = w_idx + w + 1, w_lim + w, w_size + w
        structs.append(choice)
    offset = ir.add(ir.mul(ir.const(a), idx), ir.const(c))
    if use_part:
        m = ir.udiv(size, k)
        p_j = ir.mul(ir.const(j), m)
        end_j = ir.mul(ir.const(j + 1), m) if j < k - 1 else size
        if guard:
            ir.assert_(ir.ult(idx, ir.udiv(limit, k)))
        off2 = ir.add(p_j, offset)
        ir.assert_(ir.or_(ir.ult(off2, p_j), ir.ule(end_j, off2)))
    else:
        if guard:
            ir.assert_(ir.ult(idx, limit))
        ir.assert_(ir.ule(size, offset))
    return ir, dict(w=w, target_clauses=target_clauses, cells=cells, structs=structs,
                    guard=guard, partition=use_part)


def config3(count: int = 65536, seed0: int | None = None):
    seed0 = SEED_BASE[3] if seed0 is None else seed0
    out, meta = [], []
    for i in range(count):
        ir, m = grown_query(seed0 + i)
        out.append(ir.to_array())
        meta.append(m)
    return out, meta


# --------------------------------------------------------------------------
# Uniform random 3-SAT (config 5).
# --------------------------------------------------------------------------

def random_3sat(seed: int, n_lo: int = 200, n_hi: int = 400, ratio: float = 4.26):
    """Uniform random 3-SAT: n ~ U[n_lo, n_hi], m = round(ratio*n), three
    distinct variables per clause, each negated with probability 1/2.

    Returns (nvars, lits) with lits an int32 array of shape (m, 3), DIMACS
    numbering (+-v, v in 1..n). Per clause, six candidate variables are drawn
    and the first three distinct ones are kept (rejection sampling); the rare
    clause without three distinct candidates redraws from the scalar stream."""
    r = SplitMix64(seed)
    nv = r.randint(n_lo, n_hi)
    m = int(round(ratio * nv))
    raw = r.u64_block(m * 7).reshape(m, 7)
    cand = (raw[:, :6] % np.uint64(nv)).astype(np.int64) + 1
    signs = raw[:, 6]
    out = np.zeros((m, 3), dtype=np.int64)
    out[:, 0] = cand[:, 0]
    # second: first candidate different from the first
    d1 = cand[:, 1:] != cand[:, :1]
    has1 = d1.any(axis=1)
    i1 = np.argmax(d1, axis=1) + 1
    out[:, 1] = cand[np.arange(m), i1]
    # third: first candidate after the second's position different from both
    pos = np.arange(6)[None, :]
    d2 = (cand != out[:, :1]) & (cand != out[:, 1:2]) & (pos > i1[:, None])
    has2 = d2.any(axis=1)
    out[:, 2] = cand[np.arange(m), np.argmax(d2, axis=1)]
    for i in np.flatnonzero(~(has1 & has2)):
        chosen = [int(cand[i, 0])]
        while len(chosen) < 3:
            v = r.randint(1, nv)
            if v not in chosen:
                chosen.append(v)
        out[i] = chosen
    neg = np.stack([(signs >> np.uint64(b)) & np.uint64(1) for b in range(3)], axis=1)
    out = np.where(neg == 1, -out, out)
    return nv, out.astype(np.int32)


def config4_split(count_train: int = 2048, count_test: int = 4096, w: int = 16):
    """Learned-branching workload: the config-2 generator with a seed split,
    even seeds for training traces and odd seeds for the held-out test."""
    base = SEED_BASE[4]
    tr = [config2_params(base + 2 * i, w) for i in range(count_train)]
    te = [config2_params(base + 2 * i + 1, w) for i in range(count_test)]
    return ([partition_query(**p).to_array() for p in tr], tr,
            [partition_query(**p).to_array() for p in te], te)


def config5_sat(count: int = 10000, seed0: int | None = None):
    seed0 = SEED_BASE[5] if seed0 is None else seed0
    return [random_3sat(seed0 + i) for i in range(count)]


def config5_bounds(count: int = 10000, seed0: int | None = None):
    seed0 = (SEED_BASE[5] + 500000) if seed0 is None else seed0
    return config1(count, w=32, seed0=seed0)
