"""Closed-form verdicts for the bounds and partition query families.

Written from the constraint definitions of Sec. V-B (kind 1: tid < bdim;
kind 2: offset >= size, or offset outside the partition [p_j, end_j) of the
Fig. 7b partition-size rule; kind 3: the defining equalities), independently
of the oracle. Exact integer semantics; inputs are w-bit unsigned.

Two facts make these closed forms:
  * idx = bid*bdim + tid with tid < bdim reaches every value in
    [0, 2^w - 1] (bdim = 1, tid = 0, bid = idx) and its maximum is
    IDXMAX = (2^w - 1)^2 + (2^w - 2).
  * offset = a*idx + c is increasing in idx, so only the largest admissible
    idx matters: n - 1 (guard idx < n), m - 1 (guard idx < m) or IDXMAX.

Each verdict is computed twice -- by endpoint algebra and by enumerating the
single remaining free quantity (n, or m and r) -- and the two must agree.
"""
from __future__ import annotations


def idx_max(w: int) -> int:
    top = (1 << w) - 1
    return top * top + (top - 1)


# -- bounds family (config 1): size = k1*n + k0, offset = a*idx + c ---------

def bounds_enum(w, k1, k0, a, c, guard) -> bool:
    top = (1 << w) - 1
    for n in range(0, top + 1):
        if guard:
            if n == 0:
                continue
            hi = n - 1
        else:
            hi = idx_max(w)
        if a * hi + c >= k1 * n + k0:
            return True
    return False


def bounds_algebra(w, k1, k0, a, c, guard) -> bool:
    top = (1 << w) - 1
    if not guard:
        return a * idx_max(w) + c >= k0          # n = 0 minimises the size
    # exists n in [1, top]: a(n-1) + c >= k1 n + k0  <=>  (a-k1) n >= a + k0 - c
    lhs = lambda n: (a - k1) * n
    rhs = a + k0 - c
    return lhs(1) >= rhs or lhs(top) >= rhs


# -- partition family (config 2) ---------------------------------------------
# S = k1*n + k0, m = n // k, p_j = j*m, end_j = (j+1)*m (j < k-1) or S.
# offset = p_j + a*idx + c >= p_j always, so the query is a*idx + c >= end_j - p_j.

def _part_width(n, k1, k0, k, j):
    m = n // k
    return (m if j < k - 1 else k1 * n + k0 - (k - 1) * m), m


def partition_enum(w, k1, k0, a, c, k, j, guard) -> bool:
    top = (1 << w) - 1
    for n in range(0, top + 1):
        width, m = _part_width(n, k1, k0, k, j)
        if guard:
            if m == 0:
                continue
            hi = m - 1
        else:
            hi = idx_max(w)
        if a * hi + c >= width:
            return True
    return False


def partition_algebra(w, k1, k0, a, c, k, j, guard) -> bool:
    top = (1 << w) - 1
    if not guard:
        min_width = 0 if j < k - 1 else k0      # n = 0
        return a * idx_max(w) + c >= min_width
    M = top // k
    if M < 1:
        return False
    if j < k - 1:
        # a(m-1) + c >= m  <=>  (a-1) m >= a - c
        f = lambda m: (a - 1) * m
        rhs = a - c
    else:
        # a(m-1) + c >= k1(km + r) + k0 - (k-1)m, smallest right side at r = 0
        f = lambda m: (a - k1 * k + k - 1) * m
        rhs = a - c + k0
    return f(1) >= rhs or f(M) >= rhs


# -- the C wrap-around variant (unsigned W-bit arithmetic) -------------------
# Brute force over every input: n, bdim, tid, bid each w-bit, kind 1
# tid < bdim, and every program value reduced modulo 2^W as C's unsigned
# W-bit arithmetic does; partition sizes and the bounds check are exact
# (pointer arithmetic). Nothing here shares code with the encoders or the
# front end.

def _wrap_inputs(w):
    import numpy as np
    r = np.arange(1 << w, dtype=np.int64)
    n, bdim, tid, bid = np.meshgrid(r, r, r, r, indexing="ij")
    return n, bdim, tid, bid, tid < bdim


def bounds_wrap(w, k1, k0, a, c, guard, W) -> bool:
    M = 1 << W
    n, bdim, tid, bid, ok = _wrap_inputs(w)
    idx = (bid * bdim + tid) % M
    off = (a * idx + c) % M
    size = (k1 * n + k0) % M
    if guard:
        ok = ok & (idx < n)
    return bool((ok & (off >= size)).any())


def partition_wrap(w, k1, k0, a, c, k, j, guard, W) -> bool:
    M = 1 << W
    n, bdim, tid, bid, ok = _wrap_inputs(w)
    m = n // k
    start = (j * m) % M
    end = ((j + 1) * m) % M if j < k - 1 else (k1 * n + k0) % M
    idx = (bid * bdim + tid) % M
    off = (a * idx + c) % M
    if guard:
        ok = ok & (idx < m)
    return bool((ok & (off >= end - start)).any())
