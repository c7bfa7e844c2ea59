"""Splitting one query list over several GPUs, one process per GPU.

The queries of a batch are independent (the paper decides one constraint
set per static memory instruction, Sec. V-B), so a batch shards with no
exchange during the solve:

* ``lpt_partition`` -- longest-processing-time assignment of instances to G
  shards by clause count: largest first, each to the shard with the least
  clauses so far (ties to the lowest shard). Deterministic, so every rank
  computes the same partition from the same counts without communicating.
* ``sub_csr`` -- the CSR of the instances of one shard, renumbered from 0
  (what that rank uploads and solves).
* ``gather`` -- the shards' verdicts and models written back into the
  caller's arrays in the original instance order and model layout.
* ``gather_over_ranks`` -- the same on rank 0 from every rank's host
  arrays through a CPU process group (a plain host gather: the only
  communication, after the solve).

Costs are clause counts of the encoded CNFs; the encoder is host code, so
every rank can encode the list and agree on the partition.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(costs, shards: int) -> list[np.ndarray]:
    """Indices of each shard (ascending within a shard). Every index lands in
    exactly one shard; shard loads differ by at most the largest cost."""
    if shards < 1:
        raise ValueError("shards must be >= 1")
    c = np.asarray(costs, dtype=np.int64).reshape(-1)
    order = np.argsort(-c, kind="stable")
    heap = [(0, g) for g in range(shards)]
    members: list[list[int]] = [[] for _ in range(shards)]
    for i in order:
        load, g = heapq.heappop(heap)
        members[g].append(int(i))
        heapq.heappush(heap, (load + int(c[i]), g))
    return [np.array(sorted(m), dtype=np.int64) for m in members]


def sub_csr(icb, cb, lits, nv, idx):
    """CSR (inst_clause_begin, clause_begin, lits, inst_num_vars,
    inst_var_begin) of instances `idx` of a batch, in that order, with
    clause and literal offsets renumbered from 0."""
    icb = np.asarray(icb, np.int64)
    cb = np.asarray(cb, np.int64)
    lits = np.asarray(lits, np.int32)
    nv = np.asarray(nv, np.int32)
    idx = np.asarray(idx, np.int64)
    out_icb = [0]
    out_cb = [np.zeros(1, np.int64)]
    out_lits = []
    lbase = 0
    for i in idx:
        c0, c1 = icb[i], icb[i + 1]
        l0, l1 = cb[c0], cb[c1]
        out_cb.append(cb[c0 + 1:c1 + 1] - l0 + lbase)
        out_lits.append(lits[l0:l1])
        lbase += int(l1 - l0)
        out_icb.append(out_icb[-1] + int(c1 - c0))
    snv = nv[idx] if len(idx) else np.zeros(0, np.int32)
    vb = np.concatenate([[0], np.cumsum(snv, dtype=np.int64)])
    return (np.array(out_icb, np.int64), np.concatenate(out_cb),
            np.concatenate(out_lits) if out_lits else np.zeros(0, np.int32),
            snv.astype(np.int32), vb.astype(np.int64))


def gather(n: int, var_begin, parts):
    """Host verdict[n] and model[var_begin[n]] from shard results.
    parts: iterable of (idx, verdict_shard, model_shard or None), the model of
    a shard laid out by its own sub_csr inst_var_begin."""
    vb = np.asarray(var_begin, np.int64)
    verdict = np.full(n, 2, dtype=np.uint8)
    model = np.zeros(int(vb[n]) if n else 0, dtype=np.uint8)
    seen = np.zeros(n, dtype=bool)
    for idx, v, m in parts:
        idx = np.asarray(idx, np.int64)
        if seen[idx].any():
            raise ValueError("an instance appears in two shards")
        seen[idx] = True
        verdict[idx] = np.asarray(v, np.uint8)[:len(idx)]
        if m is not None:
            m = np.asarray(m, np.uint8)
            off = 0
            for i in idx:
                k = int(vb[i + 1] - vb[i])
                model[vb[i]:vb[i] + k] = m[off:off + k]
                off += k
    if not seen.all():
        raise ValueError("an instance is in no shard")
    return verdict, model


def gather_over_ranks(n: int, var_begin, idx, verdict, model, group=None, dst: int = 0):
    """Every rank passes its shard (idx, host verdict, host model or None);
    rank `dst` returns the gathered (verdict, model), the others None. Uses
    torch.distributed.gather_object on `group` (a CPU/gloo group)."""
    import torch.distributed as dist
    mine = (np.asarray(idx, np.int64), np.asarray(verdict, np.uint8),
            None if model is None else np.asarray(model, np.uint8))
    rank = dist.get_rank()
    got = [None] * dist.get_world_size() if rank == dst else None
    dist.gather_object(mine, got, dst=dst, group=group)
    if rank != dst:
        return None
    return gather(n, var_begin, got)
