"""The N > 1 path on CPU with two gloo ranks.

* One query list split over the ranks: every rank encodes the list with the
  product encoder, takes its shard of the longest-processing-time partition
  by clause count, decides the shard's CSR, and rank 0 gathers verdicts and
  models into the original order and layout; the result equals a one-rank
  run and every gathered model passes the product's host re-verification.
* The benchmark's timing helpers: max over ranks, whole-job aggregate.

Each rank decides its shard with the CPU oracle as a stand-in for the GPU
solve (this host has no GPU); the partition, CSR extraction and gather are
the product's own code."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    w, r = bench._dist()
    assert (w, r) == (ws, rank)
    ms = 100.0 + 50.0 * rank          # per-rank step time (rank 1 is the slow one)
    ms_max = bench.max_over_ranks(ms)
    props = bench.sum_over_ranks(1000.0 * (rank + 1))
    value = bench.aggregate_value(24, w, ms_max)
    out[rank] = (ms_max, props, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_timing_helpers():
    """Max over ranks for the step time, sums for counters, and the whole-job
    value from the instances of all ranks over the slowest rank's time."""
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms_max, props, value = res[r]
        assert ms_max == 150.0                       # max over ranks, on every rank
        assert props == 3000.0                       # sum over ranks
        assert value == pytest.approx(24 * 2 / 0.150)


def test_single_process_helpers_are_identities():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.sum_over_ranks(7.0) == 7.0
    assert bench.aggregate_value(4096, 1, 800.0) == pytest.approx(5120.0)


# --------------------------------------------------------------------------
# One query list, LPT shards, host gather
# --------------------------------------------------------------------------

def _oracle_solve_csr(icb, cb, lits, nv):
    """Stand-in for the GPU solve of one shard: verdict and model per
    instance from the oracle's CDCL on the shard's own CSR."""
    import oracle
    v, models = [], []
    for i in range(len(nv)):
        c0, c1 = icb[i], icb[i + 1]
        l0 = cb[c0]
        cnf = oracle.CNF(int(nv[i]), cb[c0:c1 + 1] - l0, lits[l0:cb[c1]])
        r = oracle.cdcl(cnf)
        v.append(r["verdict"])
        models.append(r["model"][:int(nv[i])])
    model = np.concatenate(models) if models else np.zeros(0, np.uint8)
    return np.array(v, np.uint8), model.astype(np.uint8)


def _shard_rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2601_21552_gb300 import binding as B, shard
    from workloads import queries
    irs, _ = queries.config1(40, w=6)
    enc = B.scuba_encode_batch(irs)
    costs = np.diff(enc.inst_clause_begin)
    parts = shard.lpt_partition(costs, ws)
    idx = parts[rank]
    icb, cb, lits, nv, vb = shard.sub_csr(enc.inst_clause_begin, enc.clause_begin, enc.lits,
                                          enc.inst_num_vars, idx)
    v, m = _oracle_solve_csr(icb, cb, lits, nv)
    got = shard.gather_over_ranks(enc.n, enc.inst_var_begin, idx, v, m)
    if rank == 0:
        verdict, model = got
        fails, _ = B.scuba_verify_batch(enc, verdict, model)
        out[rank] = (verdict.tolist(), int(fails), [len(p) for p in parts],
                     [int(costs[p].sum()) for p in parts])
    else:
        out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_list_and_gather():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_shard_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[1] is None
    verdict, fails, sizes, loads = res[0]
    assert fails == 0 and sum(sizes) == 40 and min(sizes) > 0
    # the one-rank run of the same list
    import sys
    sys.path.insert(0, ROOT)
    from paper_2601_21552_gb300 import binding as B
    from workloads import queries
    irs, _ = queries.config1(40, w=6)
    enc = B.scuba_encode_batch(irs)
    one, _ = _oracle_solve_csr(enc.inst_clause_begin, enc.clause_begin, enc.lits,
                               enc.inst_num_vars)
    assert verdict == one.tolist()
    costs = np.diff(enc.inst_clause_begin)
    assert abs(loads[0] - loads[1]) <= costs.max()


def test_lpt_partition_properties():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2601_21552_gb300 import shard
    rng = np.random.default_rng(5)
    for G in (1, 2, 3, 8):
        c = rng.integers(1, 10_000, size=257)
        parts = shard.lpt_partition(c, G)
        allidx = np.sort(np.concatenate(parts))
        assert (allidx == np.arange(257)).all()                  # a partition
        loads = [int(c[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= c.max()                 # LPT bound
        # Graham's bound for LPT: at most (4/3 - 1/(3G)) of the optimum,
        # itself at least the mean load and the largest single cost
        opt_lb = max(c.sum() / G, c.max())
        assert max(loads) <= (4 / 3 - 1 / (3 * G)) * opt_lb + 1e-9 or G == 1
        assert all((a == b).all() for a, b in zip(parts, shard.lpt_partition(c, G)))
    # the textbook example: costs 5,5,4,4,3,3,3 on 3 machines give LPT 11
    parts = shard.lpt_partition([5, 5, 4, 4, 3, 3, 3], 3)
    assert max(sum([5, 5, 4, 4, 3, 3, 3][i] for i in p) for p in parts) == 11


def test_sub_csr_and_gather_round_trip():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2601_21552_gb300 import binding as B, shard
    from workloads import queries
    irs, _ = queries.config1(12, w=5)
    enc = B.scuba_encode_batch(irs)
    parts = shard.lpt_partition(np.diff(enc.inst_clause_begin), 3)
    results = []
    for idx in parts:
        icb, cb, lits, nv, vb = shard.sub_csr(enc.inst_clause_begin, enc.clause_begin,
                                              enc.lits, enc.inst_num_vars, idx)
        for j, i in enumerate(idx):   # every clause of every instance carried over
            a = enc.lits[enc.clause_begin[enc.inst_clause_begin[i]]:
                         enc.clause_begin[enc.inst_clause_begin[i + 1]]]
            b = lits[cb[icb[j]]:cb[icb[j + 1]]]
            assert (a == b).all()
            assert (np.diff(enc.clause_begin[enc.inst_clause_begin[i]:
                                             enc.inst_clause_begin[i + 1] + 1])
                    == np.diff(cb[icb[j]:icb[j + 1] + 1])).all()
        # a synthetic "result": verdict = instance index mod 2, model = the
        # instance index in every slot of its variables
        v = (idx % 2).astype(np.uint8)
        m = np.concatenate([np.full(enc.inst_num_vars[i], i % 251, np.uint8) for i in idx])
        results.append((idx, v, m))
    verdict, model = shard.gather(enc.n, enc.inst_var_begin, results)
    assert (verdict == np.arange(enc.n) % 2).all()
    for i in range(enc.n):
        assert (model[enc.inst_var_begin[i]:enc.inst_var_begin[i + 1]] == i % 251).all()
    with pytest.raises(ValueError):
        shard.gather(enc.n, enc.inst_var_begin, results[:-1])
