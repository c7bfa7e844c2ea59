"""The N > 1 path of the benchmark on CPU: two gloo ranks, each with its own
shard of queries (weak scaling: different seeds, no data exchange), timing
reduced as the max over ranks, and the whole-job value aggregated from the
per-rank batch size. Each rank decides its shard with the CPU oracle as a
stand-in for the GPU solve (this host has no GPU)."""
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
    import oracle
    w, r = bench._dist()
    assert (w, r) == (ws, rank)
    irs, params = bench._workload(r, 24, width=6)
    verdict = oracle.solve_queries(irs, threads=1)["verdict"]
    ms = 100.0 + 50.0 * rank          # per-rank step time (rank 1 is the slow one)
    ms_max = bench.max_over_ranks(ms)
    value = bench.aggregate_value(24, w, ms_max)
    # gather what each rank saw (test-side check only)
    sig = torch.tensor([float(sum(p["k1"] * 31 + p["c"] for p in params))], dtype=torch.float64)
    sigs = [torch.zeros(1, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(sigs, sig)
    out[rank] = (ms_max, value, [float(s.item()) for s in sigs], verdict.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms_max, value, sigs, verdict = res[r]
        assert ms_max == 150.0                       # max over ranks, on every rank
        assert value == pytest.approx(24 * 2 / 0.150)
        assert sigs[0] != sigs[1]                    # different shards per rank
        assert set(verdict) <= {0, 1}
    # each rank's shard is the workload of its own seed range
    import sys
    sys.path.insert(0, ROOT)
    import bench
    a, _ = bench._workload(0, 24, width=6)
    b, _ = bench._workload(1, 24, width=6)
    assert any((x.shape != y.shape) or (x != y).any() for x, y in zip(a, b))


def test_single_process_helpers_are_identities():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.aggregate_value(4096, 1, 800.0) == pytest.approx(5120.0)
