"""Benchmark: batched out-of-bounds satisfiability checks on GB300.

Workload (N=1): 4,096 intra-allocation partition queries with 16-bit inputs,
the partition/bounds family shaped like the paper's Figs. 1, 3 and 5 (seeded
synthetic inputs; the paper's 20 programs are not available). One step = one
complete pass of the hot path over the batch with the CNFs already resident
in HBM: device prep (clause normalisation, occurrence lists) + the
persistent DPLL search + verdict finalisation. Verdicts are checked
bit-exactly against stored oracle verdicts after timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--heuristic activity|learned]

Under torchrun each rank solves its own batch (different seeds): weak
scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "verdicts/sec + BCP propagations/sec on 1 GB300, learned vs plain, bit-exact"
WORKLOAD = "partition queries, 16-bit inputs (4,096 per GPU)"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _workload(rank: int, count: int, width: int = 16):
    from workloads import queries
    seed0 = queries.SEED_BASE[2] + rank * 1_000_000
    irs, params = queries.config2(count, w=width, seed0=seed0)
    return irs, params


def _stored_verdicts():
    p = os.path.join(ROOT, "tests", "golden", "config2_w16_oracle_verdicts.txt")
    return np.array([int(x) for x in open(p).read().split()], np.uint8)


def cpu_baseline(irs, target_s: float = 15.0, seed: int = 7):
    """The oracle as it stands, on a bounded random sample of the workload,
    on all host cores."""
    import oracle
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(irs))
    threads = oracle.default_threads()
    done, props, t_used = 0, 0, 0.0
    chunk = max(threads * 2, 32)
    k = 0
    while t_used < target_s and k < len(order):
        sel = [irs[i] for i in order[k:k + chunk]]
        t0 = time.perf_counter()
        r = oracle.solve_queries(sel, threads=threads)
        t_used += time.perf_counter() - t0
        done += len(sel)
        props += int(r["stats"][:, 2].sum())
        k += chunk
    return {"value": done / t_used, "unit": "verdicts/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} of {len(irs)} queries drawn uniformly (seed {seed}), {t_used:.1f}s",
            "propagations_per_s": props / t_used}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    irs, _ = _workload(0, 4096)
    rng = np.random.default_rng(11)
    threads = oracle.default_threads()
    per_step = 96
    times, counts, props = [], [], []
    for s in range(args.warmup + args.steps):
        sel_idx = rng.choice(len(irs), size=per_step, replace=False)
        sel = [irs[i] for i in sel_idx]
        t0 = time.perf_counter()
        r = oracle.solve_queries(sel, threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            counts.append(len(sel))
            props.append(int(r["stats"][:, 2].sum()))
    tot = sum(times)
    value = sum(counts) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "verdicts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": per_step,
                       "propagations_per_s": sum(props) / tot},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value,
                             "unit": "verdicts/s",
                             "sample": f"{per_step} queries per step drawn uniformly from the "
                                       f"4,096-query workload"},
            "e2e": {"value": value, "unit": "verdicts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2601_21552_gb300 import api, binding as B
    from paper_2601_21552_gb300 import build as pb
    pb.build()

    count = args.queries
    irs, params = _workload(rank, count, args.width)
    t_enc = time.perf_counter()
    enc = B.scuba_encode_batch(irs)
    t_enc = time.perf_counter() - t_enc
    db = api.DeviceBatch(enc, dev)
    torch.cuda.synchronize()
    heur = B.SCUBA_HEUR_LEARNED if args.heuristic == "learned" else B.SCUBA_HEUR_ACTIVITY
    stream = torch.cuda.current_stream(dev)

    def step(stats=None, events=None):
        verdict = torch.empty(count, dtype=torch.uint8, device=dev)
        o = api.options(heuristic=heur, stats=stats, time_budget_ms=300000, events=events)
        B.scuba_solve_batch_ex(db.struct(), verdict.data_ptr(), None, stream.cuda_stream, o)
        return verdict

    for _ in range(args.warmup):
        step()
    rc = api.status(stream)
    assert rc == 0, f"warm-up solve failed: {rc} {B.last_error()}"

    # timed region: K steps, per-step search-kernel events
    stats = torch.zeros((count, B.SCUBA_NSTATS), dtype=torch.int64, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for a, b in ev:  # create the underlying events on this stream
        a.record(stream)
        b.record(stream)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    verdicts = []
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            verdicts.append(step(stats=stats, events=ev[k]))
        t_end.record(stream)
        torch.cuda.synchronize()
    rc = api.status(stream)
    assert rc == 0, f"timed solve failed: {rc}"
    if ws > 1:
        torch.distributed.barrier()
    ms_total = t_start.elapsed_time(t_end)
    ms_search = [a.elapsed_time(b) for a, b in ev]
    if ws > 1:
        t = torch.tensor([ms_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())

    # parity after timing
    v = verdicts[-1].cpu().numpy()
    parity = None
    if rank == 0 and count == 4096 and args.width == 16:
        stored = _stored_verdicts()
        parity = int((v == stored).sum())
        assert parity == count, f"verdicts differ from the oracle on {count - parity} queries"
    st = stats.cpu().numpy().astype(np.float64) / args.steps
    props = st[:, 2].sum()
    visits = st[:, 3].sum()
    alg_bytes = 16 * props + 8 * visits + 4 * st[:, 4].sum() + 4 * st[:, 5].sum()
    ms_step = ms_total / args.steps
    search_ms = float(np.mean(ms_search))

    # end to end through the host entry point (host buffers, copies inside)
    h_verdict = np.zeros(count, np.uint8)
    hb = B.make_batch(enc.n, enc.max_vars, enc.total_clauses, enc.total_lits, enc.total_vars,
                      enc.inst_clause_begin.ctypes.data, enc.clause_begin.ctypes.data,
                      enc.lits.ctypes.data, enc.inst_num_vars.ctypes.data,
                      enc.inst_var_begin.ctypes.data)
    o = api.options(heuristic=heur, time_budget_ms=300000)
    B.scuba_solve_batch_host(hb, h_verdict, None, stream.cuda_stream, o)  # warm
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = B.scuba_solve_batch_host(hb, h_verdict, None, stream.cuda_stream, o)
        e2e_t.append(time.perf_counter() - t0)
        assert rc == 0
    h2d = db.h2d_bytes
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / (search_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": count * ws / (ms_step * 1e-3),
        "unit": "verdicts/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "heuristic": args.heuristic,
        "propagations_per_s": props * ws / (ms_step * 1e-3),
        "config": {"workload": WORKLOAD, "queries_per_gpu": count, "input_bits": 16,
                   "clauses_total": enc.total_clauses, "literals_total": enc.total_lits,
                   "vars_total": enc.total_vars, "l2": "inputs larger than L2 (CSR + occurrence "
                   "lists > 1 GB)", "encode_s": t_enc, "parity": f"{parity}/{count} bit-exact"},
        "e2e": {"value": count / float(np.median(e2e_t)), "unit": "verdicts/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": count},
        "gpu_launches": 10 * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "kernel": "k_solve",
                     "peak_source": src, "search_ms": search_ms},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(irs, target_s=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--heuristic", default="activity", choices=["activity", "learned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--queries", type=int, default=4096,
                    help="queries per GPU (profiling runs use smaller cases)")
    ap.add_argument("--width", type=int, default=16, help="input word width in bits")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
