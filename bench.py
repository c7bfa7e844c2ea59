"""Benchmark: batched out-of-bounds satisfiability checks on GB300.

Workload (N=1): 4,096 intra-allocation partition queries with 16-bit inputs,
the partition/bounds family shaped like the paper's Figs. 1, 3 and 5 (seeded
synthetic inputs; the paper's 20 programs are not available). One step = one
complete pass of the hot path over the batch with the CNFs already resident
in HBM: device prep (clause normalisation, occurrence lists) + the
persistent search + verdict finalisation. Verdicts are checked bit-exactly
against stored oracle verdicts after timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--arms cdcl,learned,plain]

Arms (each a full pass over the same batch, same verdicts required):
  cdcl     conflict-driven clause learning with activity branching (headline)
  learned  DPLL whose top decisions are ordered by the incidence MLP, trained
           beforehand (not timed; reported under "learned_training") on
           decision traces of the plain search over held-out seeds
  plain    DPLL with activity branching only
The headline value is the first arm; all arms are reported under "arms".

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


# DRAM traffic of the clause-learning search kernel from one single-pass ncu
# capture of a full launch (profiles/k_solve_cdcl_partition16.md: 6.61 GB read +
# 5.45 GB written for 1.4327e8 propagations), per propagation, valid only for
# the kernel sources it was taken on (sha256 prefix of solver.cu + learn.cuh +
# cdcl.cuh); scaled to each launch by the propagations it processes.
PROFILED_SOURCES = "c77c54a6c17b6968"
DRAM_BYTES_PER_PROPAGATION = {"cdcl": (6.61e9 + 5.45e9) / 1.4327e8}


def _kernel_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("solver.cu", "learn.cuh", "cdcl.cuh"):
        with open(os.path.join(ROOT, "paper_2601_21552_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# L2 traffic of the same kernel from one single-pass ncu capture of a full
# launch (lts__t_bytes.sum: 135.89 GB for 1.5016e8 propagations;
# profiles/k_solve_cdcl_partition16.md), per propagation, under the same
# source hash (idle warps polling the job ring included).
L2_BYTES_PER_PROPAGATION = {"cdcl": 135.89e9 / 1.5016e8}


def l2_probe(dev, mib: int = 32, iters: int = 200) -> float:
    """Achievable L2 bandwidth (GB/s, read + write) of a plain elementwise
    copy whose source and destination (2 x `mib` MiB) stay resident in the
    129 MB L2, timed with CUDA events after a warm-up."""
    import torch
    n = mib * (1 << 20) // 4
    x = torch.ones(n, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    for _ in range(10):
        y.copy_(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(iters):
        y.copy_(x)
    e1.record()
    e1.synchronize()
    return 2.0 * n * 4 * iters / (e0.elapsed_time(e1) * 1e-3) / 1e9


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


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank timing over all ranks (identity without a process
    group); the backend is whatever torch.distributed was initialised with."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(count_per_rank: int, world_size: int, ms_per_step: float) -> float:
    """Whole-job verdicts/s: every rank solves its own batch of
    count_per_rank queries per step (weak scaling), the step time is the max
    over ranks."""
    return count_per_rank * world_size / (ms_per_step * 1e-3)


def _workload(rank: int, count: int, width: int = 16):
    from workloads import queries
    seed0 = queries.SEED_BASE[2] + rank * 1_000_000
    irs, params = queries.config2(count, w=width, seed0=seed0)
    return irs, params


def _stored_verdicts():
    p = os.path.join(ROOT, "tests", "golden", "config2_w16_oracle_verdicts.txt")
    return np.array([int(x) for x in open(p).read().split()], np.uint8)


def cpu_baseline(irs, target_s: float = 15.0, seed: int = 7, algo: str = "cdcl"):
    """The oracle as it stands, on a bounded random sample of the workload,
    on all host cores (algo: its clause-learning or its DPLL solver)."""
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
        r = oracle.solve_queries(sel, threads=threads, algo=algo)
        t_used += time.perf_counter() - t0
        done += len(sel)
        props += int(r["stats"][:, 2].sum())
        k += chunk
    # one host thread on the first queries of the same sample (about a fifth
    # of the time budget): the per-core rate; clause learning only (the DPLL
    # solver's heavy tail would make one query's time unbounded)
    done1, props1, t1, k1 = 0, 0, 0.0, 0
    while algo == "cdcl" and t1 < target_s / 5 and k1 < min(k, len(order)):
        sel = [irs[i] for i in order[k1:k1 + 8]]
        t0 = time.perf_counter()
        r = oracle.solve_queries(sel, threads=1, algo=algo)
        t1 += time.perf_counter() - t0
        done1 += len(sel)
        props1 += int(r["stats"][:, 2].sum())
        k1 += 8
    return {"value": done / t_used, "unit": "verdicts/s", "cores": threads, "kind": "oracle",
            "algo": algo,
            "sample": f"{done} of {len(irs)} queries drawn uniformly (seed {seed}), {t_used:.1f}s",
            "propagations_per_s": props / t_used,
            **({"single_core": {"verdicts_per_s": done1 / t1, "propagations_per_s": props1 / t1,
                                "sample": f"the first {done1} of that sample, {t1:.1f}s, 1 thread"}}
               if t1 else {})}


def run_reference(args):
    """The oracle on the host cores: its clause-learning solver over the whole
    4,096-query workload per step (the DPLL solver would need minutes per
    step; it is timed on a sample inside the GPU arm's cpu_baseline_dpll)."""
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    irs, _ = _workload(0, 4096)
    threads = oracle.default_threads()
    times, counts, props = [], [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle.solve_queries(irs, threads=threads, algo="cdcl")
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            counts.append(len(irs))
            props.append(int(r["stats"][:, 2].sum()))
    tot = sum(times)
    value = sum(counts) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "verdicts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "queries_per_step": len(irs),
                       "propagations_per_s": sum(props) / tot},
            "cpu_baseline": {"kind": "oracle", "algo": "cdcl", "cores": threads, "value": value,
                             "unit": "verdicts/s",
                             "sample": "the whole 4,096-query workload every step"},
            "e2e": {"value": value, "unit": "verdicts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _train_network(api, B, dev, args):
    """Decision traces of the plain search on the training split (even seeds
    of the config-2 generator), then Adam on the GPU. Not timed as a step."""
    from workloads import queries
    t0 = time.perf_counter()
    tr_irs, _, _, _ = queries.config4_split(args.train_queries, 0, w=args.width)
    enc = B.scuba_encode_batch(tr_irs)
    db = api.DeviceBatch(enc, dev)
    trace, _, _ = api.record_trace(db, depth=args.trace_depth, max_nodes=1 << 17,
                                   max_rows=1 << 25, decision_budget=args.trace_budget,
                                   time_budget_ms=300000)
    nodes, rows = trace.used()
    net = api.Mlp(seed=3, device=dev)
    losses = net.train(trace, epochs=args.epochs, batch_nodes=64, lr=3e-3)
    torch_sync = __import__("torch").cuda.synchronize
    torch_sync()
    info = {"train_queries": args.train_queries, "trace_nodes": nodes, "trace_rows": rows,
            "epochs": args.epochs, "loss_first": losses[0] if losses else None,
            "loss_last": losses[-1] if losses else None,
            "train_s": time.perf_counter() - t0, "learned_depth": args.learned_depth,
            "trace_depth": args.trace_depth}
    del trace
    return net, info


def _timed_arm(api, B, db, dev, stream, count, heur_opts, args, use_graph=True):
    """W warm-up solves, then K timed steps (CUDA-graph replays of one solve).
    Returns per-arm timings, counters and the last verdicts."""
    import torch
    stats = torch.zeros((count, B.SCUBA_NSTATS), dtype=torch.int64, device=dev)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record(stream)
    ev[1].record(stream)
    verdict = torch.empty(count, dtype=torch.uint8, device=dev)

    def launch(st_tensor, events):
        o = api.options(stats=st_tensor, time_budget_ms=300000, events=events,
                        num_inputs=db.num_inputs, **heur_opts)
        B.scuba_solve_batch_ex(db.struct(), verdict.data_ptr(), None, stream.cuda_stream, o)

    for _ in range(args.warmup):
        launch(None, None)
    rc = api.status(stream)
    assert rc == 0, f"warm-up solve failed: {rc} {B.last_error()}"
    graph = None
    if use_graph:
        # one captured solve (no timing events inside: events recorded in a
        # capture cannot be read back); replays are timed from outside
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            launch(stats, None)
        torch.cuda.synchronize()
        stats.zero_()
    ms_search = []
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for _ in range(args.steps):
        if graph is not None:
            graph.replay()
        else:
            launch(stats, ev)
            ev[1].synchronize()
            ms_search.append(ev[0].elapsed_time(ev[1]))
    t_end.record(stream)
    torch.cuda.synchronize()
    rc = api.status(stream)
    assert rc == 0, f"timed solve failed: {rc}"
    st = stats.cpu().numpy().astype(np.float64) / args.steps
    if graph is not None:  # search-kernel time from one direct launch
        launch(None, ev)
        ev[1].synchronize()
        ms_search.append(ev[0].elapsed_time(ev[1]))
    return {"ms_total": t_start.elapsed_time(t_end), "ms_search": ms_search, "stats": st,
            "verdict": verdict.cpu().numpy().copy()}


def _l2_line(arm, head, ws, dev):
    """The search kernel's L2 throughput (ncu L2 bytes per propagation times
    the measured propagations/s) against the achievable L2 bandwidth of
    l2_probe: the survey's BCP-vs-L2 target."""
    probe = l2_probe(dev)
    per = L2_BYTES_PER_PROPAGATION.get(arm)
    ok = per is not None and _kernel_sources_sha() == PROFILED_SOURCES
    achieved = per * head["propagations_per_s"] / ws / 1e9 if ok else None
    return {"achieved": achieved, "achievable": probe, "unit": "GB/s",
            "frac": achieved / probe if achieved is not None else None,
            "source": "ncu lts__t_bytes.sum per propagation (single pass, full launch) x "
                      "propagations/s; achievable = L2-resident copy probe"}


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
    stream = torch.cuda.Stream(dev)  # graphs cannot be captured on the legacy stream

    from paper_2601_21552_gb300 import autotune
    tuned = autotune.load()  # launch shape / sharing parameters from the last sweep
    tuned_cdcl = autotune.load(section="best_cdcl")
    # the first arm is the headline; the others are measured beside it
    arms = [a for a in args.arms.split(",") if a]
    assert arms and set(arms) <= {"cdcl", "learned", "plain"}, args.arms
    net, train_info = None, None
    if "learned" in arms:
        net, train_info = _train_network(api, B, dev, args)

    def arm_options(arm):
        opts = dict(tuned)
        if arm == "learned":
            opts.update(heuristic=B.SCUBA_HEUR_LEARNED, mlp_weights=net.weights,
                        learned_depth=args.learned_depth)
        elif arm == "cdcl":
            opts.update(tuned_cdcl, search="cdcl")
        return opts

    if ws > 1:
        torch.distributed.barrier()
    results = {}
    with ClockSampler(local) as clk:
        for arm in arms:
            results[arm] = _timed_arm(api, B, db, dev, stream, count, arm_options(arm), args,
                                      use_graph=args.graph)
    if ws > 1:
        torch.distributed.barrier()
    for arm in arms:
        results[arm]["ms_total"] = max_over_ranks(results[arm]["ms_total"], dev)

    # parity after timing: both arms bit-exact against the stored oracle verdicts
    parity = {}
    if rank == 0 and count == 4096 and args.width == 16:
        stored = _stored_verdicts()
        for arm in arms:
            ok = int((results[arm]["verdict"] == stored).sum())
            assert ok == count, f"{arm}: verdicts differ from the oracle on {count - ok} queries"
            parity[arm] = f"{ok}/{count} bit-exact"
    for arm in arms[1:]:
        assert (results[arm]["verdict"] == results[arms[0]]["verdict"]).all(), arm

    # end to end through the host entry point (host buffers, copies inside)
    # the host arrays in pinned memory, so the copies inside the call are DMA
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pinned(a) for a in (enc.inst_clause_begin, enc.clause_begin, enc.lits,
                                enc.inst_num_vars, enc.inst_var_begin)]
    h_verdict = torch.zeros(count, dtype=torch.uint8).pin_memory().numpy()
    hb = B.make_batch(enc.n, enc.max_vars, enc.total_clauses, enc.total_lits, enc.total_vars,
                      *(t.data_ptr() for t in h_in))
    o = api.options(time_budget_ms=300000, **arm_options(arms[0]))  # the headline arm
    B.scuba_solve_batch_host(hb, h_verdict, None, stream.cuda_stream, o)  # warm
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = B.scuba_solve_batch_host(hb, h_verdict, None, stream.cuda_stream, o)
        e2e_t.append(time.perf_counter() - t0)
        assert rc == 0
    assert (h_verdict == results[arms[0]]["verdict"]).all(), "host-buffer verdicts differ"
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    def arm_summary(r):
        st = r["stats"]
        ms_step = r["ms_total"] / args.steps
        props = st[:, 2].sum()
        alg_bytes = 16 * props + 8 * st[:, 3].sum() + 4 * st[:, 4].sum() + 4 * st[:, 5].sum()
        search_ms = float(np.mean(r["ms_search"]))
        return {"value": aggregate_value(count, ws, ms_step), "unit": "verdicts/s",
                "ms_per_step": ms_step, "propagations_per_s": props * ws / (ms_step * 1e-3),
                "decisions_per_step": float(st[:, 0].sum()),
                "search_ms": search_ms, "search_ms_steps": r["ms_search"],
                "alg_bytes": float(alg_bytes)}

    summ = {arm: arm_summary(results[arm]) for arm in arms}
    head = summ[arms[0]]
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = head["alg_bytes"] / (head["search_ms"] * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "verdicts/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "arm": arms[0],
        "search": "cdcl" if arms[0] == "cdcl" else "dpll",
        "heuristic": "learned" if arms[0] == "learned" else "activity",
        "propagations_per_s": head["propagations_per_s"],
        "config": {"workload": WORKLOAD, "queries_per_gpu": count, "input_bits": args.width,
                   "clauses_total": enc.total_clauses, "literals_total": enc.total_lits,
                   "vars_total": enc.total_vars,
                   "l2": "inputs larger than L2 (CSR + occurrence lists > 1 GB)",
                   "encode_s": t_enc, "cuda_graph": args.graph, "parity": parity,
                   "autotuned": {"dpll": tuned, "cdcl": tuned_cdcl}},
        "arms": summ,
        "e2e": {"value": count / float(np.median(e2e_t)), "unit": "verdicts/s",
                "h2d_bytes_per_step": db.h2d_bytes, "d2h_bytes_per_step": count},
        "gpu_launches": 10 * args.steps,
        "l2": _l2_line(arms[0], head, ws, dev),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (DRAM_BYTES_PER_PROPAGATION[arms[0]] * head["propagations_per_s"]
                                 * head["ms_per_step"] * 1e-3 / ws
                                 if arms[0] in DRAM_BYTES_PER_PROPAGATION
                                 and _kernel_sources_sha() == PROFILED_SOURCES else None),
                     "traffic_unit": "bytes per launch (ncu, scaled by propagations)",
                     "kernel": f"k_solve ({arms[0]} search)", "peak_source": src,
                     "limiter": "latency: dependent L1/L2 loads and instruction issue "
                                "per propagation round, DRAM mostly idle",
                     "search_ms": head["search_ms"]},
        "clocks": clk.summary(),
    }
    if train_info:
        line["learned_training"] = train_info
    if not args.no_cpu_baseline:
        # the oracle's clause-learning solver (the stronger CPU program), and
        # its DPLL beside it
        line["cpu_baseline"] = cpu_baseline(irs, target_s=args.cpu_seconds, algo="cdcl")
        line["cpu_baseline_dpll"] = cpu_baseline(irs, target_s=args.cpu_seconds / 2, algo="dpll")
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arms", default="cdcl,learned,plain",
                    help="comma list of cdcl, learned, plain; the first is the headline")
    ap.add_argument("--graph", action="store_true",
                    help="replay each step from a captured CUDA graph")
    ap.add_argument("--learned-depth", type=int, default=6,
                    help="decisions at depth < this are scored by the network")
    ap.add_argument("--trace-depth", type=int, default=8,
                    help="decisions at depth < this are recorded for training")
    ap.add_argument("--train-queries", type=int, default=2048)
    ap.add_argument("--trace-budget", type=int, default=20000,
                    help="decision budget per training query while tracing")
    ap.add_argument("--epochs", type=int, default=20)
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
