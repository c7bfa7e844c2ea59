"""Benchmark: batched out-of-bounds satisfiability checks on GB300.

Workload (default, N=1): 4,096 intra-allocation partition queries with 16-bit
inputs, the partition/bounds family shaped like the paper's Figs. 1, 3 and 5
(seeded synthetic inputs; the paper's 20 programs are not available). One
step = one complete pass of the hot path over the batch with the CNFs
already resident in HBM: device prep (clause normalisation, occurrence lists)
+ the persistent search + verdict finalisation. Verdicts are checked
bit-exactly against stored oracle verdicts after timing.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--config 1..5] [--arms cdcl,learned,plain] [--graph]

Arms (each a full pass over the same batch, same verdicts required):
  cdcl     conflict-driven clause learning with activity branching (headline)
  learned  DPLL whose top decisions are ordered by the incidence MLP, trained
           beforehand (not timed; reported under "learned_training") on
           decision traces of the plain search over the training seeds
  plain    DPLL with activity branching only
The headline value is the first arm; all arms are reported under "arms",
with "learned_over_plain" comparing the two DPLL arms.

--config selects the workload of one configuration (1: 256 bounds queries at
8 bits; 2: the default; 3: 65,536 grown queries of widths 8/16/32 in one
launch; 4: the 4,096 odd-seed held-out partition queries of the learned
configuration, with decision counts of both DPLL arms with splitting off;
5: 10,000 random 3-SAT instances mixed with 10,000 bounds queries at 32
bits). Configs 3 and 5 run with a per-instance budget and report UNKNOWNs.

Under torchrun the ranks split ONE query list of N x (queries per GPU) by
longest-processing-time on clause counts (weak scaling), solve their shards
with no collective on the data path, and rank 0 gathers verdicts on the host.
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


# DRAM traffic of the clause-learning search kernel from one single-pass ncu
# capture of a full bench launch (profiles/k_solve_cdcl_partition16.md: 8.71 GB
# read + 7.04 GB written for 1.2389e8 propagations), per propagation, valid
# only for the kernel sources it was taken on (sha256 prefix of solver.cu +
# learn.cuh + cdcl.cuh); scaled to each launch by the propagations it processes.
PROFILED_SOURCES = "d559d46d82c2e11f"
DRAM_BYTES_PER_PROPAGATION = {"cdcl": (8.7077e9 + 7.0410e9) / 1.2389e8}


def _kernel_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("solver.cu", "learn.cuh", "cdcl.cuh"):
        with open(os.path.join(ROOT, "paper_2601_21552_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# L2 traffic of the same kernel from the same single-pass ncu capture
# (lts__t_bytes.sum: 125.93 GB for 1.2389e8 propagations), per propagation,
# under the same source hash (idle warps polling the job ring and the
# clause-sharing pools included).
L2_BYTES_PER_PROPAGATION = {"cdcl": 125.93e9 / 1.2389e8}


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


def _workload(count: int, width: int = 16):
    """The default workload: `count` partition queries of the config-2
    generator (seeds SEED_BASE[2] + i); under torchrun the one list of
    N x (queries per GPU) queries that the ranks split."""
    from workloads import queries
    return queries.config2(count, w=width, seed0=queries.SEED_BASE[2])


def _stored(name):
    """Oracle verdicts stored under tests/golden (written by the scripts there,
    which call only the oracle): (header dict, uint8 verdicts)."""
    path = os.path.join(ROOT, "tests", "golden", name)
    head, digits = {}, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("#"):
                if ":" in line:
                    k, v = line[1:].split(":", 1)
                    head[k.strip()] = v.strip()
            elif line:
                digits.append(line)
    return head, np.frombuffer("".join(digits).encode(), dtype=np.uint8) - ord("0")


def _stored_verdicts():
    return _stored("config2_w16_oracle_verdicts.txt")[1]


def _fingerprint(arrays) -> str:
    import hashlib
    h = hashlib.sha256()
    for x in arrays:
        h.update(np.ascontiguousarray(x, dtype=np.int64).tobytes())
    return h.hexdigest()[:16]


def _pack_mixed(sat, enc):
    """One CSR of raw 3-SAT instances followed by an encoded query batch."""
    icb, cb, lits, nv = [0], [np.zeros(1, np.int64)], [], []
    base_c, base_l = 0, 0
    for n, l in sat:
        m = len(l)
        cb.append(base_l + 3 * np.arange(1, m + 1, dtype=np.int64))
        lits.append(l.reshape(-1))
        base_c += m
        base_l += 3 * m
        icb.append(base_c)
        nv.append(n)
    icb = np.concatenate([np.array(icb, np.int64), enc.inst_clause_begin[1:] + base_c])
    cb.append(enc.clause_begin[1:] + base_l)
    lits.append(enc.lits)
    nv = np.concatenate([np.array(nv, np.int32), enc.inst_num_vars])
    vb = np.concatenate([[0], np.cumsum(nv, dtype=np.int64)])
    return icb, np.concatenate(cb), np.concatenate(lits).astype(np.int32), nv, vb


class Work:
    """One configuration's batch on the host: CSR arrays, input-bit counts,
    the oracle's view of each instance (for the CPU baseline), budgets, and
    the stored oracle verdicts it is checked against."""

    def __init__(self, config, name, icb, cb, lits, nv, vb, ninp, oracle_items, stored,
                 budgets, arms, enc=None, fingerprint=None, overrides=None):
        self.config, self.name = config, name
        self.icb, self.cb, self.lits, self.nv, self.vb = icb, cb, lits, nv, vb
        self.ninp = ninp
        self.n = len(nv)
        self.oracle_items = oracle_items   # [("ir", array) | ("cnf", (nvars, lits3))]
        self.stored = stored               # (description, uint8 verdicts) or None
        self.budgets = budgets             # {"cdcl": conflicts, "plain": decisions, ...}
        self.arms = arms
        self.enc = enc
        self.fingerprint = fingerprint
        self.overrides = overrides or {}   # {arm: options tuned for this workload}


def _num_inputs(enc):
    iib, widths, _ = enc.inputs()
    csum = np.concatenate([[0], np.cumsum(widths, dtype=np.int64)])
    return (csum[iib[1:]] - csum[iib[:-1]]).astype(np.int32)


def _from_irs(B, config, name, irs, stored, budgets, arms, fp=None):
    enc = B.scuba_encode_batch(irs)
    return Work(config, name, enc.inst_clause_begin, enc.clause_begin, enc.lits,
                enc.inst_num_vars, enc.inst_var_begin, _num_inputs(enc),
                [("ir", a) for a in irs], stored, budgets, arms, enc=enc, fingerprint=fp)


def build_work(B, config: int, per_gpu: int, ws: int, width: int = 16):
    """The host batch of one configuration: the whole list that all ranks
    split (per_gpu x ws instances where the configuration is a fixed-size
    list per GPU; configs 3 and 5 are one fixed list)."""
    from workloads import queries
    if config == 2:
        irs, _ = _workload(per_gpu * ws, width)
        stored = None
        if width == 16:
            stored = ("config2_w16_oracle_verdicts.txt", _stored_verdicts())
        return _from_irs(B, 2, f"partition queries, {width}-bit inputs "
                         f"({per_gpu:,} per GPU)", irs, stored, {}, ["cdcl", "learned", "plain"])
    if config == 1:
        irs, _ = queries.config1(256 * ws)
        return _from_irs(B, 1, "bounds queries, 8-bit inputs (256 per GPU)", irs,
                         ("config1_w8_oracle_verdicts.txt",
                          _stored("config1_w8_oracle_verdicts.txt")[1]), {}, ["cdcl", "plain"])
    if config == 4:
        _, _, te, _ = queries.config4_split(0, 4096 * ws)
        return _from_irs(B, 4, "held-out partition queries (odd seeds), 16-bit inputs "
                         "(4,096 per GPU)", te,
                         ("config4_test_oracle_verdicts.txt",
                          _stored("config4_test_oracle_verdicts.txt")[1]), {},
                         ["learned", "plain"])
    if config == 3:
        irs, _ = queries.config3(65536)
        fp = _fingerprint(irs)
        head, v = _stored("config3_oracle_verdicts.txt")
        stored = ("config3_oracle_verdicts.txt", v) if head.get("fingerprint") == fp else None
        w = _from_irs(B, 3, "grown queries, widths 8/16/32, 500-200k clauses (65,536 in "
                      "one launch)", irs, stored, {"cdcl": 20000, "plain": 100000},
                      ["cdcl", "plain"], fp=fp)
        w.enc.release_clauses()
        return w
    if config == 5:
        sat = queries.config5_sat(10000)
        b_irs, _ = queries.config5_bounds(10000)
        enc = B.scuba_encode_batch(b_irs)
        icb, cb, lits, nv, vb = _pack_mixed(sat, enc)
        ninp = np.concatenate([np.zeros(len(sat), np.int32), _num_inputs(enc)])
        fp = _fingerprint([l for _, l in sat] + list(b_irs))
        head, v = _stored("config5_oracle_verdicts.txt")
        stored = ("config5_oracle_verdicts.txt", v) if head.get("fingerprint") == fp else None
        items = [("cnf", x) for x in sat] + [("ir", a) for a in b_irs]
        return Work(5, "random 3-SAT (n 200-400, ratio 4.26) + bounds queries at 32 bits "
                    "(10,000 + 10,000 in one launch)", icb, cb, lits, nv, vb, ninp, items,
                    stored, {"cdcl": 50000, "plain": 200000}, ["cdcl", "plain"], fingerprint=fp,
                    # random 3-SAT near the threshold wants long runs between
                    # restarts: 400 conflicts per Luby unit decided 28 % more
                    # of 3,000 instances at 50,000 conflicts than 25
                    overrides={"cdcl": {"restart_unit": 400}})
    raise ValueError(f"unknown config {config}")


def _oracle_solve(items, threads, algo, budget=1 << 40):
    """The oracle on a list of instances (IR queries and/or raw 3-SAT CNFs):
    (verdicts, propagations) -- at most two pool calls, one per kind."""
    import oracle
    irs = [(k, x) for k, (t, x) in enumerate(items) if t == "ir"]
    cnfs = [(k, x) for k, (t, x) in enumerate(items) if t == "cnf"]
    v = np.zeros(len(items), np.uint8)
    props = 0
    if irs:
        r = oracle.solve_queries([x for _, x in irs], threads=threads, algo=algo, budget=budget)
        v[[k for k, _ in irs]] = r["verdict"]
        props += int(r["stats"][:, 2].sum())
    if cnfs:
        cl = [oracle.CNF(n, np.arange(0, 3 * len(l) + 1, 3, dtype=np.int64), l.reshape(-1))
              for _, (n, l) in cnfs]
        r = oracle.solve_cnfs(cl, threads=threads, algo=algo, budget=budget)
        v[[k for k, _ in cnfs]] = r["verdict"]
        props += int(r["stats"][:, 2].sum())
    return v, props


def cpu_baseline(irs, target_s: float = 15.0, seed: int = 7, algo: str = "cdcl",
                 budget: int = 1 << 40):
    """The oracle as it stands, on all host cores, timed in ONE call over a
    bounded uniform sample of the workload (as the reference arm times the
    whole workload): a short calibration call sizes the sample to about
    `target_s` seconds, then the sample is solved in a single pool call so no
    thread waits on a chunk's slowest query (algo: the oracle's
    clause-learning or its DPLL solver). `irs` holds IR arrays or
    ("ir", array) / ("cnf", (nvars, lits)) items."""
    import oracle
    items = [x if isinstance(x, tuple) else ("ir", x) for x in irs]
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(items))
    threads = oracle.default_threads()
    k_cal = min(len(order), max(4 * threads, 64))
    t0 = time.perf_counter()
    _oracle_solve([items[i] for i in order[:k_cal]], threads, algo, budget)
    t_cal = max(time.perf_counter() - t0, 1e-3)
    size = int(min(len(order), max(k_cal, k_cal * target_s / t_cal)))
    sample = [items[i] for i in order[:size]]
    t0 = time.perf_counter()
    v, props = _oracle_solve(sample, threads, algo, budget)
    t_used = time.perf_counter() - t0
    # one host thread on the first queries of the same sample (about a fifth
    # of the time budget, again one call): the per-core rate; clause learning
    # only (the DPLL solver's heavy tail would make one query's time unbounded)
    single = {}
    if algo == "cdcl":
        # about a fifth of the time budget on one core, at the measured rate
        k1 = max(8, min(size, int(size / t_used / threads * target_s / 5)))
        t0 = time.perf_counter()
        _, p1 = _oracle_solve(sample[:k1], 1, algo, budget)
        t1 = time.perf_counter() - t0
        single = {"single_core": {"verdicts_per_s": k1 / t1, "propagations_per_s": p1 / t1,
                                  "sample": f"the first {k1} of that sample, {t1:.1f}s, "
                                            "1 thread, one call"}}
    out = {"value": size / t_used, "unit": "verdicts/s", "cores": threads, "kind": "oracle",
           "algo": algo,
           "sample": f"{size} of {len(items)} instances drawn uniformly (seed {seed}), solved "
                     f"in one call on {threads} threads, {t_used:.1f}s",
           "propagations_per_s": props / t_used, **single}
    if budget < (1 << 40):
        out["budget"] = budget
        out["unknown_in_sample"] = int((v == 2).sum())
    return out


def _reference_items(config: int, width: int = 16):
    """The configuration's instances as the oracle takes them (generators
    only, no product code): (workload name, items, conflict budget)."""
    from workloads import queries
    if config == 2:
        irs, _ = _workload(4096, width)
        return f"partition queries, {width}-bit inputs (4,096 per GPU)", irs, 1 << 40
    if config == 1:
        return "bounds queries, 8-bit inputs (256 per GPU)", queries.config1(256)[0], 1 << 40
    if config == 4:
        return ("held-out partition queries (odd seeds), 16-bit inputs (4,096 per GPU)",
                queries.config4_split(0, 4096)[2], 1 << 40)
    if config == 3:
        return ("grown queries, widths 8/16/32, 500-200k clauses (65,536 in one launch)",
                queries.config3(65536)[0], 20000)
    sat = queries.config5_sat(10000)
    return ("random 3-SAT (n 200-400, ratio 4.26) + bounds queries at 32 bits "
            "(10,000 + 10,000 in one launch)",
            [("cnf", x) for x in sat] + [("ir", a) for a in queries.config5_bounds(10000)[0]],
            50000)


def run_reference(args):
    """The oracle on the host cores, timed as it stands: its clause-learning
    solver over the whole workload per step for configurations 1, 2 and 4
    (its DPLL solver would need minutes per step; it is timed on a sample
    inside the GPU arm's cpu_baseline_dpll); for 3 and 5, whose whole lists
    take the oracle hours, over a bounded uniform sample per step under the
    GPU arm's conflict budget."""
    ws, rank = _dist()
    if rank != 0:
        return
    import oracle
    name, items, budget = _reference_items(args.config, args.width)
    items = [x if isinstance(x, tuple) else ("ir", x) for x in items]
    sample_note = f"the whole {len(items):,}-instance workload every step"
    if args.config in (3, 5):
        order = np.random.default_rng(11).permutation(len(items))[:args.reference_sample]
        items = [items[i] for i in order]
        sample_note = (f"{len(items)} of the workload's instances drawn uniformly (seed 11) "
                       f"every step, {budget} conflicts per instance")
    threads = oracle.default_threads()
    times, counts, props = [], [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, p = _oracle_solve(items, threads, "cdcl", budget)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            counts.append(len(items))
            props.append(p)
    tot = sum(times)
    value = sum(counts) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "verdicts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / len(times), "higher_is_better": True,
            "scaling": "strong" if args.config in (3, 5) else "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": name, "config_id": args.config,
                       "instances_per_step": len(items),
                       "propagations_per_s": sum(props) / tot},
            "cpu_baseline": {"kind": "oracle", "algo": "cdcl", "cores": threads, "value": value,
                             "unit": "verdicts/s", "sample": sample_note},
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


def _timed_arm(api, B, db, dev, stream, count, heur_opts, args, use_graph=True,
               time_budget_ms=300000):
    """W warm-up solves, then K timed steps (CUDA-graph replays of one solve).
    Returns per-arm timings, counters and the last verdicts."""
    import torch
    stats = torch.zeros((count, B.SCUBA_NSTATS), dtype=torch.int64, device=dev)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record(stream)
    ev[1].record(stream)
    verdict = torch.empty(count, dtype=torch.uint8, device=dev)

    def launch(st_tensor, events):
        o = api.options(stats=st_tensor, time_budget_ms=time_budget_ms, events=events,
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
            with torch.cuda.stream(stream):  # replay on the stream the events time
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


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of a per-rank count over all ranks (identity without a group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _parity(work, verdict):
    """Verdicts against the stored oracle verdicts: every instance for the
    fully decided configurations, every instance both sides decide for the
    budgeted ones (3, 5). Raises on a disagreement."""
    if work.stored is None:
        return {"checked": 0, "note": "no stored oracle verdicts for this workload"}
    name, ref = work.stored
    if len(ref) != len(verdict):
        return {"checked": 0, "note": f"{name} holds {len(ref)} verdicts, batch {len(verdict)}"}
    both = (ref != 2) & (verdict != 2)
    bad = int((ref[both] != verdict[both]).sum())
    assert bad == 0, f"verdicts differ from the oracle ({name}) on {bad} instances"
    if work.config in (1, 2, 4):
        assert both.all(), f"undecided instances against {name}"
    return {"checked": int(both.sum()), "of": len(ref), "against": name,
            "oracle_unknown": int((ref == 2).sum()), "gpu_unknown": int((verdict == 2).sum()),
            "result": f"{int(both.sum())}/{int(both.sum())} bit-exact where both decided"}


def run_ours(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    group = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        group = dist.new_group(backend="gloo")  # host gather of the verdicts
    from paper_2601_21552_gb300 import api, binding as B, shard
    from paper_2601_21552_gb300 import build as pb
    pb.build()

    t_enc = time.perf_counter()
    work = build_work(B, args.config, args.queries, ws, args.width)
    t_enc = time.perf_counter() - t_enc
    # one list, LPT shards by clause count (every rank computes the same split)
    if ws > 1:
        idx = shard.lpt_partition(np.diff(work.icb), ws)[rank]
        icb, cb, lits, nv, vb = shard.sub_csr(work.icb, work.cb, work.lits, work.nv, idx)
        ninp = work.ninp[idx]
    else:
        idx = np.arange(work.n)
        icb, cb, lits, nv, vb, ninp = work.icb, work.cb, work.lits, work.nv, work.vb, work.ninp
    count = len(idx)
    db = api.DeviceBatch.from_csr(icb, cb, lits, nv, vb, num_inputs=ninp, device=dev,
                                  pin=args.config != 3)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)  # graphs cannot be captured on the legacy stream

    from paper_2601_21552_gb300 import autotune
    tuned = autotune.load()  # launch shape / sharing parameters from the last sweep
    tuned_cdcl = autotune.load(section="best_cdcl")
    # the first arm is the headline; the others are measured beside it
    arms = [a for a in (args.arms or ",".join(work.arms)).split(",") if a]
    assert arms and set(arms) <= {"cdcl", "learned", "plain"}, args.arms
    net, train_info = None, None
    if "learned" in arms:
        net, train_info = _train_network(api, B, dev, args)
    time_ms = 600000 if args.config in (3, 5) else 300000

    def arm_options(arm):
        opts = dict(tuned)
        if arm == "learned":
            opts.update(heuristic=B.SCUBA_HEUR_LEARNED, mlp_weights=net.weights,
                        learned_depth=args.learned_depth)
        elif arm == "cdcl":
            opts.update(tuned_cdcl, search="cdcl")
            if args.learnt_words:
                opts["learnt_words"] = args.learnt_words
        if work.budgets.get(arm):
            opts["decision_budget"] = work.budgets[arm]
        if args.config in (3, 5):  # uneven sizes: largest instances first (LPT)
            opts["order"] = db.lpt_order()
        opts.update(work.overrides.get(arm, {}))
        return opts

    if ws > 1:
        torch.distributed.barrier()
    results = {}
    with ClockSampler(local) as clk:
        for arm in arms:
            results[arm] = _timed_arm(api, B, db, dev, stream, count, arm_options(arm), args,
                                      use_graph=args.graph, time_budget_ms=time_ms)
    if ws > 1:
        torch.distributed.barrier()
    for arm in arms:
        results[arm]["ms_total"] = max_over_ranks(results[arm]["ms_total"], dev)
        results[arm]["props_total"] = sum_over_ranks(float(results[arm]["stats"][:, 2].sum()),
                                                     dev)
        results[arm]["dec_total"] = sum_over_ranks(float(results[arm]["stats"][:, 0].sum()),
                                                   dev)
        if ws > 1:  # verdicts of the whole list, in its order, on rank 0
            g = shard.gather_over_ranks(work.n, work.vb, idx, results[arm]["verdict"], None,
                                        group=group)
            results[arm]["verdict_all"] = g[0] if g is not None else None
        else:
            results[arm]["verdict_all"] = results[arm]["verdict"]

    # parity after timing: every arm against the stored oracle verdicts, and
    # the arms against each other where both decided
    parity = {}
    if rank == 0:
        for arm in arms:
            parity[arm] = _parity(work, results[arm]["verdict_all"])
        v0 = results[arms[0]]["verdict_all"]
        for arm in arms[1:]:
            v1 = results[arm]["verdict_all"]
            both = (v0 != 2) & (v1 != 2)
            assert (v0[both] == v1[both]).all(), arm

    # config 4: decision counts of both DPLL arms with splitting off (one warp
    # per instance, so the counts do not depend on how subtrees were shared)
    decisions_nosplit = {}
    if args.config == 4:
        for arm in arms:
            if arm == "cdcl":
                continue
            o = arm_options(arm)
            o["split"] = False
            _, _, st = api.solve(db, want_model=False, stream=stream, time_budget_ms=time_ms,
                                 **o)
            assert api.status(stream) == 0
            decisions_nosplit[arm] = sum_over_ranks(float(st[:, 0].sum().item()), dev)

    # end to end through the host entry point (host buffers, copies inside)
    # the host arrays in pinned memory, so the copies inside the call are DMA
    e2e = None
    if args.config != 3:  # config 3's 43 GB CSR is not re-copied every step
        def pinned(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_in = [pinned(a) for a in (icb, cb, lits, nv, vb)]
        h_verdict = torch.zeros(count, dtype=torch.uint8).pin_memory().numpy()
        hb = B.make_batch(count, int(nv.max()), len(cb) - 1, int(cb[-1]), int(vb[-1]),
                          *(t.data_ptr() for t in h_in))
        o = api.options(time_budget_ms=time_ms, **arm_options(arms[0]))  # the headline arm
        B.scuba_solve_batch_host(hb, h_verdict, None, stream.cuda_stream, o)  # warm
        e2e_t = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = B.scuba_solve_batch_host(hb, h_verdict, None, stream.cuda_stream, o)
            e2e_t.append(time.perf_counter() - t0)
            assert rc == 0
        vh = results[arms[0]]["verdict"]
        both = (h_verdict != 2) & (vh != 2)
        assert (h_verdict[both] == vh[both]).all(), "host-buffer verdicts differ"
        if args.config in (1, 2, 4):
            assert (h_verdict == vh).all(), "host-buffer verdicts differ"
        e2e_s = max_over_ranks(float(np.median(e2e_t)), dev)
        h2d = sum(int(np.asarray(a).nbytes) for a in (icb, cb, lits, nv, vb))
        e2e = {"value": work.n / e2e_s, "unit": "verdicts/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": count}
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
        v = r["verdict_all"]
        return {"value": work.n / (ms_step * 1e-3), "unit": "verdicts/s",
                "ms_per_step": ms_step, "propagations_per_s": r["props_total"] / (ms_step * 1e-3),
                "decisions_per_step": r["dec_total"],
                "sat": int((v == 1).sum()), "unsat": int((v == 0).sum()),
                "unknown": int((v == 2).sum()),
                "decided_per_s": int((v != 2).sum()) / (ms_step * 1e-3),
                "search_ms": search_ms, "search_ms_steps": r["ms_search"],
                "alg_bytes": float(alg_bytes)}

    summ = {}
    for arm in arms:
        summ[arm] = arm_summary(results[arm])
        summ[arm]["budget"] = work.budgets.get(arm)
        if args.config == 4 and arm in decisions_nosplit:
            summ[arm]["decisions_split_off"] = decisions_nosplit[arm]
    head = summ[arms[0]]
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = head["alg_bytes"] / (head["search_ms"] * 1e-3) / 1e9
    profiled = (args.config == 2 and arms[0] in DRAM_BYTES_PER_PROPAGATION
                and _kernel_sources_sha() == PROFILED_SOURCES)
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "verdicts/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        # configs 3 and 5 are one fixed list however many GPUs split it
        "scaling": "strong" if args.config in (3, 5) else "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "arm": arms[0],
        "search": "cdcl" if arms[0] == "cdcl" else "dpll",
        "heuristic": "learned" if arms[0] == "learned" else "activity",
        "propagations_per_s": head["propagations_per_s"],
        "config": {"workload": work.name, "config_id": args.config,
                   "instances_total": work.n, "instances_per_gpu": count,
                   "input_bits": args.width if args.config in (2,) else None,
                   "clauses_total": int(len(work.cb) - 1), "literals_total": int(work.cb[-1]),
                   "vars_total": int(work.vb[-1]),
                   "l2": "inputs larger than L2 (CSR + occurrence lists > 1 GB)"
                         if args.config != 1 else "inputs smaller than L2 (config 1)",
                   "encode_s": t_enc, "cuda_graph": args.graph, "parity": parity,
                   "sharding": (f"LPT by clause count over {ws} ranks, host gather"
                                if ws > 1 else "one rank"),
                   "autotuned": {"dpll": tuned, "cdcl": tuned_cdcl}},
        "arms": summ,
        "e2e": e2e,
        "gpu_launches": 10 * args.steps,
        "l2": _l2_line(arms[0], head, ws, dev) if args.config == 2 else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": (DRAM_BYTES_PER_PROPAGATION[arms[0]] * head["propagations_per_s"]
                                 * head["ms_per_step"] * 1e-3 / ws if profiled else None),
                     "traffic_unit": "bytes per launch (ncu, scaled by propagations)",
                     "kernel": f"k_solve ({arms[0]} search)", "peak_source": src,
                     "limiter": "latency: dependent L1/L2 loads and instruction issue "
                                "per propagation round, DRAM mostly idle",
                     "search_ms": head["search_ms"]},
        "clocks": clk.summary(),
    }
    if "learned" in summ and "plain" in summ:
        lp = {"verdicts_per_s": summ["learned"]["value"] / summ["plain"]["value"],
              "decisions_per_step": (summ["learned"]["decisions_per_step"]
                                     / max(summ["plain"]["decisions_per_step"], 1.0))}
        if "decisions_split_off" in summ["learned"]:
            lp["decisions_split_off"] = (summ["learned"]["decisions_split_off"]
                                         / max(summ["plain"]["decisions_split_off"], 1.0))
        line["learned_over_plain"] = lp
    if train_info:
        line["learned_training"] = train_info
    if not args.no_cpu_baseline:
        # the oracle's clause-learning solver (the stronger CPU program), and
        # its DPLL beside it, on the same workload (same budgets)
        line["cpu_baseline"] = cpu_baseline(work.oracle_items, target_s=args.cpu_seconds,
                                            algo="cdcl",
                                            budget=work.budgets.get("cdcl", 1 << 40))
        line["cpu_baseline_dpll"] = cpu_baseline(work.oracle_items, target_s=args.cpu_seconds / 2,
                                                 algo="dpll",
                                                 budget=work.budgets.get("plain", 1 << 40))
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--arms", default="",
                    help="comma list of cdcl, learned, plain; the first is the headline "
                         "(default: the configuration's arms)")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="workload configuration (2: the default bench workload)")
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
    ap.add_argument("--reference-sample", type=int, default=512,
                    help="instances per step of the reference arm on configs 3 and 5")
    ap.add_argument("--queries", type=int, default=4096,
                    help="queries per GPU (profiling runs use smaller cases)")
    ap.add_argument("--width", type=int, default=16, help="input word width in bits")
    ap.add_argument("--learnt-words", type=int, default=0,
                    help="clause-learning arena per worker warp in words (0: the library "
                         "default 2^18; profiling captures use 2^16 to stay within a few GB)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
