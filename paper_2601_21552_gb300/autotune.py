"""Offline autotuner for the persistent search: launch shape and subtree
sharing parameters.

Sweeps blocks per SM, the decisions a subtree makes before it may share work
(split_min) and the decisions between checks for idle warps (split_interval)
on a workload, timing each setting as the median of several solves (the
search is nondeterministic, so single runs are noisy), and writes the best
setting to a JSON file that bench.py and api.solve(..., tuned=True) read.

    python -m paper_2601_21552_gb300.autotune [--queries 4096] [--width 16]
           [--reps 3] [--out paper_2601_21552_gb300/autotune.json]
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "autotune.json")
SPACE = {
    "blocks_per_sm": [4, 5],
    "split_min": [128, 256, 1024],
    "split_interval": [8, 16, 64],
}


def load(path: str = DEFAULT_OUT) -> dict:
    """Best options found by a previous sweep, or {} when none was run."""
    try:
        with open(path) as f:
            return dict(json.load(f).get("best", {}))
    except (OSError, ValueError):
        return {}


def sweep(db, reps: int = 3, space: dict | None = None, time_budget_ms: int = 120000):
    import numpy as np
    import torch

    from . import api
    space = space or SPACE
    keys = list(space)
    trials = []
    for combo in itertools.product(*(space[k] for k in keys)):
        opts = dict(zip(keys, combo))
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.solve(db, want_model=False, stats=False, time_budget_ms=time_budget_ms, **opts)
            rc = api.status()
            times.append(time.perf_counter() - t0 if rc == 0 else float("inf"))
        trials.append({"options": opts, "median_s": float(np.median(times)), "times": times})
        print(json.dumps(trials[-1]), flush=True)
    best = min(trials, key=lambda t: t["median_s"])
    return best, trials


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--queries", type=int, default=4096)
    ap.add_argument("--width", type=int, default=16)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(HERE))
    import torch

    from . import api, binding as B
    from workloads import queries
    irs, _ = queries.config2(args.queries, w=args.width)
    enc = B.scuba_encode_batch(irs)
    db = api.DeviceBatch(enc, "cuda")
    torch.cuda.synchronize()
    best, trials = sweep(db, reps=args.reps)
    out = {"workload": f"partition queries, {args.width}-bit inputs, {args.queries} queries",
           "device": torch.cuda.get_device_name(0), "reps": args.reps,
           "best": best["options"], "best_median_s": best["median_s"], "trials": trials}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print("best", json.dumps(best))


if __name__ == "__main__":
    main()
