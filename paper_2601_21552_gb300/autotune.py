"""Offline autotuner for the persistent search: launch shape and subtree
sharing parameters.

Sweeps blocks per SM, the decisions a subtree makes before it may share work
(split_min) and the decisions between checks for idle warps (split_interval)
on a workload, timing each setting as the median of several solves (the
search is nondeterministic, so single runs are noisy), and writes the best
setting to a JSON file that bench.py and api.solve(..., tuned=True) read.

    python -m paper_2601_21552_gb300.autotune [--queries 4096] [--width 16]
           [--reps 3] [--search dpll|cdcl]
           [--out paper_2601_21552_gb300/autotune.json]

The DPLL sweep writes "best"; the clause-learning sweep (cube-sharing
thresholds and restart unit) writes "best_cdcl".
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
# clause learning: decisions before a job may give away cubes, decisions
# between checks for idle warps, conflicts per Luby restart unit
SPACE_CDCL = {
    "split_min": [4, 8, 16, 32],
    "split_interval": [8, 16, 32],
    "restart_unit": [12, 25, 40],
}


def load(path: str = DEFAULT_OUT, section: str = "best") -> dict:
    """Best options found by a previous sweep ("best": the DPLL search,
    "best_cdcl": the clause-learning search), or {} when none was run."""
    try:
        with open(path) as f:
            return dict(json.load(f).get(section, {}))
    except (OSError, ValueError):
        return {}


def sweep(db, reps: int = 3, space: dict | None = None, time_budget_ms: int = 120000,
          fixed: dict | None = None):
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
            api.solve(db, want_model=False, stats=False, time_budget_ms=time_budget_ms,
                      **opts, **(fixed or {}))
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
    ap.add_argument("--search", default="dpll", choices=["dpll", "cdcl"])
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(HERE))
    import torch

    from . import api, binding as B
    from workloads import queries
    irs, _ = queries.config2(args.queries, w=args.width)
    enc = B.scuba_encode_batch(irs)
    db = api.DeviceBatch(enc, "cuda")
    torch.cuda.synchronize()
    if args.search == "cdcl":
        best, trials = sweep(db, reps=args.reps, space=SPACE_CDCL, fixed={"search": "cdcl"})
    else:
        best, trials = sweep(db, reps=args.reps)
    try:  # the other search's section stays as it was
        with open(args.out) as f:
            out = json.load(f)
    except (OSError, ValueError):
        out = {}
    sfx = "_cdcl" if args.search == "cdcl" else ""
    out.update({"workload": f"partition queries, {args.width}-bit inputs, {args.queries} queries",
                "device": torch.cuda.get_device_name(0), "reps": args.reps,
                "best" + sfx: best["options"], "best_median_s" + sfx: best["median_s"],
                "trials" + sfx: trials})
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print("best", json.dumps(best))


if __name__ == "__main__":
    main()
