"""Offline autotuner for the persistent search: launch shape and subtree
sharing parameters.

Sweeps blocks per SM, the decisions a subtree makes before it may share work
(split_min) and the decisions between checks for idle warps (split_interval)
on a workload, timing each setting over several solves, and writes the
setting with the lowest MEAN time (a steady setting within 5 % of it wins
over one whose slowest solve took more than 1.5x its median) to a JSON file
that bench.py and
api.solve(..., tuned=True) read. The search is nondeterministic: a few runs
in ten can take several times the median (a hard instance's cube tree grows
much deeper in them), so the mean -- what a sequence of solves costs -- is
the objective, over enough repetitions to see those runs.

    python -m paper_2601_21552_gb300.autotune [--queries 4096] [--width 16]
           [--reps N] [--search dpll|cdcl]
           [--out paper_2601_21552_gb300/autotune.json]

The DPLL sweep writes "best"; the clause-learning sweep (cube-sharing
thresholds and depth) writes "best_cdcl".
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
# clause learning: decisions before a job may give away cubes and the
# deepest cube level that may split further (248: the prefix capacity, no
# cap); the decisions between checks for idle warps (16) and the conflicts per
# Luby restart unit (25) come from a wider sweep over {8, 16, 32} x
# {12, 25, 40}, and smaller split_min (4-16) and caps (10-18) lost to these
# on the mean; share_lbd is the LBD bound of the clauses the jobs of one
# instance share (-1: no sharing); a gate on the job's own conflicts before
# it may give cubes away (8-128) was measured no better than none
SPACE_CDCL = {
    "split_min": [32, 48, 64],
    "split_depth": [248],
    "split_interval": [16],
    "restart_unit": [25],
    "share_lbd": [-1, 2, 4, 8],
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
        times, failed = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.solve(db, want_model=False, stats=False, time_budget_ms=time_budget_ms,
                      **opts, **(fixed or {}))
            rc = api.status()
            times.append(time.perf_counter() - t0 if rc == 0 else float("inf"))
            if rc != 0:
                failed.append(rc)  # e.g. the time budget reached
        trials.append({"options": opts, "mean_s": float(np.mean(times)),
                       "median_s": float(np.median(times)), "times": times})
        if failed:
            trials[-1]["failed_status"] = failed
        print(json.dumps(trials[-1]), flush=True)
    return pick(trials), trials


def pick(trials, within: float = 0.05, tail: float = 1.5):
    """The trial with the lowest mean time, unless its slowest solve took more
    than `tail` times its median (a setting prone to the rare several-times-
    slower solve) and a steady trial lies within `within` of that mean: then
    the steady trial with the lowest mean."""
    best = min(trials, key=lambda t: t["mean_s"])
    steady = [t for t in trials if t["mean_s"] <= best["mean_s"] * (1.0 + within)
              and max(t["times"]) <= tail * t["median_s"]]
    return min(steady, key=lambda t: t["mean_s"]) if steady else best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--queries", type=int, default=4096)
    ap.add_argument("--width", type=int, default=16)
    ap.add_argument("--reps", type=int, default=0, help="solves per setting (0: 3 for "
                    "DPLL, 16 for clause learning)")
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--search", default="dpll", choices=["dpll", "cdcl"])
    ap.add_argument("--space", default="", help="JSON dict replacing the sweep space, "
                    "e.g. '{\"split_min\": [8, 16], \"split_depth\": [12, 14]}'")
    args = ap.parse_args()
    args.reps = args.reps or (16 if args.search == "cdcl" else 3)
    sys.path.insert(0, os.path.dirname(HERE))
    import torch

    from . import api, binding as B
    from workloads import queries
    irs, _ = queries.config2(args.queries, w=args.width)
    enc = B.scuba_encode_batch(irs)
    db = api.DeviceBatch(enc, "cuda")
    torch.cuda.synchronize()
    space = json.loads(args.space) if args.space else None
    if args.search == "cdcl":
        best, trials = sweep(db, reps=args.reps, space=space or SPACE_CDCL,
                             fixed={"search": "cdcl"})
    else:
        best, trials = sweep(db, reps=args.reps, space=space)
    try:  # the other search's section stays as it was
        with open(args.out) as f:
            out = json.load(f)
    except (OSError, ValueError):
        out = {}
    sfx = "_cdcl" if args.search == "cdcl" else ""
    out.update({"workload": f"partition queries, {args.width}-bit inputs, {args.queries} queries",
                "device": torch.cuda.get_device_name(0), "reps" + sfx: args.reps,
                "best" + sfx: best["options"], "best_mean_s" + sfx: best["mean_s"],
                "best_median_s" + sfx: best["median_s"], "trials" + sfx: trials})
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print("best", json.dumps(best))


if __name__ == "__main__":
    main()
