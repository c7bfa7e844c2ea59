"""Cache the oracle's verdicts for the two large workloads, every instance.

Calls only the CPU oracle (oracle/) and the seeded generators (workloads/);
nothing here touches the product library. The oracle's clause-learning
solver decides every instance under a stated per-instance conflict budget,
sharded over the host cores; an instance it does not decide within the
budget is stored as UNKNOWN (2), never guessed.

    python tests/golden/make_config_cache.py config3 [--budget 20000] [--threads N]
    python tests/golden/make_config_cache.py config5 [--budget 20000] [--threads N]
    python tests/golden/make_config_cache.py config5 --escalate 100000 --max-vars 300

Workloads (the generators' own definitions, seeds SEED_BASE[c] + i):
  config3  65,536 grown queries, widths 8/16/32, clause targets log-uniform
           in [500, 200k]
  config5  10,000 uniform random 3-SAT instances (n in [200, 400], ratio
           4.26) followed by 10,000 bounds queries at 32 bits

Output file: `#` header lines (workload, count, budget, algorithm, host
threads, wall time, and a SHA-256 fingerprint of the generated instances,
so a test can tell whether the generator still produces the same inputs),
then the verdicts in instance order, 64 digits per line: 0 UNSAT, 1 SAT,
2 UNKNOWN. Work is done in chunks and appended to `<output>.partial`, so an
interrupted run resumes where it stopped.
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import queries  # noqa: E402

FILES = {"config3": "config3_oracle_verdicts.txt", "config5": "config5_oracle_verdicts.txt"}


def fingerprint(arrays) -> str:
    """SHA-256 (first 16 hex digits) of the instances as int64 arrays, in order."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype=np.int64).tobytes())
    return h.hexdigest()[:16]


def instances(which):
    """(fingerprint, count, solve(i0, i1, budget, threads) -> (verdicts, conflicts))."""
    if which == "config3":
        irs, _ = queries.config3(65536)

        def solve(i0, i1, budget, threads):
            r = oracle.solve_queries(irs[i0:i1], threads=threads, budget=budget, algo="cdcl")
            return r["verdict"], r["stats"][:, 1]
        return fingerprint(irs), len(irs), solve
    if which == "config5":
        sat = queries.config5_sat(10000)
        b_irs, _ = queries.config5_bounds(10000)
        cnfs = [oracle.CNF(n, np.arange(0, 3 * len(l) + 1, 3, dtype=np.int64), l.reshape(-1))
                for n, l in sat]
        fp = fingerprint([l for _, l in sat] + list(b_irs))

        def solve(i0, i1, budget, threads):
            v, c = [], []
            a, b = i0, min(i1, len(cnfs))
            if a < b:
                r = oracle.solve_cnfs(cnfs[a:b], threads=threads, budget=budget, algo="cdcl")
                v.append(r["verdict"])
                c.append(r["stats"][:, 1])
            a, b = max(i0, len(cnfs)), i1
            if a < b:
                r = oracle.solve_queries(b_irs[a - len(cnfs):b - len(cnfs)], threads=threads,
                                         budget=budget, algo="cdcl")
                v.append(r["verdict"])
                c.append(r["stats"][:, 1])
            return np.concatenate(v), np.concatenate(c)
        return fp, len(cnfs) + len(b_irs), solve
    raise SystemExit(f"unknown workload {which}")


def read_cache(path):
    """(header dict, verdicts uint8 array) of a cache file."""
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


def escalate(which, budget, max_vars, threads, chunk=256):
    """Re-solve, at a larger conflict budget, the random 3-SAT instances of
    the config-5 cache that the first pass left UNKNOWN and that have at most
    `max_vars` variables (chosen by size alone), and rewrite the cache with
    their new verdicts and a header line recording the pass. Progress goes to
    `<output>.escalate.partial`, so an interrupted pass resumes."""
    if which != "config5":
        raise SystemExit("escalation is defined for config5 only")
    out = os.path.join(HERE, FILES[which])
    head, v = read_cache(out)
    fp, count, _ = instances(which)
    if head.get("fingerprint") != fp:
        raise SystemExit("the cache belongs to other instances")
    sat = queries.config5_sat(10000)
    todo = [i for i in range(len(sat)) if v[i] == 2 and sat[i][0] <= max_vars]
    part = out + ".escalate.partial"
    got = {}
    key = f"{fp} {budget} {max_vars}"
    if os.path.exists(part):
        with open(part) as f:
            if f.readline().strip() == key:
                for line in f:
                    i, x = line.split()
                    got[int(i)] = int(x)
    else:
        with open(part, "w") as f:
            f.write(key + "\n")
    rest = [i for i in todo if i not in got]
    t0 = time.time()
    with open(part, "a") as f:
        for k in range(0, len(rest), chunk):
            sel = rest[k:k + chunk]
            cnfs = [oracle.CNF(sat[i][0], np.arange(0, 3 * len(sat[i][1]) + 1, 3, dtype=np.int64),
                               sat[i][1].reshape(-1)) for i in sel]
            r = oracle.solve_cnfs(cnfs, threads=threads, budget=budget, algo="cdcl")
            for i, x in zip(sel, r["verdict"]):
                got[i] = int(x)
                f.write(f"{i} {int(x)}\n")
            f.flush()
            print(f"{which} escalation: {len(got)}/{len(todo)} ({time.time() - t0:.0f}s)",
                  flush=True)
    v = v.copy()
    for i, x in got.items():
        v[i] = x
    decided = sum(1 for x in got.values() if x != 2)
    lines = open(out).read().splitlines()
    header = [l for l in lines if l.startswith("#") and not l.startswith(("# sat:", "# unsat:",
                                                                           "# unknown:"))]
    header += [f"# escalated: the {len(todo)} UNKNOWN random 3-SAT instances with at most "
               f"{max_vars} variables re-solved at {budget} conflicts, {decided} decided",
               f"# sat: {int((v == 1).sum())}", f"# unsat: {int((v == 0).sum())}",
               f"# unknown: {int((v == 2).sum())}"]
    digits = "".join(str(int(x)) for x in v)
    with open(out, "w") as f:
        f.write("\n".join(header) + "\n")
        for k in range(0, count, 64):
            f.write(digits[k:k + 64] + "\n")
    os.remove(part)
    print(f"{which}: escalated {len(todo)}, decided {decided}; UNKNOWN now {int((v == 2).sum())}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=sorted(FILES))
    ap.add_argument("--budget", type=int, default=20000, help="conflicts per instance")
    ap.add_argument("--threads", type=int, default=0, help="0: all host cores")
    ap.add_argument("--chunk", type=int, default=2048)
    ap.add_argument("--escalate", type=int, default=0,
                    help="config5: re-solve the cache's UNKNOWN random 3-SAT instances with "
                         "at most --max-vars variables at this conflict budget")
    ap.add_argument("--max-vars", type=int, default=300)
    args = ap.parse_args()
    threads = args.threads or oracle.default_threads()
    if args.escalate:
        escalate(args.which, args.escalate, args.max_vars, threads)
        return
    fp, count, solve = instances(args.which)
    out = os.path.join(HERE, FILES[args.which])
    part = out + ".partial"
    done = []
    t_prev = 0.0
    if os.path.exists(part):
        with open(part) as f:
            first = f.readline().split()
            if first == [fp, str(args.budget)]:
                for line in f:
                    if line.startswith("t "):
                        t_prev = float(line.split()[1])
                    elif line.strip():
                        done.append(line.strip())
    else:
        with open(part, "w") as f:
            f.write(f"{fp} {args.budget}\n")
    verdicts = "".join(done)
    t0 = time.time()
    conflicts_hi = 0
    with open(part, "a") as f:
        for i0 in range(len(verdicts), count, args.chunk):
            i1 = min(count, i0 + args.chunk)
            v, c = solve(i0, i1, args.budget, threads)
            s = "".join(str(int(x)) for x in v)
            verdicts += s
            conflicts_hi += int((c >= args.budget).sum())
            f.write(s + "\n")
            f.write(f"t {t_prev + time.time() - t0:.1f}\n")
            f.flush()
            print(f"{args.which}: {i1}/{count} ({time.time() - t0:.0f}s)", flush=True)
    wall = t_prev + time.time() - t0
    a = np.frombuffer(verdicts.encode(), dtype=np.uint8) - ord("0")
    with open(out, "w") as f:
        f.write(f"# workload: {args.which}\n# count: {count}\n# fingerprint: {fp}\n"
                f"# algorithm: oracle cdcl (first-UIP clause learning)\n"
                f"# budget: {args.budget} conflicts per instance\n"
                f"# threads: {threads}\n# wall_s: {wall:.0f}\n"
                f"# sat: {int((a == 1).sum())}\n# unsat: {int((a == 0).sum())}\n"
                f"# unknown: {int((a == 2).sum())}\n"
                f"# written by: python tests/golden/make_config_cache.py {args.which} "
                f"--budget {args.budget}\n")
        for k in range(0, count, 64):
            f.write(verdicts[k:k + 64] + "\n")
    os.remove(part)
    print(f"{args.which}: SAT {(a == 1).sum()} UNSAT {(a == 0).sum()} UNKNOWN {(a == 2).sum()} "
          f"in {wall:.0f}s on {threads} threads -> {out}")


if __name__ == "__main__":
    main()
