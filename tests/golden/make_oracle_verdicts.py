"""Write stored oracle verdicts for the full-size synthetic workloads.

Calls only the CPU oracle (oracle/) and the seeded generators (workloads/);
nothing here touches the product library. Output: one verdict per line,
0 = UNSAT, 1 = SAT, 2 = UNKNOWN (decision budget reached), in query order.

    python tests/golden/make_oracle_verdicts.py config2
    python tests/golden/make_oracle_verdicts.py config1
    python tests/golden/make_oracle_verdicts.py config4

config1: the 256 bounds queries at 8 bits (oracle DPLL, no budget);
config4: the 4,096 odd-seed held-out partition queries at 16 bits of the
learned-branching configuration (oracle clause learning, no budget). Both
files start with `#` provenance lines.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import queries  # noqa: E402


def write(name, verdicts):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(str(int(v)) for v in verdicts) + "\n")


def main(which):
    t0 = time.time()
    if which == "config2":
        irs, _ = queries.config2(4096)
        r = oracle.solve_queries(irs)
        write("config2_w16_oracle_verdicts.txt", r["verdict"])
        st = r["stats"]
        print(f"config2: {len(irs)} queries in {time.time() - t0:.1f}s on "
              f"{oracle.default_threads()} threads; decisions max {st[:, 0].max()}, "
              f"propagations total {st[:, 2].sum()}")
    elif which in ("config1", "config4"):
        if which == "config1":
            irs, _ = queries.config1(256)
            name, algo = "config1_w8_oracle_verdicts.txt", "dpll"
        else:
            irs = queries.config4_split(0, 4096)[2]
            name, algo = "config4_test_oracle_verdicts.txt", "cdcl"
        r = oracle.solve_queries(irs, algo=algo)
        v = r["verdict"]
        assert (v != 2).all()
        with open(os.path.join(HERE, name), "w") as f:
            f.write(f"# workload: {which}, {len(irs)} queries\n# algorithm: oracle {algo}, "
                    f"no budget\n# sat: {int((v == 1).sum())}\n# unsat: {int((v == 0).sum())}\n"
                    f"# written by: python tests/golden/make_oracle_verdicts.py {which}\n")
            f.write("\n".join(str(int(x)) for x in v) + "\n")
        print(f"{which}: {len(irs)} queries in {time.time() - t0:.1f}s")
    else:
        raise SystemExit(f"unknown workload {which}")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "config2")
