"""Write stored oracle verdicts for the full-size synthetic workloads.

Calls only the CPU oracle (oracle/) and the seeded generators (workloads/);
nothing here touches the product library. Output: one verdict per line,
0 = UNSAT, 1 = SAT, 2 = UNKNOWN (decision budget reached), in query order.

    python tests/golden/make_oracle_verdicts.py config2
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
    else:
        raise SystemExit(f"unknown workload {which}")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "config2")
