"""The checked build on the GPU (libscuba_checked.so, compiled with
-DSCUBA_CHECKED): every kernel index into an instance's buffers -- trail,
decision stack, assignment, occurrence offsets and entries, learned-clause
pool, arena and construction buffer -- is tested against its bound, and a
failed test would end the call with SCUBA_ERR_INTERNAL and a message naming
the site, never with an access out of bounds. On small well-formed inputs
the checked build must report no failure and give the oracle's verdicts
under both searches, and the propagation entry point the CPU closure.

Runs in a child process (the binding picks its library at import, from
SCUBA_LIBRARY=checked)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
from paper_2601_21552_gb300 import api, binding as B
assert B.LIB_PATH.endswith("libscuba_checked.so"), B.LIB_PATH
import oracle
from workloads import queries
from raw_cnf import model_ok, solve_raw
out = {}
cases = {"config1": queries.config1(256)[0], "config2_w10": queries.config2(256, w=10)[0]}
for name, irs in cases.items():
    for search in ("dpll", "cdcl"):
        res = api.solve_queries(irs, search=search, time_budget_ms=30000)
        ref = oracle.solve_queries(irs, algo=search)["verdict"]
        out[name + "_" + search] = {"status": int(res["status"]), "msg": B.last_error(),
                                    "same": bool((res["verdict"] == ref).all()),
                                    "fails": int(res["fails"])}
# random 3-SAT, raw CNFs (long and short clauses through the same kernels)
inst = []
for s in range(64):
    n, l = queries.random_3sat(7700 + s, 40, 80)
    inst.append((n, [list(map(int, c)) for c in l]))
for search in ("dpll", "cdcl"):
    st, v, m, vb, _ = solve_raw(api, inst, search=search, time_budget_ms=30000)
    ok = all(model_ok(inst[i][1], m, vb[i]) for i in range(len(inst)) if v[i] == 1)
    out["3sat_" + search] = {"status": int(st), "msg": B.last_error(), "models_ok": bool(ok),
                             "verdicts": [int(x) for x in v]}
print("RESULT " + json.dumps(out))
'''


def test_checked_build_clean_on_well_formed_inputs():
    from paper_2601_21552_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, SCUBA_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    for name, d in out.items():
        assert d["status"] == 0, (name, d["msg"])
        if "same" in d:
            assert d["same"] and d["fails"] == 0, (name, d)
        else:
            assert d["models_ok"], name
    assert out["3sat_dpll"]["verdicts"] == out["3sat_cdcl"]["verdicts"]
