"""The benchmark's CPU-side pieces: the reference arm (the oracle timed on
the host cores) prints one JSON line with the keys the bench contract asks
for, and the CPU baseline reports its cores, sample and rates. No GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "workload" in d["config"]


def test_cpu_baseline_fields():
    sys.path.insert(0, ROOT)
    import bench
    irs, _ = bench._workload(64, width=8)
    c = bench.cpu_baseline(irs, target_s=0.5)
    assert c["kind"] == "oracle" and c["algo"] == "cdcl" and c["cores"] >= 1
    assert c["value"] > 0 and c["propagations_per_s"] > 0 and "sample" in c
    assert c["single_core"]["verdicts_per_s"] > 0
    d = bench.cpu_baseline(irs, target_s=0.5, algo="dpll")
    assert d["algo"] == "dpll" and "single_core" not in d


def test_cpu_baseline_times_the_sample_in_one_pool_call(monkeypatch):
    """The sample is solved by one call on every host thread (a chunked loop
    would make each chunk wait for its slowest query and understate the
    oracle), and the reported rate is that call's."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    calls = []
    real = oracle.solve_queries

    def spy(irs, threads=None, **kw):
        calls.append((len(irs), threads))
        return real(irs, threads=threads, **kw)

    monkeypatch.setattr(oracle, "solve_queries", spy)
    irs, _ = bench._workload(200, width=8)
    c = bench.cpu_baseline(irs, target_s=0.2, algo="dpll")
    threads = oracle.default_threads()
    assert len(calls) == 2  # calibration, then the timed sample
    assert all(t == threads for _, t in calls)
    size = int(c["sample"].split()[0])
    assert calls[1][0] == size and size >= calls[0][0]


def test_reference_arm_other_configs():
    """The reference arm follows --config: config 1's whole list per step,
    config 5 a bounded sample per step under the GPU arm's conflict budget."""
    for cfg, extra in (("1", []), ("5", ["--reference-sample", "4"])):
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", cfg,
                            "--steps", "1", "--warmup", "0"] + extra, cwd=ROOT,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
        assert d["impl"] == "reference" and d["config"]["config_id"] == int(cfg)
        assert d["value"] > 0
        if cfg == "1":
            assert d["config"]["instances_per_step"] == 256 and d["scaling"] == "weak"
        else:
            assert d["config"]["instances_per_step"] == 4 and d["scaling"] == "strong"


def test_parity_rules_and_workloads():
    """The bench's parity check: every instance must match the stored oracle
    verdicts on the fully decided configurations; on the budgeted ones (3, 5)
    every instance both sides decide must match and UNKNOWN is allowed; a
    disagreement always raises. The host workloads carry the stored verdicts
    that belong to them."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import pytest
    import bench
    from paper_2601_21552_gb300 import binding as B

    w1 = bench.build_work(B, 1, 256, 1)
    assert w1.n == 256 and len(w1.stored[1]) == 256 and set(w1.arms) == {"cdcl", "plain"}
    ref = w1.stored[1].copy()
    assert bench._parity(w1, ref.copy())["checked"] == 256
    unk = ref.copy()
    unk[3] = 2
    with pytest.raises(AssertionError):          # config 1 must be fully decided
        bench._parity(w1, unk)
    bad = ref.copy()
    bad[5] ^= 1
    with pytest.raises(AssertionError):
        bench._parity(w1, bad)

    class Budgeted:
        config = 5
        stored = ("x", np.array([0, 1, 2, 1, 2], np.uint8))
    r = bench._parity(Budgeted, np.array([0, 2, 1, 1, 2], np.uint8))
    assert r["checked"] == 2 and r["oracle_unknown"] == 2 and r["gpu_unknown"] == 2
    with pytest.raises(AssertionError):
        bench._parity(Budgeted, np.array([1, 2, 2, 1, 2], np.uint8))
    w2 = bench.build_work(B, 2, 64, 2, width=8)   # two ranks' worth of one list
    assert w2.n == 128 and w2.stored is None and len(w2.ninp) == 128
