"""Host-side logic on the CPU, no GPU calls. The autotuner's selection with a
fake solve: the setting with the lowest MEAN time wins even when another has
the lower median (the rare slow solves of the nondeterministic search are
what the mean sees), failed solves count as infinite time and their statuses
are recorded. The unit wrapper refuses assumption offsets that the kernels
would follow past the end of the assumption literals."""
import pytest

torch = pytest.importorskip("torch")


def test_sweep_picks_lowest_mean(monkeypatch):
    from paper_2601_21552_gb300 import api, autotune
    # per setting: a sequence of (seconds, status) for successive solves
    plan = {4: [(0.10, 0), (0.10, 0), (0.10, 0), (1.00, 0)],   # low median, a tail
            48: [(0.14, 0), (0.15, 0), (0.14, 0), (0.15, 0)],  # steady
            64: [(0.12, 0), (0.12, 0), (0.12, 0), (0.12, -4)]}  # one timeout
    state = {"t": 0.0, "status": 0}
    calls = {k: 0 for k in plan}

    def fake_solve(db, want_model=False, stats=False, time_budget_ms=0, **opts):
        k = opts["split_min"]
        dt, st = plan[k][calls[k]]
        calls[k] += 1
        state["t"] += dt
        state["status"] = st

    monkeypatch.setattr(api, "solve", fake_solve)
    monkeypatch.setattr(api, "status", lambda *a: state["status"])
    monkeypatch.setattr(autotune.time, "perf_counter", lambda: state["t"])
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    best, trials = autotune.sweep(None, reps=4, space={"split_min": [4, 48, 64]},
                                  fixed={"search": "cdcl"})
    assert best["options"] == {"split_min": 48}
    by = {t["options"]["split_min"]: t for t in trials}
    assert by[4]["median_s"] < by[48]["median_s"] < by[4]["mean_s"]
    assert by[64]["mean_s"] == float("inf") and by[64]["failed_status"] == [-4]
    assert "failed_status" not in by[48]


def test_load_sections(tmp_path):
    from paper_2601_21552_gb300 import autotune
    p = tmp_path / "t.json"
    p.write_text('{"best": {"blocks_per_sm": 5}, "best_cdcl": {"split_min": 48}}')
    assert autotune.load(str(p)) == {"blocks_per_sm": 5}
    assert autotune.load(str(p), section="best_cdcl") == {"split_min": 48}
    assert autotune.load(str(tmp_path / "missing.json")) == {}
    # the committed file holds both sections
    assert autotune.load(section="best_cdcl").get("split_min", 0) > 0


@pytest.mark.parametrize("begin,lits", [
    ([0, 1], [5, 6]),          # n_units + 1 offsets needed (3 units)
    ([0, 2, 1, 2], [5, 6]),    # decreasing
    ([0, 1, 2, 3], [5, 6]),    # past the end of asm_lits
    ([-1, 0, 1, 2], [5, 6]),   # negative
])
def test_solve_units_rejects_bad_offsets_on_the_host(begin, lits):
    """Offsets the kernels would follow past asm_lits are refused before any
    device work (the library cannot know asm_lits' length)."""
    import types

    import numpy as np

    from paper_2601_21552_gb300 import api
    db = types.SimpleNamespace(icb=torch.zeros(1), n=1,
                               enc=types.SimpleNamespace(inst_num_vars=np.array([3], np.int32)))
    with pytest.raises(ValueError):
        api.solve_units(db, [0, 0, 0], np.array(begin, np.int64), np.array(lits, np.int32))


def test_pick_prefers_steady_setting_within_five_percent():
    from paper_2601_21552_gb300 import autotune
    trials = [{"options": {"a": 1}, "mean_s": 1.00, "median_s": 0.7, "times": [0.7, 0.7, 1.6]},
              {"options": {"a": 2}, "mean_s": 1.04, "median_s": 1.05, "times": [1.0, 1.05, 1.07]},
              {"options": {"a": 3}, "mean_s": 1.20, "median_s": 1.2, "times": [1.2, 1.2, 1.2]}]
    assert autotune.pick(trials)["options"] == {"a": 2}   # the lowest mean has a tail
    trials[1]["mean_s"] = 1.06  # outside 5 %: the lowest mean wins again
    assert autotune.pick(trials)["options"] == {"a": 1}
    trials[0]["times"] = [0.9, 1.0, 1.1]
    trials[0]["median_s"] = 1.0
    trials[1]["mean_s"] = 1.01  # both steady: the lower mean
    assert autotune.pick(trials)["options"] == {"a": 1}
