"""The JSON-lines run record (paper_2206_00366_gb300.runlog) on the host,
driven by a stand-in solver whose checks are known: lines and file agree,
the mass drift and throughput follow from the check sums and the clock,
and the run stops at its step count, below a residual, or at a stability
flag."""
import json
import types

import numpy as np
import pytest

from paper_2206_00366_gb300 import runlog


class FakeSolver:
    """step(n) advances a counter; the check every k steps reports mass
    1000 (1 + 1e-15 step), momentum (step, 0, 0), kinetic energy 1/step,
    residual 2^-c at its c-th check (-1 at the first), and `flags` once
    the counter reaches `flag_at`."""

    def __init__(self, k, N=200, start=0, flag_at=None, flags=4):
        self.params = types.SimpleNamespace(check_every=k)
        self.N, self.k, self.t, self.flag_at, self.flags = N, k, start, flag_at, flags
        self.checks = []

    def step(self, n):
        for _ in range(n):
            self.t += 1
            if self.k and self.t % self.k == 0:
                c = len(self.checks)
                flags = self.flags if self.flag_at is not None and self.t >= self.flag_at else 0
                self.checks.append([1000.0 * (1 + 1e-15 * self.t), float(self.t), 0.0, 0.0, 1.0 / self.t,
                                    -1.0 if c == 0 else 2.0 ** -c, float(self.t), float(flags)])

    def stats(self, allow_unstable=False):
        assert allow_unstable
        return np.array([0, 0, 0, 0, 0, -1, float(self.t), 0.0])

    def last_check(self, allow_unstable=False):
        assert allow_unstable
        return np.array(self.checks[-1]) if self.checks else np.array([0, 0, 0, 0, 0, -1, -1, 0.0])


def ticking_clock(dt):
    t = [0.0]

    def clock():
        t[0] += dt
        return t[0]
    return clock


def test_lines_file_and_figures(tmp_path):
    s = FakeSolver(10)
    path = tmp_path / "run.jsonl"
    recs = runlog.run_logged(s, 35, path=str(path), config={"workload": "stand-in"}, clock=ticking_clock(0.5))
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines == json.loads(json.dumps(recs))
    assert recs[0] == {"event": "config", "workload": "stand-in", "nodes": 200, "check_every": 10}
    checks = recs[1:-1]
    assert [c["step"] for c in checks] == [10, 20, 30, 40]          # the first check past 35 steps ends the run
    assert checks[0]["residual"] is None and checks[2]["residual"] == 0.25
    assert checks[0]["mass_drift"] == 0.0
    np.testing.assert_allclose([c["mass_drift"] for c in checks[1:]], [1e-14, 2e-14, 3e-14], rtol=1e-3)
    assert [c["momentum"][0] for c in checks] == [10.0, 20.0, 30.0, 40.0]
    for c in checks:                                                 # each line: 10 steps of 200 nodes in 0.5 s
        assert c["steps"] == 10 and c["wall_s"] == pytest.approx(0.5)
        assert c["mlups"] == pytest.approx(200 * 10 / 0.5 / 1e6)
        assert c["flags"] == 0 and "flag_names" not in c
    assert recs[-1] == {"event": "end", "steps": 40, "checks": 4, "stopped": "steps",
                        "wall_s": pytest.approx(2.0), "mlups": pytest.approx(200 * 40 / 2.0 / 1e6)}


def test_appends_to_an_existing_file(tmp_path):
    path = tmp_path / "run.jsonl"
    runlog.run_logged(FakeSolver(5), 5, path=str(path))
    runlog.run_logged(FakeSolver(5), 10, path=str(path))
    events = [json.loads(x)["event"] for x in path.read_text().splitlines()]
    assert events == ["config", "check", "end", "config", "check", "check", "end"]


def test_stops_below_the_residual():
    recs = runlog.run_logged(FakeSolver(10), 1000, stop_below=0.1)
    assert recs[-1]["stopped"] == "residual"
    assert [c["residual"] for c in recs[1:-1]] == [None, 0.5, 0.25, 0.125, 0.0625]
    assert recs[-1]["steps"] == 50 and recs[-1]["checks"] == 5


def test_stops_at_a_stability_flag():
    recs = runlog.run_logged(FakeSolver(10, flag_at=30, flags=1 | 4), 1000)
    assert recs[-1]["stopped"] == "unstable" and recs[-1]["steps"] == 30
    assert recs[-2]["flags"] == 5 and recs[-2]["flag_names"] == ["nan_or_inf", "speed_at_or_above_cs"]
    assert runlog.flag_names(8) == ["e3m12_saturated"] and runlog.flag_names(2) == ["density_not_positive"]


def test_zero_steps_and_invalid_use():
    recs = runlog.run_logged(FakeSolver(10), 0)
    assert [r["event"] for r in recs] == ["config", "end"] and recs[-1]["mlups"] is None
    with pytest.raises(ValueError):
        runlog.run_logged(FakeSolver(0), 10)                        # no periodic check
    with pytest.raises(ValueError):
        runlog.run_logged(FakeSolver(10), -1)
    s = FakeSolver(10, start=3)
    with pytest.raises(ValueError):
        runlog.run_logged(s, 30)                                    # counter not at a multiple of k
    assert s.t == 3                                                 # refused before any step
    recs = runlog.run_logged(FakeSolver(10, start=20), 20)          # a multiple of k: checks at 30 and 40
    assert [c["step"] for c in recs[1:-1]] == [30, 40]
