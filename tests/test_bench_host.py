"""Host-side logic of the benchmark, on CPU with a stand-in simulation.

* The FP64 leg reads the per-phase profile before switching profiling off
  (pic_profile clears the accumulated times), so its hot-kernel time is the
  measured one, not zero.
* Per-step phase costs divide the sort by its interval; per-launch means are
  reported under their own key.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class FakeSim:
    """Mimics the binding: profile(False) clears the accumulated times."""

    def __init__(self):
        self.prof_ms, self.enabled = 0.0, False

    def load(self, *a):
        pass

    def step(self, n):
        if self.enabled:
            self.prof_ms += 2.5 * n

    def profile(self, enable=True):
        self.enabled = enable
        self.prof_ms = 0.0

    def get_profile(self):
        names = ["particles", "reduce", "filter", "fields", "inject", "sort"]
        return {k: (self.prof_ms / 20 if k == "particles" else 0.0) for k in names}, 20

    def live(self):
        return 1000

    def fields(self):
        return np.ones((6, 3, 3))

    def moments(self):
        return {"gauss_residual": 0.0, "live": 1000, "axis_ties": 0}

    def close(self):
        pass

    def axis_ties(self):
        return {"step": np.zeros(0, np.int64), "id": np.zeros(0, np.int64), "sign": np.zeros(0, np.int32)}

    def set_axis_hints(self, ties):
        self.hints = ties


def test_fp64_leg_reads_the_profile_before_disabling_it(monkeypatch):
    import torch

    import bench

    monkeypatch.setattr(bench.W, "make_sim", lambda *a, **k: (FakeSim(), 1.0, 0.1, 1.0))
    monkeypatch.setattr(bench.W, "load_plasma", lambda *a, **k: 1000)

    def fake_time_steps(sim, K, stream):
        sim.step(K)
        return 50.0, 1000.0 * K, 3 * K

    monkeypatch.setattr(bench, "time_steps", fake_time_steps)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a, **k: None)
    cfg = {"nr": 4, "nth": 4, "pairs_per_cell": 1, "T": 0.3, "seed": 0}
    args = bench.parse(["--fp64-steps", "20", "--compare-steps", "30"])

    class _S:
        cuda_stream = 0

    res = bench.fp64_run(cfg, "cpu", _S(), args)
    assert res["hot_kernel"]["ms_per_launch"] == 2.5
    assert res["hot_kernel"]["achieved_GBps"] > 0


def test_phase_costs_per_step_divide_the_sort_by_its_interval():
    import bench

    prof = {"particles": 22.0, "reduce": 0.2, "filter": 0.0, "fields": 1.5, "inject": 0.0, "sort": 18.0}
    per_step = bench.phase_per_step(prof, 20)
    assert per_step["sort"] == 0.9
    assert per_step["particles"] == 22.0
