"""Ties of the azimuth branch at the polar axis (reading 19 of the design;
oracle reading R15) on both GPU paths, through the C-ABI.

A particle 0.1 cell from the north axis moves straight towards and past it
(u_th < 0, no fields) with a tiny azimuthal momentum u_ph: the move crosses
the axis and the swept azimuth is +-pi with the sign of u_ph, so the two
branches put +1/2 and -1/2 of the charge through the meridional half-plane.
|u_ph| = 1e-9 |u| is a tie: logged as (step, id, sign), and a hint for that
(step, id) fixes the branch; a hint for another step or particle, or a
crossing with |u_ph| = 0.017 |u|, leaves the branch alone.  The oracle, given
the same hints, takes the same branch.  On the FP32 path the crossing is taken
once by a binned particle (shared-memory window) and once by a particle
loaded after the sort (global-memory path).
"""
import numpy as np
import pytest

import oracle as O
from paper_1407_1810_gb300 import configs

from gpu_common import setup

pytestmark = pytest.mark.gpu
QW = 0.37


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()
    O.build_oracle()


def _cfg(precision):
    return dict(configs.CONFIGS["monopole-64x64"], nr=16, nth=64, th_map="linear", vacuum="none",
                precision=precision, pairs_per_cell=0, absorb_cells=4)


def _one(uph, x1=7.3):
    return {"x1": np.array([x1]), "x2": np.array([0.1]), "ur": np.array([0.0]), "uth": np.array([-3.0]),
            "uph": np.array([uph]), "qw": np.array([QW])}


def _azimuthal(sim):
    return sim.flux()[2].sum() / QW


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tie_branch_log_and_hints(precision):
    for uph, half in ((1e-9, 0.5), (-1e-9, -0.5)):
        s, o, _, _ = setup(_cfg(precision), plasma=_one(uph))
        s.step(1)
        o.step(1)
        t = s.axis_ties()
        assert list(t["step"]) == [0] and list(t["id"]) == [0] and list(t["sign"]) == [1 if half > 0 else -1]
        assert s.moments()["axis_ties"] == 1 and o.axis_ties() == 1
        assert _azimuthal(s) == pytest.approx(half, abs=1e-5)
        assert _azimuthal(s) == pytest.approx(_azimuthal(o), abs=1e-5)
        assert 0.0 < s.particles()["x2"][0] < 0.1  # reflected through the axis
    # a hint for (step 0, particle 0) flips the branch, on the GPU as in the oracle
    flip = {"step": [0], "id": [0], "sign": [1]}
    s, o, _, _ = setup(_cfg(precision), plasma=_one(-1e-9))
    s.set_axis_hints(flip)
    o.set_axis_hints(flip)
    s.step(1)
    o.step(1)
    assert _azimuthal(s) == pytest.approx(0.5, abs=1e-5) and list(s.axis_ties()["sign"]) == [1]
    assert _azimuthal(o) == pytest.approx(0.5, abs=1e-5)
    # hints for another step or another particle leave it alone
    s, _, _, _ = setup(_cfg(precision), plasma=_one(-1e-9))
    s.set_axis_hints({"step": [1, 0], "id": [0, 5], "sign": [1, 1]})
    s.step(1)
    assert _azimuthal(s) == pytest.approx(-0.5, abs=1e-5)
    # |u_ph| = 0.017 |u|: no tie, the hint is not consulted
    s, _, _, _ = setup(_cfg(precision), plasma=_one(-0.05))
    s.set_axis_hints(flip)
    s.step(1)
    assert s.moments()["axis_ties"] == 0 and _azimuthal(s) < -0.49


def test_tie_on_the_global_memory_path():
    """FP32: a particle binned in the second tile column (x2 = 16.5, whose
    window spans columns 11-36) drifts to the axis without a sort and crosses
    it outside its window, i.e. on the global-memory path; its tie is logged
    at that step and a hint for it flips the branch as on the window path."""
    cfg = dict(_cfg("fp32"), sort_interval=1000)

    def run(hints=None):
        s, _, _, _ = setup(cfg, plasma=_one(-1e-9) | {"x2": np.array([16.5])})
        if hints:
            s.set_axis_hints(hints)
        for n in range(400):
            s.step(1)
            if s.moments()["axis_ties"]:
                return s, n, _azimuthal(s)
        pytest.fail("the particle did not reach the axis")

    s, n, f = run()
    t = s.axis_ties()
    assert n > 50  # far from its tile: the crossing is on the global-memory path
    assert list(t["step"]) == [n] and list(t["id"]) == [0] and list(t["sign"]) == [-1]
    assert f == pytest.approx(-0.5, abs=1e-5)
    s2, n2, f2 = run({"step": [n], "id": [0], "sign": [1]})
    assert n2 == n and list(s2.axis_ties()["sign"]) == [1]
    assert f2 == pytest.approx(0.5, abs=1e-5)
