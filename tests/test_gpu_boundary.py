"""GPU parity of the boundary's read-out calls (through the C-ABI).

* pic_get_fields(PIC_FIELDS_TOTAL): plasma plus analytic field at every
  staggered point, after 30 steps of the rotator with injection, against the
  oracle's total field (1e-12 FP64 path, 1e-5 FP32 path).
* pic_get_charge: the node charge of the GPU's own particles, raw and after
  the n_filt passes with the polar fold, against the oracle given the same
  particles (1e-13 of the largest node charge); its sum is the total charge.
* pic_grid_coords: the inverse grid maps in all four coordinate systems
  against the oracle's (1e-12 cell).
"""
import numpy as np
import pytest

import oracle as O
from paper_1407_1810_gb300 import configs

from gpu_common import KEYS, rel_l2, setup

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()
    O.build_oracle()


def _rotator(precision):
    return dict(configs.CONFIGS["rotator-512x512"], nr=40, nth=32, pairs_per_cell=2, absorb_cells=8, t_spin=2.0,
                precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_total_fields_against_oracle(precision):
    s, o, _, _ = setup(_rotator(precision))
    s.step(30)
    o.step(30)
    g, r = s.fields(total=True), o.fields(total=True)
    assert rel_l2(g, r) < TOL[precision]
    # the analytic part alone is the same function of the clock on both sides
    assert rel_l2(g - s.fields(), r - o.fields()) < 1e-13
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_node_charge_against_oracle(precision):
    cfg = _rotator(precision)
    s, o, _, dt = setup(cfg)
    s.step(30)
    st = s.particles()
    b0, _ = configs.physics(cfg, dt)
    o2 = O.Oracle(O.params(**configs.oracle_kwargs(cfg, dt, b0)))
    o2.load(*(st[k] for k in KEYS), ids=st["id"])
    q_o = o2.node_charge()
    scale = np.max(np.abs(q_o))
    q_g = s.charge()
    assert np.max(np.abs(q_g - q_o)) < 1e-13 * scale
    assert q_g.sum() == pytest.approx(st["qw"].sum(), abs=1e-12 * np.abs(st["qw"]).sum())
    qf = q_o
    for _ in range(cfg["n_filt"]):
        qf = o2.filter_pass(qf, 0, +1)
    assert np.max(np.abs(s.charge(filtered=True) - qf)) < 1e-13 * scale
    s.close()


@pytest.mark.parametrize("r_map,th_map", [("linear", "linear"), ("log", "equal_area"), ("log", "linear"),
                                          ("linear", "equal_area")])
def test_grid_coords_against_oracle(r_map, th_map):
    cfg = dict(configs.CONFIGS["monopole-64x64"], r_map=r_map, th_map=th_map, pairs_per_cell=0)
    s, o, _, _ = setup(cfg, plasma={k: np.zeros(0) for k in KEYS})
    rng = np.random.default_rng(5)
    r = rng.uniform(cfg["r_min"], cfg["r_max"], 4000)
    th = rng.uniform(0.0, np.pi, 4000)
    x1, x2 = s.grid_coords(r, th)
    assert np.max(np.abs(x1 - o.f_r_inv(r))) < 1e-12
    assert np.max(np.abs(x2 - o.f_th_inv(th))) < 1e-12
    s.close()
