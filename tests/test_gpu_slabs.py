"""One simulation split into radial slabs (the grid decomposition the paper
parallelises over MPI, Sec. 2) against the same simulation on one context and
against the oracle, through the C-ABI.

Each slab is a context of its own on one GPU; every step exchanges field
halos, sums back the flux deposited across each interface before the filter
and hands migrating particles to the neighbouring slab.  Bars: on the FP64
path fields and fluxes within 1e-12 relative (L2 and per-component max-norm)
of the unsplit run and of the oracle, particle counts, deletions, injections
and the set of live ids exactly equal; on the FP32 path the split run equals
the unsplit FP32 run bit for bit (fields, fluxes, every particle) and the
oracle at the FP32 bar.
"""
import numpy as np
import pytest

import oracle as O
from paper_1407_1810_gb300 import configs, synthetic

from gpu_common import KEYS, MAX_FP32, by_id, close, follow_ties, maxnorm_rel, rel_l2, setup

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()
    O.build_oracle()


def _slabs(cfg, dt, b0, nslabs, rows=None):
    from paper_1407_1810_gb300 import picsar as P

    return P.Slabs(P.make_desc(**configs.desc_kwargs(cfg, dt, b0)), nslabs, rows)


CASES = {
    # hot monopole plasma: particles cross the interfaces and both conductors
    "monopole": dict(configs.CONFIGS["monopole-64x64"], nr=64, nth=40, pairs_per_cell=3, T=1.0),
    # rotator with surface injection, 3 filter passes and a quadratic lossy layer
    "rotator": dict(configs.CONFIGS["rotator-512x512"], nr=64, nth=32, pairs_per_cell=2, absorb_cells=8,
                    t_spin=2.0, precision="fp64"),
}


@pytest.mark.parametrize("case", ["monopole", "rotator"])
@pytest.mark.parametrize("nslabs,rows", [(2, None), (4, None), (3, [0, 13, 40, 64])])
def test_slabs_match_one_context_and_the_oracle(case, nslabs, rows):
    cfg = CASES[case]
    s, o, plasma, dt = setup(cfg)
    b0 = s.desc.b0
    g = _slabs(cfg, dt, b0, nslabs, rows)
    g.load(*(np.ascontiguousarray(plasma[k]) for k in KEYS))
    o.gauss_snapshot()
    for _ in range(4):
        s.step(25)
        g.step(25)
        o.step(25)
    fs, fg, fo = s.fields(), g.fields(), o.fields()
    assert rel_l2(fg, fs) < TOL and maxnorm_rel(fg, fs) < TOL
    assert rel_l2(fg, fo) < TOL and maxnorm_rel(fg, fo) < TOL
    assert rel_l2(g.flux(), s.flux()) < TOL
    ms, mg, cnt = s.moments(), g.moments(), o.counters()
    for k in ("live", "deleted", "injected", "step"):
        assert mg[k] == ms[k], k
    assert mg["live"] == cnt["live"] and mg["injected"] == cnt["injected"]
    assert mg["deleted"] > 0
    assert mg["kinetic_energy"] == pytest.approx(ms["kinetic_energy"], rel=TOL)
    assert mg["field_energy"] == pytest.approx(ms["field_energy"], rel=1e-11)
    assert mg["gauss_residual"] < 1e-11
    assert mg["gauss_residual"] == pytest.approx(ms["gauss_residual"], abs=1e-12)
    pg, ps = by_id(g.particles()), by_id(s.particles())
    assert np.array_equal(pg["id"], ps["id"])
    for k in KEYS:
        assert np.max(np.abs(pg[k] - ps[k])) < 1e-9, k


def test_one_slab_is_the_whole_grid():
    """nslabs = 1 has no interface: the same kernels and schedule as one
    context (equal up to the order of the FP64 atomic current sums)."""
    cfg = CASES["rotator"]
    s, o, plasma, dt = setup(cfg)
    g = _slabs(cfg, dt, s.desc.b0, 1)
    g.load(*(np.ascontiguousarray(plasma[k]) for k in KEYS))
    s.step(30)
    g.step(30)
    assert rel_l2(g.fields(), s.fields()) < 1e-13
    assert g.moments()["live"] == s.moments()["live"]


def test_particles_migrate_both_ways():
    """A hot plasma seeded in the rows next to one interface: after a few
    steps particles have crossed it in both directions, and the particle set
    equals the unsplit run's."""
    cfg = dict(CASES["monopole"], T=3.0)
    dt = O.oracle.courant_dt(O.params(**configs.oracle_kwargs(cfg, 0.0, 0.0)), cfg["courant"])
    b0, qw = configs.physics(cfg, dt)
    cells = np.array([i * cfg["nth"] + j for i in (30, 31, 32, 33) for j in range(cfg["nth"])])
    plasma = synthetic.pair_plasma_cells(cfg["nr"], cfg["nth"], cells, 4, cfg["T"], qw, 3)
    s, _, _, _ = setup(cfg, plasma=plasma)
    g = _slabs(cfg, dt, b0, 2)  # interface at row 32
    g.load(*(np.ascontiguousarray(plasma[k]) for k in KEYS))
    x0 = plasma["x1"]
    s.step(6)
    g.step(6)
    pg, ps = by_id(g.particles()), by_id(s.particles())
    assert np.array_equal(pg["id"], ps["id"])
    start = x0[pg["id"]]
    assert np.sum((start < 32) & (pg["x1"] >= 32)) > 0 and np.sum((start >= 32) & (pg["x1"] < 32)) > 0
    assert rel_l2(g.fields(), s.fields()) < TOL


FP32_CASES = {
    "monopole": dict(CASES["monopole"], precision="fp32"),
    "rotator": dict(CASES["rotator"], precision="fp32"),
}


@pytest.mark.parametrize("case", ["monopole", "rotator"])
@pytest.mark.parametrize("nslabs,rows", [(2, None), (3, [0, 13, 40, 64]), (4, None)])
def test_fp32_slabs_equal_one_context_bit_for_bit(case, nslabs, rows):
    """The FP32 path split into slabs: one fixed-point quantum for all slabs
    and exact int64 sums across the interfaces, so the split run equals the
    unsplit one in every bit; both against the oracle at the FP32 bar."""
    cfg = FP32_CASES[case]
    s, o, plasma, dt = setup(cfg)
    g = _slabs(cfg, dt, s.desc.b0, nslabs, rows)
    g.load(*(np.ascontiguousarray(plasma[k]) for k in KEYS))
    o.gauss_snapshot()
    for _ in range(4):
        s.step(25)
        g.step(25)
    assert np.array_equal(g.fields(), s.fields())
    assert np.array_equal(g.flux(), s.flux())
    ms, mg = s.moments(), g.moments()
    for k in ("live", "deleted", "injected", "step"):
        assert mg[k] == ms[k], k
    assert mg["deleted"] > 0
    assert mg["gauss_residual"] < 1e-6
    pg, ps = by_id(g.particles()), by_id(s.particles())
    assert np.array_equal(pg["id"], ps["id"])
    for k in KEYS:
        assert np.array_equal(pg[k], ps[k]), k
    follow_ties(s, o)
    o.step(100)
    close(g.fields(), o.fields(), 1e-5, MAX_FP32 if cfg["th_map"] == "equal_area" else 1e-3)
