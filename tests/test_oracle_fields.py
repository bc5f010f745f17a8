"""Pins of the oracle's field solve (Appendix A) against closed forms.

* Sec. 4.1: the l = 1 spherical TM mode between the first and fourth roots of
  du_1/dr converges at second order in all four coordinate systems.
* The vacuum monopole B_r = B0 (r0/r)^2 is an exact discrete steady state, and
  the discrete div B stays zero (Sec. 2: Yee keeps the constraints).
* The lossy layer (Sec. 3.4.1) absorbs an outgoing pulse.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle as O
from oracle.oracle import courant_dt


def u1(r):
    return np.sin(r) / r - np.cos(r)


def du1(r):
    return np.cos(r) / r - np.sin(r) / r**2 + np.sin(r)


def du1_roots(n):
    roots, a = [], 0.5
    while len(roots) < n:
        b = a + 0.05
        if du1(a) * du1(b) < 0:
            roots.append(brentq(du1, a, b, xtol=1e-15))
        a = b
    return roots


R_IN, _, _, R_OUT = du1_roots(4)


def tm_error(N, r_map, th_map, courant=0.5):
    """L2 error of r B_phi at t = 1.25/omega (k = omega = 1), Sec. 4.1."""
    p = O.params(nr=N, nth=N, r_min=R_IN, r_max=R_OUT, r_map=r_map, th_map=th_map, n_filt=0)
    dtc = courant_dt(p, courant)
    nsteps = int(math.ceil(1.25 / dtc))
    p.dt = 1.25 / nsteps
    o = O.Oracle(p)
    rb = o.f_r(np.arange(N) + 0.5)
    tb = o.f_th(np.arange(N) + 0.5)
    f = np.zeros(o.field_shape)
    # B at -dt/2 (B lags E by half a step); E(0) = 0 for the real part
    f[5, :N, :N] = (u1(rb) / rb)[:, None] * np.sin(tb)[None, :] * math.cos(0.5 * p.dt)
    o.set_fields(f)
    o.field_step(nsteps)
    g = o.fields()
    exact = (u1(rb) / rb)[:, None] * np.sin(tb)[None, :] * math.cos(1.25)
    w = rb[:, None] ** 2
    return math.sqrt(np.sum(w * (g[5, :N, :N] - exact) ** 2) / np.sum(w * exact**2))


@pytest.mark.parametrize("r_map,th_map", [("linear", "linear"), ("log", "equal_area"),
                                          ("log", "linear"), ("linear", "equal_area")])
def test_tm_mode_second_order(oracle_mod, r_map, th_map):
    errs = [tm_error(N, r_map, th_map) for N in (16, 32, 64)]
    # mean slope over two doublings of the resolution (time step halves too)
    slope = 0.5 * math.log2(errs[0] / errs[2])
    assert errs[2] < 1e-2, errs
    assert abs(slope - 2.0) < 0.15, (errs, slope)


def _monopole_oracle(r_map="log", th_map="equal_area", N=24):
    p = O.params(nr=N, nth=N + 8, r_min=1.0, r_max=20.0, r_map=r_map, th_map=th_map, n_filt=0)
    p.dt = courant_dt(p, 0.5)
    o = O.Oracle(p)
    f = np.zeros(o.field_shape)
    r = o.f_r(np.arange(N + 1))
    f[3, :, : p.nth] = (1.0 / r**2)[:, None]
    o.set_fields(f)
    return o, f


@pytest.mark.parametrize("r_map,th_map", [("log", "equal_area"), ("linear", "linear")])
def test_static_monopole_is_steady(oracle_mod, r_map, th_map):
    o, f0 = _monopole_oracle(r_map, th_map)
    o.field_step(200)
    f = o.fields()
    assert np.max(np.abs(f - f0)) < 1e-14
    # discrete div B of the monopole vanishes cell by cell
    db = o.divb()
    scale = np.max(np.abs(f0[3])) * 4 * np.pi
    assert np.max(np.abs(db)) < 1e-14 * scale


def test_divb_stays_zero_from_random_e(oracle_mod):
    p = O.params(nr=20, nth=24, r_min=1.0, r_max=8.0, r_map="log", th_map="linear", n_filt=0)
    p.dt = courant_dt(p, 0.5)
    o = O.Oracle(p)
    rng = np.random.default_rng(3)
    f = np.zeros(o.field_shape)
    f[0, :20, :] = rng.standard_normal((20, 25))
    f[1, 1:20, :24] = rng.standard_normal((19, 24))
    f[2, 1:20, 1:24] = rng.standard_normal((19, 23))
    o.set_fields(f)
    o.field_step(50)
    g = o.fields()
    assert np.max(np.abs(g[3:])) > 1e-3  # B did develop
    db = o.divb()
    assert np.max(np.abs(db)) < 1e-12 * np.max(np.abs(g[3:]))


def test_field_energy_bounded_without_layer(oracle_mod):
    """Control for the lossy-layer test: with two conductors and no layer the
    leapfrog keeps the field energy bounded (no growth, no loss)."""
    o, e0 = _pulse_oracle("none", 0)
    o.field_step(o._nsteps)
    e1 = o.field_energy()
    assert 0.8 * e0 < e1 < 1.2 * e0


def _pulse_oracle(profile, cells):
    # grid of the small monopole workload (log r in [1, 10]); the outer cells
    # (0.18 r0) still resolve the pulse, so the waves reach the layer
    N, nth, rmax = 128, 32, 10.0
    p = O.params(nr=N, nth=nth, r_min=1.0, r_max=rmax, r_map="log", th_map="equal_area",
                 n_filt=0, absorb_cells=cells, absorb_profile=profile)
    p.dt = courant_dt(p, 0.5)
    o = O.Oracle(p)
    # a TM-like B_phi shell near r = 4; E = 0 splits it into in/outgoing halves
    rb = o.f_r(np.arange(N) + 0.5)
    tb = o.f_th(np.arange(nth) + 0.5)
    f = np.zeros(o.field_shape)
    f[5, :N, :nth] = np.exp(-(((rb - 4.0) / 0.6) ** 2))[:, None] * np.sin(tb)[None, :] / rb[:, None]
    o.set_fields(f)
    e0 = o.field_energy()
    # 2.5 light-crossing times: out, through the layer, off the conductor, back
    o._nsteps = int(2.5 * (rmax - 1.0) / p.dt)
    return o, e0


@pytest.mark.parametrize("profile,cells", [("linear", 16), ("quadratic", 32)])
def test_lossy_layer_absorbs_outgoing_pulse(oracle_mod, profile, cells):
    o, e0 = _pulse_oracle(profile, cells)
    o.field_step(o._nsteps)
    assert o.field_energy() < 0.01 * e0
