"""Pins of the oracle's diagnostics against closed forms and an independent
restatement of the discrete Gauss law.

* Field energy 1/2 sum (E^2 + B^2) dV (Sec. 2, the energy of the fields the
  Yee update advances): a uniform value of any one component fills cells that
  tile the spherical shell exactly, so its energy is 1/2 v^2 (4 pi / 3)
  (r_max^3 - r_min^3) to rounding; the static vacuum monopole
  B_r = B0 (r0/r)^2 and a meridional profile E_th = cos(th) converge at
  second order in the cell size to their integrals.
* Kinetic energy sum |qw| / (q/m) (gamma - 1): exact values at gamma = 1, 2, 3
  and the non-relativistic limit u^2 / 2.
* Gauss law in integral form (App. A, App. B): G_ij, the outward flux of E
  through the dual cell of node (i, j) with the polar caps closed at the axis,
  written out here from the area elements dA_thph and dA_rph, minus the node
  charge filtered with the fold of App. B, stays constant to rounding; the
  same charge filtered with the opposite fold sign does not.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.oracle import courant_dt


def _oracle(nr, nth, r_map="log", th_map="linear", r_min=1.0, r_max=10.0, **kw):
    p = O.params(nr=nr, nth=nth, r_min=r_min, r_max=r_max, r_map=r_map, th_map=th_map, **kw)
    p.dt = courant_dt(p, 0.5)
    return O.Oracle(p)


# staggering of Eq. (offseteq) in the plane layout of orc_get_fields:
# (half-integer i, half-integer j) and the index ranges of each component
STAG = {0: (1, 0), 1: (0, 1), 2: (0, 0), 3: (0, 1), 4: (1, 0), 5: (1, 1)}


@pytest.mark.parametrize("r_map,th_map", [("log", "linear"), ("linear", "equal_area")])
@pytest.mark.parametrize("comp", range(6))
def test_field_energy_of_a_uniform_component_is_the_shell_volume(oracle_mod, r_map, th_map, comp):
    nr, nth, v = 20, 14, 1.7
    o = _oracle(nr, nth, r_map, th_map, r_max=5.0)
    f = np.zeros(o.field_shape)
    si, sj = STAG[comp]
    f[comp, : nr + 1 - si, : nth + 1 - sj] = v
    o.set_fields(f)
    shell = 4.0 * math.pi / 3.0 * (5.0**3 - 1.0**3)
    assert o.field_energy() == pytest.approx(0.5 * v * v * shell, rel=1e-13)


def _monopole_energy_error(nr):
    o = _oracle(nr, 8, "log", "linear", r_max=10.0)
    f = np.zeros(o.field_shape)
    r = o.f_r(np.arange(nr + 1))
    f[3, :, :8] = (1.0 / r**2)[:, None]  # B_r at (i, j + 1/2), B0 = r0 = 1
    o.set_fields(f)
    exact = 2.0 * math.pi * (1.0 - 1.0 / 10.0)  # 1/2 int B^2 dV = 2 pi B0^2 r0^4 (1/r0 - 1/r_max)
    return abs(o.field_energy() - exact) / exact


def _meridional_energy_error(nth):
    o = _oracle(4, nth, "linear", "linear", r_min=1.0, r_max=2.0)
    f = np.zeros(o.field_shape)
    tb = o.f_th(np.arange(nth) + 0.5)
    f[1, :, :nth] = np.cos(tb)[None, :]  # E_th at (i, j + 1/2)
    o.set_fields(f)
    # 1/2 int cos^2(th) dV over r in [1, 2]: (2 pi / 3)(8 - 1)(1/2)(2/3)
    exact = 0.5 * 2.0 * math.pi / 3.0 * 7.0 * (2.0 / 3.0)
    return abs(o.field_energy() - exact) / exact


@pytest.mark.parametrize("err", [_monopole_energy_error, _meridional_energy_error])
def test_field_energy_converges_at_second_order(oracle_mod, err):
    e = [err(n) for n in (32, 64, 128, 256)]
    slopes = [math.log2(a / b) for a, b in zip(e, e[1:])]
    assert all(1.8 < s < 2.2 for s in slopes), (e, slopes)
    assert e[-1] < 1e-3


def test_kinetic_energy_closed_values(oracle_mod):
    o = _oracle(8, 8, q_over_m=2.0)
    # gamma = 1, 2, 3 and a slow particle (u = 1e-4: gamma - 1 = u^2/2 - u^4/8)
    ur = np.array([0.0, 0.0, 2.0, 1e-4])
    ut = np.array([0.0, 1.0, 2.0, 0.0])
    up = np.array([0.0, math.sqrt(2.0), 0.0, 0.0])
    qw = np.array([0.5, -0.25, 3.0, 4.0])
    x = np.full(4, 3.5)
    o.load(x, x, ur, ut, up, qw)
    expect = (0.5 * 0 + 0.25 * 1.0 + 3.0 * 2.0 + 4.0 * (0.5e-8 - 1.25e-17)) / 2.0
    assert o.kinetic_energy() == pytest.approx(expect, rel=1e-12)


# --------------------------------------------------------------------------
# Gauss law, restated from the area elements of App. A
# --------------------------------------------------------------------------
def _gauss_flux(o, f):
    """G[i, j] for 1 <= i <= nr - 1, every j: outward flux of E through the
    dual cell [rb_{i-1}, rb_i] x [tb_{j-1}, tb_j] of node (i, j), the
    meridional range closed at the axis for j = 0 and j = nth."""
    nr, nth = o.nr, o.nth
    rb = o.f_r(np.arange(nr) + 0.5)          # rb_i, i = 0..nr-1
    tb = o.f_th(np.arange(nth) + 0.5)        # tb_j, j = 0..nth-1
    tlo = np.concatenate([[0.0], tb])        # lower meridional edge of node j's dual cell
    thi = np.concatenate([tb, [math.pi]])    # upper edge
    G = np.zeros((nr + 1, nth + 1))
    for i in range(1, nr):
        ra, rbb = rb[i - 1], rb[i]
        band = np.cos(tlo) - np.cos(thi)
        G[i] = f[0, i] * 2 * math.pi * rbb**2 * band - f[0, i - 1] * 2 * math.pi * ra**2 * band
        side = math.pi * (rbb**2 - ra**2)
        G[i, :nth] += f[1, i, :nth] * side * np.sin(tb)
        G[i, 1:] -= f[1, i, :nth] * side * np.sin(tb)
    return G


def _filtered(o, q, sign):
    for _ in range(o.p.n_filt):
        q = o.filter_pass(q, 0, sign)
    return q


def test_gauss_law_restated_and_the_wrong_fold_breaks_it(oracle_mod):
    """Control of the filter's fold sign (App. B): with the fold of R7 the
    restated G - Qbar stays constant to rounding over 30 steps of a plasma
    crossing the axis; folding the charge with the opposite sign leaves a
    residual far above the 1e-6 bar."""
    from paper_1407_1810_gb300 import synthetic

    N = 16
    p = O.params(nr=N, nth=N, r_min=1.0, r_max=6.0, r_map="log", th_map="linear", n_filt=2,
                 absorb_cells=4, absorb_profile="linear", vacuum="monopole_rotator", b0=20.0, omega=0.2,
                 t_spin=0.5)
    p.dt = courant_dt(p, 0.5)
    o = O.Oracle(p)
    d = synthetic.pair_plasma(N, N, 3, 0.5, 0.01, 0)
    o.load(d["x1"], d["x2"], d["ur"], d["uth"], d["uph"], d["qw"])
    o.step(2)
    g = o.g
    imax = N - 4 - 1

    def diffs():
        G = _gauss_flux(o, o.fields())
        q = o.node_charge()
        good = G - _filtered(o, q, +1)[g: g + N + 1]
        bad = G - _filtered(o, q, -1)[g: g + N + 1]
        return good[1: imax + 1], bad[1: imax + 1]

    o.gauss_snapshot()
    good0, bad0 = diffs()
    assert o.step(30) == 0
    good1, bad1 = diffs()
    den = np.max(o.node_charge(absolute=True))
    res_good = np.max(np.abs(good1 - good0)) / den
    res_bad = np.max(np.abs(bad1 - bad0)) / den
    assert res_good < 1e-12
    assert o.gauss_residual() == pytest.approx(res_good, abs=1e-13)
    assert res_bad > 1e-6, res_bad
