"""Pins of the oracle's spin-down luminosity (Sec. 5.3, Fig. 7d): the
radial Poynting flux (E x B)_r of the total field through the sphere of each
node radius.

* Uniform fields: E_th = B_ph = 1 give exactly 4 pi r^2 on every sphere (the
  ring areas telescope); E_ph = B_th = 1 give -4 pi r^2 (the sign of (E x B)_r).
* The analytic field is part of the total: a uniform B along +z
  (B_th = -b0 sin th) with a plasma E_ph = e carries e b0 2 pi r^2 times the
  integral of sin^2 th over [0, pi], pi^2 r^2 e b0.
* The force-free monopole wind (Michel): B_ph = E_th = -Omega r sin th B_r with
  B_r = B0 r0^2 / r^2 carries L0 = (8 pi / 3) B0^2 r0^4 Omega^2 in
  Lorentz-Heaviside units, (2 c / 3) (B0 r0^2 / R_l)^2 in the paper's Gaussian
  units, through every sphere, to the quadrature's O(dxi^2, dth^2).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.oracle import courant_dt

ER, ETH, EPH, BR, BTH, BPH = range(6)


def _o(**kw):
    base = dict(nr=32, nth=64, r_min=1.0, r_max=10.0, r_map="log", th_map="linear", n_filt=0, vacuum="none")
    base.update(kw)
    p = O.params(**base)
    p.dt = courant_dt(p, 0.5)
    return O.Oracle(p)


def test_uniform_fields_give_the_sphere_area_with_the_poynting_sign(oracle_mod):
    o = _o()
    r = o.f_r(np.arange(o.nr + 1))
    f = np.zeros(o.field_shape)
    f[ETH] = 1.0
    f[BPH] = 1.0
    o.set_fields(f)
    L = o.luminosity(0.0)
    assert L[0] == 0.0 and L[-1] == 0.0
    np.testing.assert_allclose(L[1:-1], 4 * math.pi * r[1:-1] ** 2, rtol=1e-13)
    f[:] = 0.0
    f[EPH] = 1.0
    f[BTH] = 1.0
    o.set_fields(f)
    np.testing.assert_allclose(o.luminosity(0.0)[1:-1], -4 * math.pi * r[1:-1] ** 2, rtol=1e-13)


def test_analytic_field_is_part_of_the_flux(oracle_mod):
    b0, e = 2.0, 0.7
    o = _o(vacuum="uniform_bz", b0=b0, nth=128)
    r = o.f_r(np.arange(o.nr + 1))
    f = np.zeros(o.field_shape)
    f[EPH] = e
    o.set_fields(f)
    L = o.luminosity(0.0)
    np.testing.assert_allclose(L[1:-1], math.pi ** 2 * r[1:-1] ** 2 * e * b0, rtol=2e-4)


@pytest.mark.parametrize("th_map", ["linear", "equal_area"])
def test_michel_monopole_wind_carries_l0(oracle_mod, th_map):
    B0, W = 3.0, 0.2
    o = _o(th_map=th_map, nr=64, nth=128)
    i = np.arange(o.nr + 1)
    j = np.arange(o.nth + 1)
    r_n = o.f_r(i)
    r_h = o.f_r(i + 0.5)
    s_h = np.zeros(o.nth + 1)
    s_h[:-1] = np.sin(o.f_th(j[:-1] + 0.5))  # half-integer entries j < nth
    f = np.zeros(o.field_shape)
    f[BR] = B0 / r_n[:, None] ** 2 * np.ones_like(s_h)[None, :]
    f[ETH] = -W * B0 * s_h[None, :] / r_n[:, None]  # -Omega r sin th B_r at (i, j+1/2)
    f[BPH] = -W * B0 * s_h[None, :] / r_h[:, None]  # the same at (i+1/2, j+1/2)
    o.set_fields(f)
    L0 = 8 * math.pi / 3 * B0 ** 2 * W ** 2
    L = o.luminosity(0.0)[1:-1]
    np.testing.assert_allclose(L / L0, 1.0, atol=2e-3)
