"""Pins of the oracle's injection variants and the aligned dipole rotator.

* Variable-count injection, Eq. (volinjeq) as printed (reading R13): each
  surface cell gets floor(n_j) or floor(n_j) + 1 pairs of charge -+q, with
  n_j = f_inj |sigma_j| dA_j / q from the closed-form surface charge of the
  rotating monopole; over many seeds the mean count is n_j; counts above the
  cap are cut to it and counted.  The uniform numbers come from SplitMix64,
  whose published outputs the oracle's generator reproduces.
* Smoothing of sigma along theta (Sec. 5.3, reading R12): the 1-2-1 stencil
  leaves a profile linear in j unchanged away from the poles; each polar cell
  is its own mirror image, so one pass gives (3 s_0 + s_1) / 4 there.  On the
  equal-area grid the rotating monopole's sigma_j is exactly linear in j.
* Aligned dipole rotator (reading R14): outside, E = -grad of the l = 2
  potential -(Omega mu r0^2 / 3 r^3)(3 cos^2 th - 1), which is harmonic and
  carries no net charge through any sphere; inside, the corotation field
  -(Omega x r) x B with E.B = 0; E_th continuous across r0; B the dipole.
  The injected charge is the jump of E_r across the surface, integrated.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from oracle.oracle import courant_dt, splitmix64


def test_splitmix64_reproduces_published_outputs(oracle_mod):
    # first outputs of SplitMix64 (Steele, Lea and Flood 2014) as printed by
    # the public-domain reference implementation, for seeds 0 and 1234567
    assert [splitmix64(0, n) for n in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [splitmix64(1234567, n) for n in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431, 16408922859458223821]


B0, OM, FIN, R0 = 3.0, 0.2, 0.5, 1.0


def _rotator(nth=32, th_map="equal_area", **kw):
    base = dict(nr=16, nth=nth, r_min=R0, r_max=10.0, r_map="log", th_map=th_map, vacuum="monopole_rotator",
                b0=B0, omega=OM, t_spin=0.0, inject=1, pairs_per_cell=2, f_inj=FIN)
    base.update(kw)
    p = O.params(**base)
    p.dt = courant_dt(p, 0.5)
    o = O.Oracle(p)
    o.step(1)  # no particles: the plasma field stays 0, then one injection
    return o


def _monopole_sigma(o, nth):
    """sigma_j of the rotating monopole, closed form: the mean over the cell's
    two nodes of E_r = -2 B0 r0^4 Omega cos(th) / r^3 at r = f_r(1/2)."""
    rb = float(o.f_r(0.5))
    ct = np.cos(o.f_th(np.arange(nth + 1)))
    er = -2.0 * B0 * R0**4 * OM * ct / rb**3
    return 0.5 * (er[:-1] + er[1:]), 2.0 * math.pi * R0**2 * (ct[:-1] - ct[1:])


def _counts(d, nth):
    pos = d["qw"] > 0
    return np.bincount(np.floor(d["x2"][pos]).astype(int), minlength=nth)


def test_variable_counts_are_the_expected_number_rounded(oracle_mod):
    nth, q, cap = 32, 0.02, 64
    x = None
    total, seeds = np.zeros(nth), 300
    for seed in range(seeds):
        o = _rotator(nth, inject=2, inject_q=q, inject_seed=seed, pairs_per_cell=cap)
        if x is None:
            sig, dA = _monopole_sigma(o, nth)
            x = FIN * np.abs(sig) * dA / q
        d = o.particles()
        c = _counts(d, nth)
        lo, hi = np.floor(x - 1e-9), np.floor(x + 1e-9) + 1
        assert np.all((c >= lo) & (c <= hi)), (seed, c, x)
        # co-located pairs of charge -+q, spread evenly over the cell
        assert np.all(np.abs(d["qw"]) == q)
        assert d["qw"].sum() == 0.0
        assert np.all(d["x1"] == 0.5)
        for j in range(nth):
            xs = np.sort(d["x2"][(d["qw"] > 0) & (np.floor(d["x2"]) == j)])
            np.testing.assert_allclose(xs, j + (np.arange(len(xs)) + 0.5) / max(len(xs), 1), atol=1e-15)
        assert o.counters()["capped"] == 0
        assert o.counters()["next_id"] == 2 * cap * nth
        total += c
    # mean over seeds: the expected count, within 5 standard errors per cell
    f = x - np.floor(x)
    se = np.sqrt(np.maximum(f * (1 - f), 1e-12) / seeds)
    assert np.all(np.abs(total / seeds - x) <= 5 * se + 1e-12), (total / seeds - x) / se
    z = (total - seeds * x).sum() / math.sqrt(seeds * (f * (1 - f)).sum())
    assert abs(z) < 5, z


def test_variable_counts_above_the_cap_are_cut_and_counted(oracle_mod):
    nth, q, cap = 32, 0.002, 3
    o = _rotator(nth, inject=2, inject_q=q, inject_seed=7, pairs_per_cell=cap)
    sig, dA = _monopole_sigma(o, nth)
    x = FIN * np.abs(sig) * dA / q
    c = _counts(o.particles(), nth)
    assert np.all(c <= cap)
    assert np.all(c[x >= cap] == cap)
    capped = o.counters()["capped"]
    assert (x >= cap + 1).sum() <= capped <= (x > cap).sum()


@pytest.mark.parametrize("passes", [1, 3])
def test_sigma_smoothing_keeps_linear_profiles_and_mirrors_at_the_poles(oracle_mod, passes):
    nth, npp = 32, 2
    o = _rotator(nth, inject_smooth=passes)
    sig, dA = _monopole_sigma(o, nth)  # exactly linear in j on the equal-area grid
    d = o.particles()
    pos = d["qw"] > 0
    j = np.floor(d["x2"][pos]).astype(int)
    w = np.zeros(nth)
    w[j] = d["qw"][pos]  # one charge per cell (all pairs of a cell are equal)
    inner = slice(passes, nth - passes)
    expect = FIN * np.abs(sig) * dA / npp
    # the equator cells have sigma = 0 up to rounding: compare where it is not
    big = np.abs(sig) > 1e-6 * np.abs(sig).max()
    sel = np.zeros(nth, bool)
    sel[inner] = True
    np.testing.assert_allclose(w[sel & big], expect[sel & big], rtol=1e-12)
    if passes == 1:
        s0 = (3 * sig[0] + sig[1]) / 4
        s1 = (3 * sig[-1] + sig[-2]) / 4
        assert w[0] == pytest.approx(FIN * abs(s0) * dA[0] / npp, rel=1e-12)
        assert w[-1] == pytest.approx(FIN * abs(s1) * dA[-1] / npp, rel=1e-12)
        assert abs(w[0] - expect[0]) > 1e-3 * expect[0]  # the pole cell did change


def _dipole(**kw):
    base = dict(nr=16, nth=24, r_min=R0, r_max=10.0, r_map="log", th_map="equal_area", vacuum="dipole_rotator",
                b0=B0, omega=OM, t_spin=4.0)
    base.update(kw)
    p = O.params(**base)
    p.dt = courant_dt(p, 0.5)
    return O.Oracle(p)


def test_dipole_rotator_fields(oracle_mod):
    o = _dipole()
    t, h, mu = 10.0, 1e-5, B0 * R0**3

    def phi(r, th):
        return -OM * mu * R0**2 / (3 * r**3) * (3 * math.cos(th) ** 2 - 1)

    def field(r, th):
        x1, x2 = float(o.f_r_inv(r)), float(o.f_th_inv(th))
        return o.vacuum(x1, x2, t)

    for r, th in ((1.7, 0.4), (4.2, 1.3), (8.5, 2.6)):
        E, B = field(r, th)
        assert E[0] == pytest.approx(-(phi(r + h, th) - phi(r - h, th)) / (2 * h), rel=1e-7)
        assert E[1] == pytest.approx(-(phi(r, th + h) - phi(r, th - h)) / (2 * h * r), rel=1e-7)
        assert E[2] == 0.0 and B[2] == 0.0
        assert B[0] == pytest.approx(2 * mu * math.cos(th) / r**3, rel=1e-14)
        assert B[1] == pytest.approx(mu * math.sin(th) / r**3, rel=1e-14)
        # the potential is harmonic: (1/r^2) d_r (r^2 d_r phi) + (1/(r^2 sin)) d_th (sin d_th phi) = 0
        g = 1e-3
        lap = ((r + g) ** 2 * (phi(r + 2 * g, th) - phi(r, th)) - (r - g) ** 2 * (phi(r, th) - phi(r - 2 * g, th))) / (
            4 * g * g * r * r)
        lap += (math.sin(th + g) * (phi(r, th + 2 * g) - phi(r, th)) - math.sin(th - g) * (phi(r, th) - phi(r, th - 2 * g))) / (
            4 * g * g * r * r * math.sin(th))
        assert abs(lap) < 1e-4 * 6 * abs(phi(r, th)) / r**2  # each of the two terms is 6 phi / r^2
    # no net charge: the flux of E through any sphere outside vanishes
    for r in (1.5, 6.0):
        flux = quad(lambda th: field(r, th)[0][0] * 2 * math.pi * r * r * math.sin(th), 0, math.pi)[0]
        scale = quad(lambda th: abs(field(r, th)[0][0]) * 2 * math.pi * r * r * math.sin(th), 0, math.pi)[0]
        assert abs(flux) < 1e-12 * scale
    # inside: corotation field, perpendicular to B
    x1, x2 = -0.4, 7.3
    r, th = float(o.f_r(x1)), float(o.f_th(x2))
    E, B = o.vacuum(x1, x2, t)
    pos = r * np.array([math.sin(th), 0.0, math.cos(th)])
    rhat, thhat = pos / r, np.array([math.cos(th), 0.0, -math.sin(th)])
    Bc = B[0] * rhat + B[1] * thhat
    Ec = -np.cross(np.cross([0.0, 0.0, OM], pos), Bc)
    assert E[0] == pytest.approx(Ec @ rhat, rel=1e-13)
    assert E[1] == pytest.approx(Ec @ thhat, rel=1e-13)
    assert abs(E[0] * B[0] + E[1] * B[1]) < 1e-14 * math.hypot(*E[:2]) * math.hypot(*B[:2])
    # tangential E continuous across r0; linear spin-up
    Ei, _ = o.vacuum(-1e-12, 5.0, t)
    Eo, _ = o.vacuum(0.0, 5.0, t)
    assert Ei[1] == pytest.approx(Eo[1], rel=1e-9)
    Eh, _ = o.vacuum(3.2, 2.5, 2.0)
    Ef, _ = o.vacuum(3.2, 2.5, 10.0)
    assert Eh[0] == pytest.approx(0.5 * Ef[0], rel=1e-14)


def test_dipole_rotator_injects_the_surface_charge(oracle_mod):
    """Fixed-count injection on the dipole rotator: the injected charge is
    f_inj times the integral of |E_r,out(r_1/2) - E_r,in(r0)| over the star,
    E_r,out = -Omega mu r0^2 (3 cos^2 - 1) / r^4 and E_r,in = Omega mu sin^2 / r0^2."""
    nth = 256
    o = _dipole(nth=nth, t_spin=0.0, inject=1, pairs_per_cell=2, f_inj=FIN, th_map="linear")
    o.step(1)
    d = o.particles()
    rb, mu = float(o.f_r(0.5)), B0 * R0**3

    def sigma(th):
        c, s = math.cos(th), math.sin(th)
        return -OM * mu * R0**2 * (3 * c * c - 1) / rb**4 - OM * mu * s * s / R0**2

    expect = FIN * quad(lambda th: abs(sigma(th)) * 2 * math.pi * R0**2 * math.sin(th), 0, math.pi, limit=200)[0]
    assert d["qw"][d["qw"] > 0].sum() == pytest.approx(expect, rel=2e-3)
