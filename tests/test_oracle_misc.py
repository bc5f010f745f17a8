"""Pins of the oracle's grid maps, analytic fields, gather and azimuthal flux.

* Sec. 3.2: the log map keeps dr/r constant, the equal-area map gives every
  meridional cell the same solid angle; inverses round-trip.
* Sec. 5.2: the outside "initial" field of the rotating monopole is the
  gradient of a dipole-type potential, the inside field is the corotation
  field -(Omega x r) x B, E_th is continuous across r0, and Omega ramps
  linearly over t_spin.
* gather (reading R2): bilinear interpolation reproduces fields that are
  linear in grid coordinates exactly, which fixes every component's stagger
  offset and the axis parity of the half-integer components.
* azimuthal flux (reading R4): the charge crossing the meridional half-plane
  equals qw * (swept azimuth) / 2 pi of the straight 3-D move.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.oracle import courant_dt


def _o(**kw):
    base = dict(nr=16, nth=12, r_min=1.0, r_max=10.0, r_map="log", th_map="equal_area", n_filt=0)
    base.update(kw)
    p = O.params(**base)
    p.dt = courant_dt(p, 0.5)
    return O.Oracle(p)


def test_maps(oracle_mod):
    o = _o()
    r = o.f_r(np.arange(17))
    assert np.allclose(r[1:] / r[:-1], (10.0) ** (1 / 16), rtol=1e-14)
    assert r[0] == 1.0 and r[-1] == pytest.approx(10.0, rel=1e-15)
    th = o.f_th(np.arange(13))
    # equal area: -cos(theta) uniform on [-1, 1]
    assert np.allclose(np.diff(-np.cos(th)), 2.0 / 12, atol=1e-15)
    x = np.linspace(-3, 19, 23)
    assert np.allclose(o.f_r_inv(o.f_r(x)), x, atol=1e-12)
    x2 = np.linspace(0, 12, 25)
    assert np.allclose(o.f_th_inv(o.f_th(x2)), x2, atol=1e-12)
    ol = _o(r_map="linear", th_map="linear")
    assert np.allclose(np.diff(ol.f_r(np.arange(17))), 9.0 / 16, atol=1e-14)
    assert np.allclose(np.diff(ol.f_th(np.arange(13))), math.pi / 12, atol=1e-15)


def test_rotator_vacuum_fields(oracle_mod):
    b0, om = 2.0, 0.2
    o = _o(vacuum="monopole_rotator", b0=b0, omega=om, t_spin=4.0)
    t = 10.0  # after spin-up
    h = 1e-6

    def phi(r, th):  # potential of the outside field
        return -b0 * om * math.cos(th) / r**2

    for x1, x2 in ((3.2, 2.5), (10.7, 7.1), (0.3, 11.0)):
        r, th = float(o.f_r(x1)), float(o.f_th(x2))
        E, B = o.vacuum(x1, x2, t)
        assert B[0] == pytest.approx(b0 / r**2, rel=1e-14)
        assert E[0] == pytest.approx(-(phi(r + h, th) - phi(r - h, th)) / (2 * h), rel=1e-7)
        assert E[1] == pytest.approx(-(phi(r, th + h) - phi(r, th - h)) / (2 * h * r), rel=1e-7)
    # inside the star: corotation field -(Omega x r) x B in Cartesian components
    x1, x2 = -1.3, 4.4
    r, th = float(o.f_r(x1)), float(o.f_th(x2))
    E, B = o.vacuum(x1, x2, t)
    pos = r * np.array([math.sin(th), 0.0, math.cos(th)])
    Bc = B[0] * pos / r
    Ec = -np.cross(np.cross([0.0, 0.0, om], pos), Bc)
    rhat, thhat = pos / r, np.array([math.cos(th), 0.0, -math.sin(th)])
    assert E[0] == pytest.approx(Ec @ rhat, abs=1e-14)
    assert E[1] == pytest.approx(Ec @ thhat, rel=1e-13)
    # tangential E is continuous across the conductor surface r = r0
    Ei, _ = o.vacuum(-1e-12, 3.0, t)
    Eo, _ = o.vacuum(0.0, 3.0, t)
    assert Ei[1] == pytest.approx(Eo[1], rel=1e-9)
    # linear spin-up
    Eh, _ = o.vacuum(3.2, 2.5, 2.0)
    Ef, _ = o.vacuum(3.2, 2.5, 10.0)
    assert Eh[0] == pytest.approx(0.5 * Ef[0], rel=1e-14)


def test_gather_reproduces_linear_fields(oracle_mod):
    nr, nth = 10, 8
    o = _o(nr=nr, nth=nth)
    # component c at its staggered point (a, b) holds c0 + c1 a + c2 b; odd
    # components vanish on the axis so their axisymmetric continuation is the
    # same linear function; B_r (even) is taken independent of x2.
    coef = {0: (1.0, 0.3, 0.2), 1: (0.0, 0.0, 0.7), 2: (0.0, 0.0, 0.0),
            3: (0.4, -0.2, 0.0), 4: (0.0, 0.0, 0.0), 5: (0.0, 0.0, -0.5)}
    stag = {0: (0.5, 0), 1: (0, 0.5), 2: (0, 0), 3: (0, 0.5), 4: (0.5, 0), 5: (0.5, 0.5)}
    f = np.zeros(o.field_shape)
    for c, (c0, c1, c2) in coef.items():
        si, sj = stag[c]
        ni = nr - 1 if si else nr
        nj = nth - 1 if sj else nth
        for i in range(ni + 1):
            for j in range(nj + 1):
                f[c, i, j] = c0 + c1 * (i + si) + c2 * (j + sj)
    # theta-odd quantities keep their sign pattern about the south pole too;
    # only the northern half is checked for them
    o.set_fields(f)
    rng = np.random.default_rng(1)
    for _ in range(200):
        x1 = rng.uniform(1.0, nr - 1.0)  # away from the conductors' zero ghosts
        x2 = rng.uniform(0.0, nth / 2)
        E, B = o.gather(x1, x2, 0.0)
        want = [coef[c][0] + coef[c][1] * x1 + coef[c][2] * x2 for c in range(6)]
        assert np.allclose(np.concatenate([E, B]), want, atol=1e-13), (x1, x2)


def test_azimuthal_flux_is_swept_angle(oracle_mod):
    o = _o(nr=16, nth=16, th_map="linear", vacuum="none")
    x1, x2 = 7.3, 5.6
    r, th = float(o.f_r(x1)), float(o.f_th(x2))
    R = r * math.sin(th)
    uph = 2.0
    v = uph / math.sqrt(1 + uph**2)
    qw = 0.37
    o.load([x1], [x2], [0.0], [0.0], [uph], [qw])
    o.step(1)
    F = o.flux()
    swept = math.atan2(v * o.p.dt, R)  # straight tangential chord from (R, 0)
    assert F[2].sum() == pytest.approx(qw * swept / (2 * math.pi), rel=1e-12)
    # angular momentum R u_phi is kept by the rotation back to phi = 0
    d = o.particles()
    r1, th1 = float(o.f_r(d["x1"][0])), float(o.f_th(d["x2"][0]))
    assert r1 * math.sin(th1) * d["uph"][0] == pytest.approx(R * uph, rel=1e-12)


def test_particles_only_is_the_particle_part_of_a_step(oracle_mod):
    """orc_particles_only moves, pushes, deposits and removes exactly as the
    particle part of orc_step does (with no filtering the step's fluxes are
    the raw deposit), and leaves the fields and the clock alone."""
    rng = np.random.default_rng(3)
    n = 400
    a, b = _o(vacuum="monopole", b0=2.0), _o(vacuum="monopole", b0=2.0)
    f = rng.normal(0, 0.1, a.field_shape)
    x1 = np.concatenate([rng.uniform(0, 16, n - 2), [-0.95, 16.95]])  # two leave the domain
    x2 = rng.uniform(0, 12, n)
    u = rng.normal(0, 0.5, (3, n))
    u[0, -2], u[0, -1] = -3.0, 3.0
    qw = np.where(np.arange(n) % 2 == 0, 0.01, -0.01)
    for o in (a, b):
        o.set_fields(f)
        o.load(x1, x2, u[0], u[1], u[2], qw)
        o.set_clock(4, n)
    fa = a.fields()
    assert a.particles_only() == 0 and b.step(1) == 0
    pa, pb = a.particles(), b.particles()
    assert len(pa["x1"]) < n
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    assert np.array_equal(a.flux(), b.flux())
    assert a.counters() == b.counters()
    assert np.array_equal(a.fields(), fa)
    assert a.lib.orc_get_step(a.h) == 4 and b.lib.orc_get_step(b.h) == 5


def test_total_fields_add_the_analytic_field_at_each_stagger(oracle_mod):
    """Sec. 5.2: the total field is the plasma field plus the analytic field,
    each component at its own staggered point of Eq. (offseteq) (E_r at
    (i+1/2, j), E_th at (i, j+1/2), B_r at (i, j+1/2)), at time step * dt."""
    b0, om = 2.0, 0.2
    o = _o(vacuum="monopole_rotator", b0=b0, omega=om, t_spin=0.0, nr=12, nth=10)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(o.field_shape)
    o.set_fields(f)
    f = o.fields()
    o.set_clock(7, 0)
    tot = o.fields(total=True)
    i, j = np.arange(o.nr + 1), np.arange(o.nth + 1)
    rn, rh = o.f_r(i), o.f_r(i + 0.5)
    tn, th = o.f_th(j), o.f_th(np.arange(o.nth) + 0.5)
    a = lambda r: b0 * om / r**3  # B0 r0^4 Omega / r^3 with r0 = 1
    N, M = o.nr, o.nth
    np.testing.assert_allclose(tot[0, :N, :] - f[0, :N, :], (-2 * a(rh[:N]))[:, None] * np.cos(tn)[None, :],
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(tot[1, :, :M] - f[1, :, :M], (-a(rn))[:, None] * np.sin(th[:M])[None, :],
                               rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(tot[3, :, :M] - f[3, :, :M], (b0 / rn**2)[:, None] * np.ones(M)[None, :], rtol=1e-13)
    for c in (2, 4, 5):
        np.testing.assert_array_equal(tot[c], f[c])
    # outside a component's range nothing is added
    assert np.array_equal(tot[0, N, :], f[0, N, :]) and np.array_equal(tot[1, :, M], f[1, :, M])


def _axis_crosser(uph, hints=None):
    """A particle 0.1 cell from the north axis moving straight towards and
    past it (u_th < 0; it moves 0.16 cell of arc), with a tiny azimuthal
    momentum uph; no fields."""
    o = _o(nr=16, nth=64, th_map="linear", vacuum="none")
    if hints is not None:
        o.set_axis_hints(hints)
    qw = 0.37
    o.load([7.3], [0.1], [0.0], [-3.0], [uph], [qw])
    o.step(1)
    return o, o.flux()[2].sum() / qw


def test_axis_crossing_tie_branch_and_hints(oracle_mod):
    """R15: the move crosses the axis (the displaced point lies past it) with
    |u_ph| far below 2^-13 |u|, so the swept azimuth is +-pi with the sign of
    u_ph: the two branches put +1/2 and -1/2 of the charge through the
    meridional half-plane.  Both are ties; a hint fixes the branch; a
    crossing with a larger u_ph is no tie and ignores the table."""
    for uph, half in ((1e-9, 0.5), (-1e-9, -0.5)):
        o, f = _axis_crosser(uph)
        assert o.axis_ties() == 1
        assert f == pytest.approx(half, abs=1e-6)
        assert 0.0 < o.particles()["x2"][0] < 0.1  # reflected through the axis to the other side
    step0 = {"step": [0], "id": [0], "sign": [1]}
    o, f = _axis_crosser(-1e-9, hints=step0)
    assert o.axis_ties() == 1 and f == pytest.approx(0.5, abs=1e-6)
    # a hint for another step or particle leaves the branch alone
    o, f = _axis_crosser(-1e-9, hints={"step": [1, 0], "id": [0, 5], "sign": [1, 1]})
    assert f == pytest.approx(-0.5, abs=1e-6)
    # |u_ph| = 0.017 |u|: no tie, hints ignored
    o, f = _axis_crosser(-0.05, hints=step0)
    assert o.axis_ties() == 0 and f < -0.49
