"""The paper's test problems (Sec. 4) run through the C-ABI on both GPU paths.

* E1, Sec. 4.1: the l = 1 TM mode between the 1st and 4th roots of du_1/dr
  converges at second order in all four coordinate systems; the GPU's field
  solve equals the oracle's to 1e-12.
* E2, Sec. 4.2.1: a pair shot along the equator at -+0.95c is deleted at the
  predicted steps, and the inverse-square E_r of the charge left on the star
  is established within 2 % once the transient has left (4 t_c).
* E3, Sec. 4.2.2: the same pair next to the polar axis rings along the axis
  in spherical coordinates (measured 22 times the field at 3.5 t_c) and not
  in equal-area coordinates (0.13 %).
* E4, Sec. 4.3: a particle at rest at 3 r0 in the dipole + corotation field
  drifts at 0.15c within 2 % with the Vay pusher for omega_c dt from 0.1 to
  50; the Boris pusher does so at 0.1 and departs from it at 50.

Each run is compared with the oracle on the same input: fields within 1e-12
(FP64 path) or 1e-5 (FP32 path) relative, deletion steps exact; the one
ill-conditioned case (FP32, axis pair, spherical coordinates) is held to 1e-4,
for the reason given at E3.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.oracle import courant_dt
from paper_1407_1810_gb300 import configs

from gpu_common import KEYS, rel_l2, setup

pytestmark = pytest.mark.gpu
FIELD_TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()
    O.build_oracle()


def _cfg(**kw):
    base = dict(configs.CONFIGS["monopole-64x64"], vacuum="none", absorb_profile="none", absorb_cells=0,
                pairs_per_cell=0, n_filt=0, inject=0)
    base.update(kw)
    return base


def _particles(**cols):
    return {k: np.asarray(cols[k], dtype=np.float64) for k in KEYS}


# E1 ---------------------------------------------------------------------------

def _du1(r):
    return np.cos(r) / r - np.sin(r) / r**2 + np.sin(r)


def _du1_roots():
    from scipy.optimize import brentq

    return brentq(_du1, 2.5, 3.0), brentq(_du1, 12.0, 13.0)


def _tm_run(N, r_map, th_map):
    rin, rout = _du1_roots()
    cfg = _cfg(nr=N, nth=N, r_min=rin, r_max=rout, r_map=r_map, th_map=th_map, courant=0.5)
    p = O.params(**configs.oracle_kwargs(cfg, 0.0, 0.0))
    nsteps = int(math.ceil(1.25 / courant_dt(p, 0.5)))
    dt = 1.25 / nsteps
    s, o, _, _ = setup(cfg, plasma=_particles(**{k: [] for k in KEYS}), dt=dt)
    rb = o.f_r(np.arange(N) + 0.5)
    tb = o.f_th(np.arange(N) + 0.5)
    u1 = np.sin(rb) / rb - np.cos(rb)
    f = np.zeros(o.field_shape)
    f[5, :N, :N] = (u1 / rb)[:, None] * np.sin(tb)[None, :] * math.cos(0.5 * dt)  # B(-dt/2), E(0) = 0
    s.set_fields(f)
    o.set_fields(f)
    s.step(nsteps)
    g = s.fields()
    exact = (u1 / rb)[:, None] * np.sin(tb)[None, :] * math.cos(1.25)
    w = rb[:, None] ** 2
    err = math.sqrt(np.sum(w * (g[5, :N, :N] - exact) ** 2) / np.sum(w * exact**2))
    if N == 32:
        o.field_step(nsteps)
        assert rel_l2(g, o.fields()) < 1e-12
    s.close()
    return err


@pytest.mark.parametrize("r_map,th_map", [("linear", "linear"), ("log", "equal_area"),
                                          ("log", "linear"), ("linear", "equal_area")])
def test_e1_tm_mode_second_order_on_gpu(r_map, th_map):
    errs = [_tm_run(N, r_map, th_map) for N in (16, 32, 64)]
    slope = 0.5 * math.log2(errs[0] / errs[2])
    assert errs[2] < 1e-2, errs
    assert abs(slope - 2.0) < 0.15, (errs, slope)


# E2, E3 -----------------------------------------------------------------------

N_PAIR, NF_PAIR, L_PAIR, TC = 64, 3, 16, 9.0


def _pair(precision, th_map, x2):
    cfg = _cfg(nr=N_PAIR, nth=N_PAIR, r_map="linear", th_map=th_map, n_filt=NF_PAIR, absorb_cells=L_PAIR,
               absorb_profile="linear", precision=precision)
    ur = 0.95 / math.sqrt(1 - 0.95**2)
    p = O.params(**configs.oracle_kwargs(cfg, 0.0, 0.0))
    x1 = float(O.Oracle(O.params(**configs.oracle_kwargs(cfg, courant_dt(p, 0.5), 0.0))).f_r_inv(5.5))
    Q = 1e-6
    plasma = _particles(x1=[x1, x1], x2=[x2, x2], ur=[-ur, ur], uth=[0, 0], uph=[0, 0], qw=[Q, -Q])
    s, o, plasma, dt = setup(cfg, plasma=plasma, precision=precision)
    return s, o, dt, Q, plasma


def _inverse_square(o, Q):
    rb = o.f_r(np.arange(N_PAIR) + 0.5)
    inner = slice(4, N_PAIR - L_PAIR - 4)
    return inner, Q / (4 * math.pi * rb[inner] ** 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("th_map", ["linear", "equal_area"])
def test_e2_equator_pair_deletion_and_inverse_square(precision, th_map):
    s, o, dt, Q, plasma = _pair(precision, th_map, N_PAIR / 2)
    x1 = plasma["x1"][0]
    r0 = o.f_r(x1)
    v = 0.95 * dt
    n_in = next(n for n in range(1, 10**6) if math.floor(o.f_r_inv(r0 - v * n)) < -(NF_PAIR + 1))
    n_out = next(n for n in range(1, 10**6) if math.floor(o.f_r_inv(r0 + v * n)) >= N_PAIR + NF_PAIR + 1)
    for n in range(1, max(n_in, n_out) + 1):
        s.step(1)
        o.step(1)
        ids = set(s.particles()["id"].tolist())
        assert (0 in ids) == (n < n_in), n
        assert (1 in ids) == (n < n_out), n
        assert ids == set(o.particles()["id"].tolist()), n
    rest = int(4.0 * TC / dt) - max(n_in, n_out)
    s.step(rest)
    o.step(rest)
    f = s.fields()
    assert rel_l2(f, o.fields()) < FIELD_TOL[precision]
    inner, exact = _inverse_square(o, Q)
    err = np.max(np.abs(f[0, inner, :] - exact[:, None])) / np.max(exact)
    assert err < 0.02, err
    s.close()


# In spherical coordinates the axis ringing is ill-conditioned: on the oracle
# itself a 1e-6 cell shift of the pair's start moves the fields at 3.5 t_c by
# 8.9e-6 relative (6e-9 in equal-area coordinates), and the FP32 path's
# position rounding over the ~200 steps of flight is of that order; measured
# 4.7e-5 against the oracle.  That case is held to 1e-4, and its ringing
# amplitude to the oracle's within 1 %.
E3_TOL = {("fp64", "linear"): 1e-12, ("fp64", "equal_area"): 1e-12,
          ("fp32", "linear"): 1e-4, ("fp32", "equal_area"): 1e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_e3_polar_axis_pair_rings_only_in_spherical_coordinates(precision):
    dev = {}
    for th_map in ("linear", "equal_area"):
        s, o, dt, Q, _ = _pair(precision, th_map, 0.5)
        n = int(3.5 * TC / dt)
        s.step(n)
        o.step(n)
        f, fo = s.fields(), o.fields()
        assert rel_l2(f, fo) < E3_TOL[precision, th_map], th_map
        inner, exact = _inverse_square(o, Q)
        dev[th_map] = np.max(np.abs(f[0, inner, 0] - exact)) / np.max(exact)
        dev_o = np.max(np.abs(fo[0, inner, 0] - exact)) / np.max(exact)
        assert abs(dev[th_map] - dev_o) <= 0.01 * dev_o + 1e-4, (th_map, dev[th_map], dev_o)
        assert s.live() == 0
        s.close()
    assert dev["equal_area"] < 0.01, dev
    assert dev["linear"] > 1.0, dev


# E4 ---------------------------------------------------------------------------

def _drift(precision, pusher, wdt, nsteps=2000):
    """Mean v_ph / 0.15c of a particle at rest at 3 r0 on the equator of the
    dipole + corotation field with r0 / R_l = 0.05; omega_c held at 50 / dt_max
    (Larmor radius ~1e-4 r) and omega_c dt set through dt."""
    cfg = _cfg(nr=32, nth=32, r_map="log", th_map="linear", vacuum="dipole_corot", omega=0.05, pusher=pusher,
               precision=precision)
    p = O.params(**configs.oracle_kwargs(cfg, 0.0, 0.0))
    omega_c = 50.0 / courant_dt(p, 0.5)
    dt, b0 = wdt / omega_c, 27.0 * omega_c  # |B| at r = 3 on the equator is b0 / 27
    o0 = O.Oracle(O.params(**configs.oracle_kwargs(cfg, dt, b0)))
    x1 = float(o0.f_r_inv(3.0))
    plasma = _particles(x1=[x1], x2=[16.0], ur=[0], uth=[0], uph=[0], qw=[1e-12])
    s, o, _, _ = setup(cfg, plasma=plasma, precision=precision, dt=dt, b0=b0)
    vg, vo = [], []
    for _ in range(nsteps):
        s.step(1)
        o.step(1)
        for d, acc in ((s.particles(), vg), (o.particles(), vo)):
            u = np.array([d["ur"][0], d["uth"][0], d["uph"][0]])
            acc.append(u[2] / math.sqrt(1 + u @ u))
    s.close()
    return abs(np.mean(vg)) / 0.15, abs(np.mean(vo)) / 0.15


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_e4_exb_drift_vay_and_boris(precision):
    tol = 1e-9 if precision == "fp64" else 1e-3
    for wdt in (0.1, 1.0, 10.0, 50.0):
        g, r = _drift(precision, "vay", wdt)
        assert g == pytest.approx(1.0, abs=0.02), (wdt, g)
        assert abs(g - r) < tol, (wdt, g, r)
    g, r = _drift(precision, "boris", 0.1)
    assert g == pytest.approx(1.0, abs=0.02)
    assert abs(g - r) < tol
    g, r = _drift(precision, "boris", 50.0)
    assert abs(g - 1.0) > 0.05, g
    assert abs(g - r) < max(tol, 1e-6 if precision == "fp64" else 1e-2)
