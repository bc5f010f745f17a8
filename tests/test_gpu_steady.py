"""The aligned monopole rotator of Table 1 run to its steady state (Sec. 5.3).

1024 x 512 cells, log r over [1, 54] r0, equal-area theta, R_l = 5 r0,
Courant 0.6, two rotation periods (26830 steps, ~20 s on a GB300), plasma
from surface injection only.  The paper finds the spin-down luminosity
through spheres out to 25 r0 within ~1 % of the force-free value L0 and
B_ph / B_r on the split-monopole (Michel) curve -Omega r sin(theta); it ends
with ~2e7 particles.  This implementation measures L / L0 = 0.969-0.983 over
r in [1.5, 25] r0 (mean 0.977; 0.979 after three periods, 0.980 with a field
twice as strong), B_ph / B_r at 98.6-98.8 % of the Michel value at R_l / 2,
R_l and 3 R_l / 2, r^2 J_r on -J0 cos(theta) to a scale of 0.989, and
1.98e7 particles.  The bars hold those results: L / L0 within 4 %, B_ph / B_r
within 3 % (median over the cells away from the axis), r^2 J_r within 3 % in
scale and 0.06 J0 rms over theta bins,
the particle count within 25 % of the paper's, Gauss's law to 1e-6.  The
last test finds the cause of the ~2 % luminosity deficit (the rate at which
the surface charge is released) and holds the f_inj = 1 run to 1 %.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def steady_run():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build, steady

    build.build()
    torch.cuda.set_device(0)
    return steady.run()


def test_spindown_luminosity_matches_the_force_free_value(steady_run):
    r, L = steady_run["r"], steady_run["L_over_L0"]
    sel = (r >= 1.5) & (r <= 25.0)
    assert np.all(np.abs(L[sel] - 1.0) <= 0.04), (L[sel].min(), L[sel].max())
    assert L[sel].max() - L[sel].min() <= 0.03  # approximately constant with radius


def test_bphi_over_br_follows_michel(steady_run):
    for name, p in steady_run["bphi"].items():
        mid = (p["theta"] > 0.3) & (p["theta"] < math.pi - 0.3)
        ratio = np.median(p["bphi_over_br"][mid] / p["michel"][mid])
        assert abs(ratio - 1.0) <= 0.03, (name, ratio)


def test_radial_current_follows_michel(steady_run):
    """r^2 J_r = -J0 r0^2 cos(theta) (Fig. 7a) from the radial charge flux
    averaged over ~50 steps: measured best-fit scale 0.989 and rms deviation
    0.034 J0 over bins of 16 theta nodes (shot noise of the sampled steps)."""
    for name, p in steady_run["bphi"].items():
        t, jr = p["theta_j"], p["r2jr"]
        c = np.cos(t)
        scale = -(jr @ c) / (c @ c)
        assert abs(scale - 1.0) <= 0.03, (name, scale)
        n = len(t) // 16 * 16
        dev = jr[:n].reshape(-1, 16).mean(1) + c[:n].reshape(-1, 16).mean(1)
        assert np.sqrt(np.mean(dev ** 2)) <= 0.06, (name, dev)


def test_energy_flux_is_conserved_across_radii(steady_run):
    """The Poynting flux falls outward as the plasma gains energy; Poynting
    plus the particles' kinetic energy flux is the same through every sphere
    in [1.5, 25] r0 (measured 0.988-0.990 of L0), and the particles reach a
    median gamma of 23.7 beyond 2 r0 (the paper: about 28)."""
    r, L = steady_run["r"], steady_run["L_over_L0"]
    rad, lp = steady_run["lp_radii"], steady_run["Lp_over_L0"]
    total = np.array([L[np.argmin(np.abs(r - x))] for x in rad]) + lp
    assert np.all(np.abs(total - 1.0) <= 0.03), total
    assert total.max() - total.min() <= 0.01, total
    assert np.all(lp > 0) and lp[-1] > lp[0]  # the plasma carries energy outward and gains it
    assert 15.0 <= steady_run["gamma_median"] <= 45.0, steady_run["gamma_median"]


def test_plasma_is_charge_separated_by_hemisphere(steady_run):
    """Fig. 7c: surface injection gives a charge-separated plasma.  Beyond
    2 r0 the charge is mostly negative in the northern hemisphere and mostly
    positive in the southern one, the sign of -2 Omega.B for the monopole
    (measured: 29.8 % and 70.5 % of the charge positive), mirror images of
    each other."""
    sh = steady_run["positive_share"]
    assert sh["north"] < 0.4 and sh["south"] > 0.6, sh
    assert abs(sh["north"] + sh["south"] - 1.0) < 0.02, sh


def test_particle_count_and_gauss(steady_run):
    assert 1.5e7 <= steady_run["particles"] <= 2.5e7, steady_run["particles"]
    assert steady_run["gauss_residual"] <= 1e-6


def test_full_injection_reaches_the_force_free_luminosity():
    """The 2.3 % deficit of the f_inj = 0.5 run is the surface-charge supply:
    one change at a time, a lossy layer of 64 cells or with the linear
    profile, 1 or 4 pairs per cell, an averaging window four times longer and
    a field twice as strong move the mean L / L0 by at most 0.4 %, while
    releasing the whole surface charge every step (f_inj = 1) gives
    L / L0 = 0.999 (0.983-1.005 over [1.5, 25] r0), within the paper's ~1 %
    (the paper: f_inj closer to unity agrees better with the analytic
    solution, Sec. 5.3)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import steady

    res = steady.run(dict(steady.ROTATOR_STEADY, f_inj=1.0))
    r, L = res["r"], res["L_over_L0"]
    sel = (r >= 1.5) & (r <= 25.0)
    assert abs(L[sel].mean() - 1.0) <= 0.01, L[sel].mean()
    assert np.all(np.abs(L[sel] - 1.0) <= 0.025), (L[sel].min(), L[sel].max())
    assert res["gauss_residual"] <= 1e-6


def test_luminosity_and_lorentz_factor_together():
    """Table 1 fixes f_inj = 0.5 but not the field strength B0 (only that the
    gyro-radius of the gamma ~ 28 particles stays below a cell at the
    surface).  Faster charge release raises L / L0 and lowers the median
    gamma, a stronger field raises gamma: with f_inj = 0.8 and
    omega_c dt = 160 the run has both the paper's results at once -- L / L0 =
    0.989 (0.986-0.992 over [1.5, 25] r0) and a median gamma of 32 beyond
    2 r0, with 2.5e7 particles (the paper: ~1 %, gamma ~ 28, ~2e7)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import steady

    res = steady.run(dict(steady.ROTATOR_STEADY, f_inj=0.8, wc_dt=160.0))
    r, L = res["r"], res["L_over_L0"]
    sel = (r >= 1.5) & (r <= 25.0)
    assert abs(L[sel].mean() - 1.0) <= 0.015, L[sel].mean()
    assert np.all(np.abs(L[sel] - 1.0) <= 0.025), (L[sel].min(), L[sel].max())
    assert 20.0 <= res["gamma_median"] <= 40.0, res["gamma_median"]
    assert 1.5e7 <= res["particles"] <= 3.5e7, res["particles"]
    assert res["gauss_residual"] <= 1e-6
