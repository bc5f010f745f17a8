"""The steady-state diagnostics of paper_1407_1810_gb300.steady on exact
Michel fields (CPU, no GPU): a stand-in simulation holds the split-monopole
B_ph = -Omega r sin(theta) B_r at its staggered points and the radial charge
flux of the current r^2 J_r = -J0 r0^2 cos(theta) (Sec. 5.3, Eq. monosteady),
so the helpers must return the closed forms.
"""
import math

import numpy as np

from paper_1407_1810_gb300 import steady

CFG = dict(steady.ROTATOR_STEADY, nr=256, nth=128)
B0, OM, DT = 3.0, 0.2, 0.01


class _FakeSim:
    def __init__(self, fields=None, flux=None):
        self._f, self._F = fields, flux

    def fields(self):
        return self._f

    def flux(self):
        return self._F


def _grid():
    nr, nth = CFG["nr"], CFG["nth"]
    dxi = math.log(CFG["r_max"] / CFG["r_min"]) / nr
    return nr, nth, dxi


def test_michel_l0_closed_form():
    assert math.isclose(steady.michel_l0(B0, OM), 8 * math.pi / 3 * B0 ** 2 * OM ** 2, rel_tol=1e-15)
    assert math.isclose(steady.michel_l0(B0, OM, r0=2.0), 16 * steady.michel_l0(B0, OM), rel_tol=1e-15)


def test_bphi_over_br_recovers_the_michel_ratio():
    nr, nth, dxi = _grid()
    rh = CFG["r_min"] * np.exp((np.arange(nr + 1) + 0.5) * dxi)      # B_ph rows at i + 1/2
    th = np.arccos(1.0 - 2.0 * (np.arange(nth) + 0.5) / nth)         # and columns at j + 1/2
    f = np.zeros((6, nr + 1, nth + 1))
    f[5, :, :nth] = (-OM * rh[:, None] * np.sin(th)[None, :]) * (B0 / rh[:, None] ** 2)
    for r in (2.5, 5.0, 7.5):
        ri, t, ratio = steady.bphi_over_br(_FakeSim(fields=f), CFG, B0, r)
        assert abs(ri / r - 1) < dxi
        # B_ph averaged over i -+ 1/2 against B_r at node i: equal to O(dxi^2)
        np.testing.assert_allclose(ratio, -OM * ri * np.sin(t), rtol=2 * dxi ** 2)


def test_r2jr_recovers_the_michel_current():
    nr, nth, dxi = _grid()
    g = CFG["n_filt"] + 2
    j0r02 = 2.0 * B0 * OM * CFG["r_min"] ** 2
    ct = 1.0 - 2.0 * np.arange(nth + 1) / nth
    F = np.zeros((3, nr + 2 * g + 1, nth + 1))
    # charge through the dual face of (i + 1/2, j) per step: J_r dt dA with
    # dA = 2 pi r^2 dcos and r^2 J_r = -J0 r0^2 cos(theta_j)
    F[0, :, 1:nth] = (-j0r02 * ct[1:nth] * 2 * math.pi * DT * (2.0 / nth))[None, :]
    for r in (2.5, 5.0, 7.5):
        t, prof = steady.r2jr(F, CFG, B0, DT, r)
        np.testing.assert_allclose(prof, -np.cos(t), atol=1e-12)
