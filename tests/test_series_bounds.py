"""The grid bounds under which the FP32 step uses its short series without
the general fallback (dxi <= 1/16, dt / r <= 1/40; the context computes them
at creation): at those bounds every series' relative truncation, evaluated
in FP64, stays below 2^-28 = 1/16 of an FP32 ulp, so the series add nothing
to the step's FP32 rounding.  The series are the Taylor polynomials the step
evaluates: exp to y^5, log1p to s^6, atan to t^7 (odd), and sin / cos - 1 of
the turning angle to x^5 / x^6."""
import numpy as np

BOUND = 2.0 ** -28
DXI, EPS = 1.0 / 16, 1.0 / 40


def test_exp_series_at_the_cell_bound():
    y = np.linspace(-DXI, DXI, 100001)
    ser = 1 + y * (1 + y * (0.5 + y * (1 / 6 + y * (1 / 24 + y / 120))))
    assert np.max(np.abs(ser - np.exp(y)) / np.exp(y)) <= BOUND / 16


def test_log1p_series_at_the_step_bound():
    smax = 2 * EPS + 3 * EPS ** 2  # (r'/r)^2 - 1 with |dr|, |dt| <= eps r
    s = np.linspace(-smax, smax, 100001)
    s = s[s != 0]
    ser = s * (1 - s * (0.5 - s * (1 / 3 - s * (0.25 - s * (0.2 - s / 6)))))
    assert np.max(np.abs(ser - np.log1p(s)) / np.abs(np.log1p(s))) <= BOUND


def test_atan_and_rotation_series_at_the_step_bound():
    t = np.linspace(-1.1 * EPS, 1.1 * EPS, 20001)
    t = t[t != 0]
    at = t * (1 - t * t * (1 / 3 - t * t * (0.2 - t * t / 7)))
    assert np.max(np.abs(at - np.arctan(t)) / np.abs(np.arctan(t))) <= BOUND / 1000
    d2 = t * t
    sd = t * (1 - d2 * (1 / 6 - d2 / 120))
    cd1 = -0.5 * d2 * (1 - d2 * (1 / 12 - d2 / 360))
    ref = -2 * np.sin(t / 2) ** 2  # cos t - 1 without cancellation
    assert np.max(np.abs(sd - np.sin(t)) / np.abs(np.sin(t))) <= BOUND / 1000
    assert np.max(np.abs(cd1 - ref) / np.abs(ref)) <= BOUND / 1000


def test_the_bounds_exclude_what_would_exceed():
    """Just past the log1p bound the truncation passes 2^-28: the bound on
    dt / r is the binding one."""
    eps = 1.0 / 30
    smax = 2 * eps + 3 * eps ** 2
    ser = smax * (1 - smax * (0.5 - smax * (1 / 3 - smax * (0.25 - smax * (0.2 - smax / 6)))))
    assert abs(ser - np.log1p(smax)) / np.log1p(smax) > BOUND
