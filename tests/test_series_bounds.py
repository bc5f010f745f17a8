"""The grid bounds under which the FP32 step uses its short series without
the general fallback (dxi <= 1/16, dt / r <= 1/40; the context computes them
at creation): at those bounds every series' relative truncation, evaluated
in FP64, stays below 2^-28 = 1/16 of an FP32 ulp, so the series add nothing
to the step's FP32 rounding.  The series are the Taylor polynomials the step
evaluates: exp to y^5, log1p to s^6, atan to t^7 (odd), and sin / cos - 1 of
the turning angle to x^5 / x^6.  The same sin / cos - 1 series turn a column's
node angle to the particle's angle on the linear theta map of the monopole
specialisation (nth >= 32)."""
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


def _turned_node_angle(nth, cj, dy, pole_side=True):
    """sin th, cos th of the point (cj + dy) pi / nth of a linear theta map as
    the monopole step forms them, in FP32 operations (each rounded; the kernel
    fuses some of them, which only rounds less): the (sin, cos) of a column's
    node angle, rounded once to FP32 from FP64 as the context's table holds
    them, turned by the offset's angle b with the short series.  pole_side
    takes the node on the pole side of the particle's hemisphere (node cj,
    b >= 0 in the north; node cj + 1, b <= 0 in the south); without it node
    cj serves both hemispheres."""
    f = np.float32
    north = 2 * cj < nth if pole_side else np.ones_like(cj, bool)
    j = np.where(north, cj, cj + 1).astype(np.float64)
    m = np.minimum(j, nth - j)
    S = np.sin(np.pi * m / nth).astype(f)
    C = np.sin(np.pi * (nth - 2 * j) / (2 * nth)).astype(f)
    o = np.where(north, dy, dy - f(1)).astype(f)
    b = (o * f(np.pi / nth)).astype(f)
    x2 = b * b
    sb = b * (f(1) - x2 * (f(1 / 6) - x2 * f(1 / 120)))
    cb1 = (f(-0.5) * x2) * (f(1) - x2 * (f(1 / 12) - x2 * f(1 / 360)))
    st = C * sb + (S * cb1 + S)
    ct = -S * sb + (C * cb1 + C)
    return st.astype(np.float64), ct.astype(np.float64)


def _column_points(nth):
    """Columns and offsets (including both ends of a cell) with the exact
    sin th and cos th, each the sine of an angle measured from the nearer pole
    or from the equator: x2 = cj + dy and nth - x2 are exact in FP64, so the
    reference keeps full relative precision next to either pole."""
    dys = np.array([0.0, 2.0 ** -24, 1e-3, 0.25, 0.5, 0.75, 1 - 1e-3, 1 - 2.0 ** -24], np.float32)
    cj = np.repeat(np.arange(nth), len(dys))
    dy = np.tile(dys, nth)
    x2 = cj + dy.astype(np.float64)
    s_ref = np.sin(np.pi * np.minimum(x2, nth - x2) / nth)
    c_ref = np.sin(np.pi * (nth - 2 * x2) / (2 * nth))
    return cj, dy, s_ref, c_ref


def test_column_angle_series_at_the_bound():
    """nth >= 32 (the monopole specialisation's condition) keeps the turn's
    angle within pi / 32, where the sin / cos - 1 series truncate below 2^-28."""
    t = np.linspace(-np.pi / 32, np.pi / 32, 20001)
    t = t[t != 0]
    d2 = t * t
    sd = t * (1 - d2 * (1 / 6 - d2 / 120))
    cd1 = -0.5 * d2 * (1 - d2 * (1 / 12 - d2 / 360))
    ref = -2 * np.sin(t / 2) ** 2
    assert np.max(np.abs(sd - np.sin(t)) / np.abs(np.sin(t))) <= BOUND
    assert np.max(np.abs(cd1 - ref) / np.abs(ref)) <= BOUND


def test_turned_node_angle_keeps_sin_theta_relative_precision_to_the_poles():
    """With the pole-side node, sin th keeps a few FP32 ulps of relative
    precision everywhere, down to the last cells at both poles, and cos th a
    few ulps of absolute precision; node cj on both hemispheres loses the
    relative precision of sin th next to the south pole (cancellation)."""
    ulp = 2.0 ** -24
    for nth in (32, 64, 4096):
        cj, dy, s_ref, c_ref = _column_points(nth)
        st, ct = _turned_node_angle(nth, cj, dy)
        nz = s_ref > 0
        assert np.max(np.abs(st - s_ref)[nz] / s_ref[nz]) <= 4 * ulp, nth
        assert np.all(st[~nz] == 0.0)
        assert np.max(np.abs(ct - c_ref)) <= 3 * ulp, nth
    cj, dy, s_ref, _ = _column_points(4096)
    st, _ = _turned_node_angle(4096, cj, dy, pole_side=False)
    nz = s_ref > 0
    assert np.max(np.abs(st - s_ref)[nz] / s_ref[nz]) > 1e-3
