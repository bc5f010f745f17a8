"""The five workloads of the hot path as plain descriptor values and plasma recipes.

Physics scales the paper leaves open are set from dimensionless numbers:
B0 from omega_c(r0) dt, the preloaded macro-charge from omega_p(r0) dt using the
volume of the equatorial cell next to the star.  These only pick input values;
the method itself runs in the library (GPU) or in the oracle (CPU tests).
"""
from __future__ import annotations

import math

CONFIGS = {
    # small monopole plasma, plain FP64 path
    "monopole-64x64": dict(
        nr=64, nth=64, r_min=1.0, r_max=10.0, r_map="log", th_map="linear", courant=0.5, n_filt=0,
        absorb_cells=8, absorb_profile="linear", vacuum="monopole", omega=0.0, t_spin=0.0, inject=0,
        pusher="vay", precision="fp64", pairs_per_cell=12, T=0.1, seed=0, steps=100, wc_dt=0.5, wp_dt=0.05),
    # monopole rotator with injection, FP64 path
    "rotator-512x512": dict(
        nr=512, nth=512, r_min=1.0, r_max=40.0, r_map="log", th_map="equal_area", courant=0.5, n_filt=3,
        absorb_cells=32, absorb_profile="quadratic", vacuum="monopole_rotator", omega=0.2,
        t_spin=0.5 * 2 * math.pi / 0.2, inject=1, inject_pairs=2, f_inj=0.5, pusher="vay", precision="fp64",
        pairs_per_cell=38, T=0.1, seed=0, steps=2000, wc_dt=4.0, wp_dt=0.05),
    # precision variant of the rotator at 1024^2, 1e8 particles
    "rotator-1024x1024": dict(
        nr=1024, nth=1024, r_min=1.0, r_max=40.0, r_map="log", th_map="equal_area", courant=0.5, n_filt=3,
        absorb_cells=32, absorb_profile="quadratic", vacuum="monopole_rotator", omega=0.2,
        t_spin=0.5 * 2 * math.pi / 0.2, inject=1, inject_pairs=2, f_inj=0.5, pusher="vay", precision="fp32",
        pairs_per_cell=48, T=0.1, seed=0, steps=100, wc_dt=4.0, wp_dt=0.05),
    # large single run, FP32 path
    "monopole-4096x4096": dict(
        nr=4096, nth=4096, r_min=1.0, r_max=100.0, r_map="log", th_map="linear", courant=0.5, n_filt=0,
        absorb_cells=32, absorb_profile="linear", vacuum="monopole", omega=0.0, t_spin=0.0, inject=0,
        pusher="vay", precision="fp32", pairs_per_cell=30, T=0.3, seed=0, steps=200, sort_interval=20,
        wc_dt=0.5, wp_dt=0.05),
    # the large run's plasma on a 1024^2 grid (6.3e7 particles, 2.3 GB of FP32
    # state): the small case for hardware-counter captures of the same kernel
    "monopole-1024x1024": dict(
        nr=1024, nth=1024, r_min=1.0, r_max=100.0, r_map="log", th_map="linear", courant=0.5, n_filt=0,
        absorb_cells=32, absorb_profile="linear", vacuum="monopole", omega=0.0, t_spin=0.0, inject=0,
        pusher="vay", precision="fp32", pairs_per_cell=30, T=0.3, seed=0, steps=200, sort_interval=20,
        wc_dt=0.5, wp_dt=0.05),
}


def _fr(cfg, x):
    if cfg["r_map"] == "log":
        return cfg["r_min"] * math.exp(x * math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"])
    return cfg["r_min"] + x * (cfg["r_max"] - cfg["r_min"]) / cfg["nr"]


def _cos_th(cfg, x):
    if cfg["th_map"] == "equal_area":
        return 1.0 - 2.0 * x / cfg["nth"]
    return math.cos(math.pi * x / cfg["nth"])


def physics(cfg: dict, dt: float, q_over_m: float = 1.0):
    """(b0, |qw|) for the config at time step dt."""
    b0 = cfg["wc_dt"] / (dt * q_over_m)
    j = cfg["nth"] // 2  # equatorial cell (upper edge at the equator for even nth)
    vol = 2 * math.pi / 3 * (_fr(cfg, 1) ** 3 - _fr(cfg, 0) ** 3) * (_cos_th(cfg, j - 1) - _cos_th(cfg, j))
    n_in_cell = 2 * max(cfg["pairs_per_cell"], 1)
    wp = cfg["wp_dt"] / dt
    qw = wp * wp * vol / (n_in_cell * q_over_m)
    return b0, qw


def desc_kwargs(cfg: dict, dt: float, b0: float, **over):
    """Keyword arguments of picsar.make_desc for a config."""
    kw = dict(nr=cfg["nr"], nth=cfg["nth"], r_min=cfg["r_min"], r_max=cfg["r_max"], r_map=cfg["r_map"],
              th_map=cfg["th_map"], dt=dt, n_filt=cfg["n_filt"], absorb_cells=cfg["absorb_cells"],
              absorb_profile=cfg["absorb_profile"], vacuum=cfg["vacuum"], b0=b0, omega=cfg["omega"],
              t_spin=cfg["t_spin"], inject=cfg["inject"], pairs_per_cell=cfg.get("inject_pairs", 2),
              f_inj=cfg.get("f_inj", 0.0), precision=cfg["precision"], pusher=cfg["pusher"], q_over_m=1.0,
              sort_interval=cfg.get("sort_interval", 20), tile_shape=cfg.get("tile_shape", 0),
              inject_smooth=cfg.get("inject_smooth", 0), inject_q=cfg.get("inject_q", 0.0),
              inject_seed=cfg.get("inject_seed", 0))
    kw.update(over)
    return kw


def ensemble_member_config(m: int) -> dict:
    """Member m of the batched ensemble: the small monopole plasma's physics
    (log r in [1, 10], linear theta, lossy 8 cells) on the member's grid, FP32."""
    from .synthetic import ensemble_member

    r = ensemble_member(m)
    return dict(CONFIGS["monopole-64x64"], nr=r["nr"], nth=r["nth"], T=r["T"], seed=r["seed"],
                particles=r["particles"], precision="fp32", steps=200)


def oracle_kwargs(cfg: dict, dt: float, b0: float, **over):
    """Keyword arguments of oracle.params for a config."""
    kw = dict(nr=cfg["nr"], nth=cfg["nth"], r_min=cfg["r_min"], r_max=cfg["r_max"], r_map=cfg["r_map"],
              th_map=cfg["th_map"], dt=dt, n_filt=cfg["n_filt"], absorb_cells=cfg["absorb_cells"],
              absorb_profile=cfg["absorb_profile"], vacuum=cfg["vacuum"], b0=b0, omega=cfg["omega"],
              t_spin=cfg["t_spin"], inject=cfg["inject"], pairs_per_cell=cfg.get("inject_pairs", 2),
              f_inj=cfg.get("f_inj", 0.0), pusher=cfg["pusher"], q_over_m=1.0,
              inject_smooth=cfg.get("inject_smooth", 0), inject_q=cfg.get("inject_q", 0.0),
              inject_seed=cfg.get("inject_seed", 0))
    kw.update(over)
    return kw


def courant_dt(cfg: dict) -> float:
    """dt = courant * min over domain cells of min(dr, r_inner dtheta)."""
    import numpy as np

    i = np.arange(cfg["nr"] + 1, dtype=np.float64)
    if cfg["r_map"] == "log":
        r = cfg["r_min"] * np.exp(i * math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"])
    else:
        r = cfg["r_min"] + i * (cfg["r_max"] - cfg["r_min"]) / cfg["nr"]
    j = np.arange(cfg["nth"] + 1, dtype=np.float64)
    th = np.arccos(1.0 - 2.0 * j / cfg["nth"]) if cfg["th_map"] == "equal_area" else math.pi * j / cfg["nth"]
    dr = np.diff(r)
    dth = np.diff(th)
    m = min(dr.min(), (r[:-1] * dth.min()).min())
    return cfg["courant"] * float(m)
