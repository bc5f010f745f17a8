"""Helpers shared by the GPU parity tests: build both sides from one config."""
from __future__ import annotations

import numpy as np

import oracle as O
from oracle.oracle import courant_dt
from paper_1407_1810_gb300 import configs, synthetic

KEYS = ("x1", "x2", "ur", "uth", "uph", "qw")


def fp32_state(d):
    """The FP32 path stores x as (cell, FP32 offset) and u, qw in FP32; this is
    the exact FP64 value of that state, which both sides then start from."""
    out = dict(d)
    for k in ("x1", "x2"):
        c = np.floor(d[k])
        out[k] = c + (d[k] - c).astype(np.float32).astype(np.float64)
    for k in ("ur", "uth", "uph", "qw"):
        out[k] = d[k].astype(np.float32).astype(np.float64)
    return out


def setup(cfg: dict, plasma: dict | None = None, precision: str | None = None, **over):
    """(gpu Simulation, oracle, plasma dict, dt) for a config dict."""
    from paper_1407_1810_gb300 import picsar as P

    prec = precision or cfg["precision"]
    ok = configs.oracle_kwargs(cfg, 0.0, 0.0)
    ok.update({k: v for k, v in over.items() if k in ok})
    p = O.params(**ok)
    dt = over.get("dt") or courant_dt(p, cfg["courant"])
    b0, qw = configs.physics(cfg, dt)
    if "b0" in over:
        b0 = over["b0"]
    p.dt, p.b0 = dt, b0
    o = O.Oracle(p)
    dk = configs.desc_kwargs(cfg, dt, b0, precision=prec)
    dk.update({k: v for k, v in over.items() if k in dk})
    s = P.Simulation(P.make_desc(**dk))
    if plasma is None:
        plasma = synthetic.pair_plasma(cfg["nr"], cfg["nth"], cfg["pairs_per_cell"], cfg["T"], qw, cfg["seed"])
    if prec == "fp32":
        plasma = fp32_state(plasma)
    if len(plasma["x1"]):
        o.load(*(plasma[k] for k in KEYS))
        s.load(*(np.ascontiguousarray(plasma[k]) for k in KEYS))
    return s, o, plasma, dt


# element-wise bars (per-component max-norm relative to that component's
# largest value) beside the relative L2 bars of the two paths.  On a grid
# with spherical (linear) theta the cells next to the polar axis are tiny and
# magnify any perturbation: there the FP32 path's fields after 100 steps sit
# at 7.9e-4 element-wise on the 40 x 32 rotator, against 6.9e-5 for the
# oracle whose own state is rounded to FP32 storage every step and 5.8e-6 for
# the oracle from a start 6e-8 cell apart (FP32 arithmetic near the axis adds
# to the storage rounding), so those comparisons take MAX_FP32_SPHERICAL.
MAX_FP64 = 1e-10
MAX_FP32 = 1e-4
MAX_FP32_SPHERICAL = 1e-3


def close(a, b, l2, mx):
    """Both checks of stacked planes (fields or fluxes) at once: relative L2
    below l2 and the per-component max-norm below mx."""
    e2, em = rel_l2(a, b), maxnorm_rel(a, b)
    assert e2 < l2, ("rel_l2", e2, l2)
    assert em < mx, ("maxnorm", em, mx)
    return e2, em


def follow_ties(src, dst):
    """dst (an oracle or a GPU context) takes src's branch at every
    axis-crossing tie src logged (reading R15 of the oracle): a replay of src
    then follows src where the sign of a vanishing u_ph is set by rounding."""
    dst.set_axis_hints(src.axis_ties())


def by_id(d):
    order = np.argsort(d["id"])
    return {k: v[order] for k, v in d.items()}


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def maxnorm_rel(a, b):
    """Element-wise check of stacked planes (fields or fluxes): the largest
    |a - b| of each component relative to that component's own largest |b|,
    maximised over the components.  A localised error that a global L2 norm
    would average away shows up here."""
    out = 0.0
    for c in range(a.shape[0]):
        den = float(np.max(np.abs(b[c])))
        num = float(np.max(np.abs(a[c] - b[c])))
        out = max(out, num / den if den > 0 else num)
    return out


def replay_compare_fp32(g, r, tau):
    """Compare the FP32 path's step with the oracle's replay of it, both given
    as particle dicts.  Removals agree: ids kept by one side only (a removal
    decided on a coordinate within rounding of the boundary) count with the
    near-tie particles, which the oracle places within tau of a grid line and
    which may be at most 1e-4 of all; elsewhere cells agree exactly.
    Positions agree within tau, momenta within 2e-6 of |u| (+1e-2), charges
    exactly.  Returns the number of near-tie particles."""
    g, r = by_id(g), by_id(r)
    common = np.intersect1d(g["id"], r["id"])
    one_sided = len(g["id"]) + len(r["id"]) - 2 * len(common)
    g = {k: v[np.isin(g["id"], common)] for k, v in g.items()}
    r = {k: v[np.isin(r["id"], common)] for k, v in r.items()}
    tie = (np.abs(r["x1"] - np.round(r["x1"])) < tau) | (np.abs(r["x2"] - np.round(r["x2"])) < tau)
    ok = ~tie
    assert tie.sum() + one_sided <= max(1, 1e-4 * len(tie)), (tie.sum(), one_sided)
    assert np.array_equal(np.floor(g["x1"][ok]), np.floor(r["x1"][ok]))
    assert np.array_equal(np.floor(g["x2"][ok]), np.floor(r["x2"][ok]))
    assert np.max(np.abs(g["x1"] - r["x1"]), initial=0.0) < tau
    assert np.max(np.abs(g["x2"] - r["x2"]), initial=0.0) < tau
    umag = np.sqrt(r["ur"] ** 2 + r["uth"] ** 2 + r["uph"] ** 2) + 1e-2
    for k in ("ur", "uth", "uph"):
        assert np.max(np.abs(g[k] - r[k]) / umag, initial=0.0) < 2e-6, k
    assert np.array_equal(g["qw"], r["qw"])
    return int(tie.sum())
