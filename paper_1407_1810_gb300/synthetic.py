"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module draws random numbers only: particle positions in grid coordinates,
Maxwell-Juttner momenta and the ensemble member recipe.  It contains none of the
PIC method's arithmetic (no stretching functions, no metric, no push), so both
the GPU path and the CPU oracle can take its arrays as given inputs.

Recipe (matching the paper's workloads):
  * pair plasma: ``pairs_per_cell`` co-located e+/e- pairs in every cell of a
    block of cells, each pair at a uniform random point of the cell in grid
    coordinates; equal weights; co-location makes the initial charge density
    exactly zero, as the paper's injected pairs are (Sec. 5.3).
  * momenta: isotropic Maxwell-Juttner with temperature T (units of m c^2),
    |u| drawn by inverting the tabulated CDF of u^2 exp(-sqrt(1+u^2)/T); each
    member of a pair gets its own momentum.
"""
from __future__ import annotations

import numpy as np


def _mj_table(T: float, n: int = 1 << 16):
    umax = max(40.0 * T + 10.0 * np.sqrt(T), 1.0)
    # the density falls like exp(-u/T) for large u: 40 T is far in the tail
    u = np.linspace(0.0, umax, n)
    pdf = u * u * np.exp(-(np.sqrt(1.0 + u * u) - 1.0) / T)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(u))])
    cdf /= cdf[-1]
    return cdf, u


def mj_momenta(n: int, T: float, rng: np.random.Generator):
    """n isotropic Maxwell-Juttner momenta u = gamma v (c = 1), shape (n, 3)."""
    cdf, ugrid = _mj_table(T)
    mag = np.interp(rng.random(n), cdf, ugrid)
    cosa = 2.0 * rng.random(n) - 1.0
    beta = 2.0 * np.pi * rng.random(n)
    sina = np.sqrt(np.maximum(0.0, 1.0 - cosa * cosa))
    return np.stack([mag * cosa, mag * sina * np.cos(beta), mag * sina * np.sin(beta)], axis=1)


def pair_plasma(nr: int, nth: int, pairs_per_cell: int, T: float, qw: float, seed: int,
                rows: tuple[int, int] | None = None, dtype=np.float64):
    """Co-located e+/e- pairs, ``pairs_per_cell`` per cell of rows x [0, nth).

    Returns a dict of arrays x1, x2, ur, uth, uph, qw (length 2 * pairs), with
    the positive member of each pair at even index and the negative at odd.
    """
    rng = np.random.default_rng(seed)
    r0, r1 = rows if rows is not None else (0, nr)
    ncell = (r1 - r0) * nth
    npair = ncell * pairs_per_cell
    cell = np.repeat(np.arange(ncell, dtype=np.int64), pairs_per_cell)
    ci = r0 + cell // nth
    cj = cell % nth
    ox = rng.random(npair)
    oy = rng.random(npair)
    x1 = np.repeat(ci + ox, 2)
    x2 = np.repeat(cj + oy, 2)
    u = mj_momenta(2 * npair, T, rng)
    q = np.tile(np.array([qw, -qw]), npair)
    out = {"x1": x1, "x2": x2, "ur": u[:, 0], "uth": u[:, 1], "uph": u[:, 2], "qw": q}
    return {k: np.ascontiguousarray(v, dtype=dtype) for k, v in out.items()}


def splitmix64(seed: int):
    """Stream of uniforms in [0, 1) from splitmix64 (Steele et al. 2014)."""
    mask = (1 << 64) - 1
    x = seed & mask
    while True:
        x = (x + 0x9E3779B97F4A7C15) & mask
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z = z ^ (z >> 31)
        yield (z >> 11) * (1.0 / (1 << 53))


def ensemble_member(m: int):
    """Grid and plasma recipe of ensemble member m (64 uneven vacuum-monopole plasmas)."""
    g = splitmix64(m)
    U, U2 = next(g), next(g)
    nr = (64, 128, 256)[m % 3]
    nth = (64, 128, 256, 512)[(m // 3) % 4]
    n = int(round(10 ** (4 + 2.301 * U)))
    T = 0.05 + 0.95 * U2
    return {"nr": nr, "nth": nth, "particles": n, "T": T, "seed": m}


def pair_plasma_cells(nr: int, nth: int, cells, pairs_per_cell: int, T: float, qw: float, seed: int,
                      dtype=np.float64):
    """As pair_plasma, restricted to the listed cells (flat indices i * nth + j
    counted from row 0); used to draw a bounded sample of a large workload."""
    rng = np.random.default_rng(seed)
    cells = np.asarray(cells, dtype=np.int64)
    npair = len(cells) * pairs_per_cell
    cell = np.repeat(cells, pairs_per_cell)
    ox, oy = rng.random(npair), rng.random(npair)
    x1 = np.repeat(cell // nth + ox, 2)
    x2 = np.repeat(cell % nth + oy, 2)
    u = mj_momenta(2 * npair, T, rng)
    q = np.tile(np.array([qw, -qw]), npair)
    out = {"x1": x1, "x2": x2, "ur": u[:, 0], "uth": u[:, 1], "uph": u[:, 2], "qw": q}
    return {k: np.ascontiguousarray(v, dtype=dtype) for k, v in out.items()}


def pair_plasma_torch(nr: int, nth: int, pairs_per_cell: int, T: float, qw: float, seed: int, device,
                      rows_per_chunk: int = 64):
    """The pair-plasma recipe drawn with torch's generator on a device, yielded
    in chunks of rows (dicts of float64 tensors), for workloads too large for
    host generation.  Same distribution as pair_plasma, different stream."""
    import torch

    cdf, ugrid = _mj_table(T)
    cdf_t = torch.tensor(cdf, device=device, dtype=torch.float64)
    u_t = torch.tensor(ugrid, device=device, dtype=torch.float64)
    for r0 in range(0, nr, rows_per_chunk):
        r1 = min(nr, r0 + rows_per_chunk)
        g = torch.Generator(device=device)
        g.manual_seed(seed * 1000003 + r0)
        ncell = (r1 - r0) * nth
        npair = ncell * pairs_per_cell
        cell = torch.arange(ncell, device=device, dtype=torch.int64).repeat_interleave(pairs_per_cell)
        ox = torch.rand(npair, generator=g, device=device, dtype=torch.float64)
        oy = torch.rand(npair, generator=g, device=device, dtype=torch.float64)
        x1 = (r0 + cell // nth).to(torch.float64).add_(ox).repeat_interleave(2)
        x2 = (cell % nth).to(torch.float64).add_(oy).repeat_interleave(2)
        del cell, ox, oy
        n = 2 * npair
        U = torch.rand(n, generator=g, device=device, dtype=torch.float64)
        k = torch.searchsorted(cdf_t, U).clamp_(1, len(ugrid) - 1)
        c0, c1 = cdf_t[k - 1], cdf_t[k]
        mag = u_t[k - 1] + (U - c0) / (c1 - c0).clamp_min(1e-300) * (u_t[k] - u_t[k - 1])
        del k, c0, c1, U
        cosa = torch.rand(n, generator=g, device=device, dtype=torch.float64).mul_(2.0).sub_(1.0)
        beta = torch.rand(n, generator=g, device=device, dtype=torch.float64).mul_(2.0 * np.pi)
        sina = (1.0 - cosa * cosa).clamp_min_(0.0).sqrt_()
        ur = mag * cosa
        uth = mag * sina * torch.cos(beta)
        uph = mag * sina * torch.sin(beta)
        q = torch.tensor([qw, -qw], device=device, dtype=torch.float64).repeat(npair)
        yield {"x1": x1, "x2": x2, "ur": ur, "uth": uth, "uph": uph, "qw": q}
