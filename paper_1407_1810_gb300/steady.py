"""The aligned monopole rotator run to its steady state (Sec. 5.3, Table 1).

The paper's run: 1024 x 512 cells, log r over [r0, ~54 r0] (r0 spans 256
radial cells), equal-area theta, light cylinder R_l = 5 r0, Courant number
0.6, spin-up over half a rotation period, two periods in all, three filter
passes, surface pair injection with f_inj = 0.5 and the Vay pusher; the
plasma comes from injection alone.  After two periods the spin-down
luminosity through spheres out to 25 r0 is within ~1 % of the force-free
value L0 = (8 pi / 3) B0^2 r0^4 Omega^2 (Lorentz-Heaviside units; the paper
writes (2c/3) (B0 r0^2 / R_l)^2 in Gaussian units), and B_ph / B_r follows
the split-monopole (Michel) solution -Omega r sin(theta) / c; the radial
current follows r^2 J_r = -J0 r0^2 cos(theta) with J0 r0^2 = 2 B0 Omega r0^2
(Fig. 7a, b, d).  The run also measures the plasma's kinetic energy flux
through the same spheres (Poynting plus particle flux is the conserved
total), the particles' median gamma (the paper: about 28) and the charge
separation of Fig. 7c (the share of positive charge in each hemisphere).

The paper gives no B0; it asks for a Larmor radius below a cell at the
surface for particles of gamma ~ 28, i.e. omega_c dt above ~17: omega_c dt = 40
here.  No plasma is preloaded.
"""
from __future__ import annotations

import math

import numpy as np

from . import configs

ROTATOR_STEADY = dict(
    nr=1024, nth=512, r_min=1.0, r_max=54.0, r_map="log", th_map="equal_area", courant=0.6, n_filt=3,
    absorb_cells=32, absorb_profile="quadratic", vacuum="monopole_rotator", omega=0.2,
    t_spin=0.5 * 2 * math.pi / 0.2, inject=1, inject_pairs=2, f_inj=0.5, pusher="vay", precision="fp32",
    pairs_per_cell=0, T=0.0, seed=0, wc_dt=40.0, wp_dt=0.05, sort_interval=20)


def michel_l0(b0: float, omega: float, r0: float = 1.0) -> float:
    """Force-free spin-down luminosity of the aligned monopole (Lorentz-Heaviside, c = 1)."""
    return 8.0 * math.pi / 3.0 * b0 * b0 * r0 ** 4 * omega * omega


def bphi_over_br(sim, cfg: dict, b0: float, r: float):
    """(theta, B_ph / B_r) on the sphere of the node radius nearest r: B_ph
    averaged from i -+ 1/2, B_r of the total field (plasma + monopole)."""
    nr, nth = cfg["nr"], cfg["nth"]
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    i = int(round(math.log(r / cfg["r_min"]) / dxi))
    ri = cfg["r_min"] * math.exp(i * dxi)
    f = sim.fields()
    j = np.arange(nth)
    th = np.arccos(1.0 - 2.0 * (j + 0.5) / nth)  # equal-area meridional cell centres
    br = f[3, i, :nth] + b0 * (cfg["r_min"] / ri) ** 2
    bp = 0.5 * (f[5, i - 1, :nth] + f[5, i, :nth])
    return ri, th, bp / br


def r2jr(fr_mean, cfg: dict, b0: float, dt: float, r: float, band: float = 0.04):
    """(theta, r^2 J_r / (J0 r0^2)) from the time-averaged radial charge flux
    F_r (charge through the dual face at (i + 1/2, j) per step): J_r = F_r /
    (dt dA) with dA = 2 pi r^2 (cos th_{j-1/2} - cos th_{j+1/2}), so
    r^2 J_r = F_r / (2 pi dt dcos); averaged over the rows whose radius lies
    within `band` of r (the analytic profile does not depend on r).  Equal-area
    theta only; the polar nodes j = 0, nth are left out."""
    nr, nth = cfg["nr"], cfg["nth"]
    assert cfg["th_map"] == "equal_area"
    g = cfg["n_filt"] + 2
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / nr
    rh = cfg["r_min"] * np.exp((np.arange(nr) + 0.5) * dxi)
    rows = np.nonzero(np.abs(rh / r - 1.0) <= band)[0]
    j = np.arange(1, nth)
    dcos = 2.0 / nth  # equal-area: cos th_j = 1 - 2 j / nth
    prof = fr_mean[0, rows + g][:, j].mean(axis=0) / (2 * math.pi * dt * dcos)
    j0r02 = 2.0 * b0 * cfg["omega"] * cfg["r_min"] ** 2
    return np.arccos(1.0 - 2.0 * j / nth), prof / j0r02


def particle_energy_flux(sim, cfg: dict, radii, band: float = 0.05, q_over_m: float = 1.0):
    """Kinetic energy carried outward by the plasma through the sphere of each
    radius: the sum over the particles in the shell r (1 -+ band) of
    (gamma - 1) |qw| / (q/m) v_r, divided by the shell's width (c = 1, the
    units of the Poynting flux).  Also the median gamma beyond 2 r0."""
    import torch

    d = sim.particles(device="cuda")
    gam = torch.sqrt(1.0 + d["ur"] ** 2 + d["uth"] ** 2 + d["uph"] ** 2)
    e = (gam - 1.0) * d["qw"].abs() / q_over_m * d["ur"] / gam
    if cfg["r_map"] == "log":
        r = cfg["r_min"] * torch.exp(d["x1"] * (math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]))
    else:
        r = cfg["r_min"] + d["x1"] * ((cfg["r_max"] - cfg["r_min"]) / cfg["nr"])
    flux = []
    for rad in radii:
        m = (r > rad * (1 - band)) & (r < rad * (1 + band))
        flux.append(float(e[m].sum()) / (2 * band * rad))
    far = r > 2.0 * cfg["r_min"]
    gmed = float(gam[far].median()) if bool(far.any()) else float("nan")
    # charge separation (Fig. 7c): share of the charge that is positive in
    # each hemisphere (theta < 80 deg, theta > 100 deg), beyond 2 r0; the
    # Goldreich-Julian density of a monopole, -2 Omega.B, changes sign with
    # cos(theta)
    if cfg["th_map"] == "equal_area":
        th = torch.arccos(torch.clamp(1.0 - 2.0 * d["x2"] / cfg["nth"], -1.0, 1.0))
    else:
        th = d["x2"] * (math.pi / cfg["nth"])
    sep = {}
    for name, zone in (("north", th < 4 * math.pi / 9), ("south", th > 5 * math.pi / 9)):
        m = far & zone
        q = d["qw"][m]
        tot = float(q.abs().sum())
        sep[name] = float(q[q > 0].sum()) / tot if tot > 0 else float("nan")
    del d, gam, e, r, far, th
    torch.cuda.empty_cache()
    return np.array(flux), gmed, sep


def run(cfg: dict | None = None, periods: float = 2.0, chunk: int = 500, average_over: float = 0.05, log=None):
    """Run the rotator for `periods` rotation periods on the current GPU.

    Returns the luminosity profile over the last `average_over` of the run
    (nr + 1 values) normalised by L0, the node radii, B_ph / B_r at R_l / 2,
    R_l and 3 R_l / 2 with the Michel values, the particle count and the
    measured particle-steps per second."""
    import time

    from . import picsar as P

    cfg = dict(cfg or ROTATOR_STEADY)
    dt = configs.courant_dt(cfg)
    b0, _ = configs.physics(cfg, dt)
    desc = P.make_desc(**configs.desc_kwargs(cfg, dt, b0))
    sim = P.Simulation(desc)
    omega = cfg["omega"]
    steps = int(round(periods * 2 * math.pi / omega / dt))
    n_avg = max(1, int(average_over * steps))
    L = np.zeros(cfg["nr"] + 1)
    F = None
    samples, done, units, t0 = 0, 0, 0.0, time.perf_counter()

    def advance(k):
        nonlocal done, units
        live0 = sim.live()
        sim.step(k)
        units += 0.5 * (live0 + sim.live()) * k
        done += k

    while done < steps - n_avg:
        advance(min(chunk, steps - n_avg - done))
        if log and done % (10 * chunk) == 0:
            log(f"step {done}/{steps}: {sim.live()} particles")
    every = max(1, n_avg // 50)  # ~50 samples over the averaging window
    while done < steps:
        advance(min(every, steps - done))
        L += sim.luminosity()
        F = sim.flux() if F is None else F + sim.flux()
        samples += 1
    elapsed = time.perf_counter() - t0
    L /= max(samples, 1)
    F /= max(samples, 1)
    dxi = math.log(cfg["r_max"] / cfg["r_min"]) / cfg["nr"]
    r = cfg["r_min"] * np.exp(np.arange(cfg["nr"] + 1) * dxi)
    rl = 1.0 / omega
    profiles = {}
    for name, rad in (("half_rl", 0.5 * rl), ("rl", rl), ("three_half_rl", 1.5 * rl)):
        ri, th, ratio = bphi_over_br(sim, cfg, b0, rad)
        tj, jr = r2jr(F, cfg, b0, dt, rad)
        profiles[name] = {"r": ri, "theta": th, "bphi_over_br": ratio, "michel": -omega * ri * np.sin(th),
                          "theta_j": tj, "r2jr": jr, "r2jr_err": float(np.linalg.norm(jr + np.cos(tj)) /
                                                                      np.linalg.norm(np.cos(tj)))}
    m = sim.moments()
    radii = np.array([1.5, 2.0, 3.0, 5.0, 7.5, 10.0, 15.0, 20.0, 25.0])
    lp, gmed, sep = particle_energy_flux(sim, cfg, radii)
    sim.close()
    return {"r": r, "L_over_L0": L / michel_l0(b0, omega, cfg["r_min"]), "steps": steps, "dt": dt, "b0": b0,
            "particles": m["live"], "injected": m["injected"], "gauss_residual": m["gauss_residual"],
            "particle_steps_per_s": units / elapsed, "seconds": elapsed, "bphi": profiles,
            "lp_radii": radii, "Lp_over_L0": lp / michel_l0(b0, omega, cfg["r_min"]), "gamma_median": gmed,
            "positive_share": sep}
