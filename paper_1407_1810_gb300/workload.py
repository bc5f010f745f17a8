"""A named workload's simulation, built and filled on the device.

One recipe for every caller that runs a workload at its full size: the
simulation is made from the config's parameters (time step at the config's
Courant number, B0 and macro-charge from its cyclotron and plasma frequencies)
and the pair plasma is drawn on the device in row chunks and loaded through
pic_load_particles without passing through host memory.
"""
from __future__ import annotations

from . import configs


def capacity_for(cfg: dict) -> int:
    """Particle slots for a config: its plasma plus room for ~1.6% growth."""
    ntot = cfg["nr"] * cfg["nth"] * cfg["pairs_per_cell"] * 2
    return ntot + ntot // 64 + (1 << 20)


def make_sim(cfg: dict, precision: str | None = None, stream=0, capacity: int | None = None):
    """(Simulation, |qw|, dt, b0) for a config dict; stream is a raw CUDA stream handle."""
    from . import picsar as P

    prec = precision or cfg["precision"]
    dt = configs.courant_dt(cfg)
    b0, qw = configs.physics(cfg, dt)
    kw = configs.desc_kwargs(cfg, dt, b0, precision=prec, capacity=capacity or capacity_for(cfg))
    if prec == "fp32":
        kw["tile_shape"] = cfg.get("tile_shape", 0)
    return P.Simulation(P.make_desc(**kw), stream=stream), qw, dt, b0


def load_plasma(sim, cfg: dict, qw: float, device, stream=None, rows_per_chunk: int = 128,
                fp32_state: bool = False) -> int:
    """Draw the config's pair plasma on the device and load it; returns the
    count.  fp32_state: round it first to what the FP32 path stores (cell +
    FP32 offset, FP32 momenta and charge), so that both paths can start from
    one state."""
    import torch

    from . import synthetic

    n = 0
    ctx = torch.cuda.stream(stream) if stream is not None else torch.cuda.device(device)
    with ctx:
        for ch in synthetic.pair_plasma_torch(cfg["nr"], cfg["nth"], cfg["pairs_per_cell"], cfg["T"], qw,
                                              cfg["seed"], device, rows_per_chunk=rows_per_chunk):
            if fp32_state:
                for k in ("x1", "x2"):
                    c = torch.floor(ch[k])
                    ch[k] = c + (ch[k] - c).float().double()
                for k in ("ur", "uth", "uph", "qw"):
                    ch[k] = ch[k].float().double()
            sim.load(ch["x1"], ch["x2"], ch["ur"], ch["uth"], ch["uph"], ch["qw"])
            n += ch["x1"].numel()
            del ch
    return n
