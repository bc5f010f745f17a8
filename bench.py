#!/usr/bin/env python
"""Throughput of the PICsar particle hot path on GB300: particle-steps/s.

Default workload: the large single run on the FP32 cell+offset path (4096 x 4096
cells, log r in [1, 100], 30 e+/e- pairs per cell = 1.0066e9 particles,
Maxwell-Juttner T = 0.3 over a monopole field, tile sort every 20 steps), a
seeded synthetic plasma generated on the device.  One step = the whole time
step (gather, push, move, deposit, field update, lossy layer, periodic sort).

Printed as one JSON line: the device-timed rate (value), the same metric end to
end through the C-ABI with the particle state loaded from pinned host memory
(e2e), the plain FP64 path on the same workload, the hot kernel's roofline,
the FP64 CPU oracle on bounded samples on every host core and on one
(cpu_baseline) and the SM clocks seen during the timed region.

The FP64 leg also runs both paths for 100 steps from one FP32-rounded state
and reports their field difference on the whole grid (relative L2 and per
component max-norm), the FP64 run following the FP32 run's branches at its
axis-crossing ties.  On one GPU the default run then measures the batched
64-member ensemble for 200 steps (ensemble_64; --no-ensemble skips it).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
  python bench.py --workload NAME [--precision fp32|fp64]   # any workload on either path
  python bench.py --workload ensemble-64                     # 64 uneven members, one launch per phase
  python bench.py --workload rotator-steady                  # the Table 1 run and its physics
  python bench.py --workload NAME --slabs S                  # the workload split into S radial slabs
Under torchrun every rank runs an independent replica (weak scaling); the
ensemble's members are split across the ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1407_1810_gb300 import workload as W  # noqa: E402

DEFAULT_WORKLOAD = "monopole-4096x4096"  # the largest single-GPU configuration
METRIC = "particle-steps/s (gather+push+deposit), FP32 vs FP64 path, at stated Gauss residual"
UNIT = "particle-steps/s"
ALG_BYTES_FP32 = 52  # per particle-step: read cell, dx, dy, u (3), qw = 28 B; write cell, dx, dy, u = 24 B
ALG_BYTES_FP64 = 88  # read x1, x2, u (3), qw = 48 B; write x1, x2, u = 40 B


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--compare-steps", type=int, default=100,
                    help="steps of the FP32 against FP64 field comparison (the FP64 timing is inside them)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--precision", choices=("fp32", "fp64"), default=None,
                    help="run the workload on this particle path instead of its own")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched 64-member ensemble the default run measures after the main workload")
    ap.add_argument("--tile-shape", type=int, default=None, help="FP32 tile: 0 = 16x16, 1 = 8x32, 2 = 32x8 cells")
    ap.add_argument("--sort-interval", type=int, default=None)
    ap.add_argument("--slabs", type=int, default=0,
                    help="run the workload split into this many radial slabs on this GPU (pic_slabs_*)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(ms, units, device):
    """Whole-job timing of N independent replicas: the slowest rank's time and
    the particle-steps of all ranks (plain values when not distributed)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, units
    t = torch.tensor([ms, units], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic():
    """DRAM bytes per particle of the tile kernel from the committed ncu
    summary, if the kernel source has not changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "k_tiles32_traffic.json")
    src = os.path.join(ROOT, "paper_1407_1810_gb300", "csrc", "particles32.cu")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if d.get("source_sha256_16") != h:
        return None
    return float(d["dram_bytes_per_particle"])


def phase_per_step(prof, sort_interval):
    """Per-step cost of each phase: every phase runs once per step except the
    tile sort (or compaction), which runs once per sort interval."""
    out = dict(prof)
    out["sort"] = prof["sort"] / max(1, sort_interval)
    return out


def time_steps(sim, K, stream):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    live0 = sim.live()
    torch.cuda.synchronize()
    l0 = sim.launches()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler keep to the timed launches
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    l1 = sim.launches()
    live1 = sim.live()
    return ms, 0.5 * (live0 + live1) * K, l1 - l0


L2_BYTES = 129e6


def l2_note(state_bytes):
    if state_bytes > L2_BYTES:
        return "inputs larger than L2 (particle state %.1f GB)" % (state_bytes / 1e9)
    return "particle state %.1f MB fits in L2: an L2-resident figure, not an HBM one" % (state_bytes / 1e6)


def gpu_arm(args):
    import torch

    from paper_1407_1810_gb300 import configs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(configs.CONFIGS[args.workload])
    if args.tile_shape is not None:
        cfg["tile_shape"] = args.tile_shape
    if args.sort_interval is not None:
        cfg["sort_interval"] = args.sort_interval
    if args.precision is not None:
        cfg["precision"] = args.precision
    stream = torch.cuda.Stream(device=dev)
    sim, qw, _, _ = W.make_sim(cfg, stream=stream.cuda_stream)
    n = W.load_plasma(sim, cfg, qw, dev, stream)
    torch.cuda.synchronize()
    sim.step(args.warmup)
    torch.cuda.synchronize()
    sim.profile(True)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms, units, launches = time_steps(sim, args.steps, stream)
    ck = clocks.stop()
    ms_max, units_all = combine_ranks(ms, units, dev)
    prof, psteps = sim.get_profile()
    mom = sim.moments()
    value = units_all / (ms_max * 1e-3)
    live = mom["live"]
    precision = cfg["precision"]
    alg = ALG_BYTES_FP32 if precision == "fp32" else ALG_BYTES_FP64
    kname = "k_tiles32" if precision == "fp32" else "k_particles64"
    peak, peak_kind = measured_peaks()
    kms = prof["particles"]
    achieved = alg * live / (kms * 1e-3) / 1e9 if kms > 0 else None
    tr = recorded_traffic() if precision == "fp32" else None
    hot_rate = live / (kms * 1e-3) if kms > 0 else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{cfg['nr']}x{cfg['nth']}", "particles": n,
                   "pairs_per_cell": cfg["pairs_per_cell"], "T": cfg["T"], "path": precision,
                   "sort_interval": cfg.get("sort_interval", 20), "tile_shape": cfg.get("tile_shape", 0),
                   "field_update": "f64",
                   "l2": l2_note(n * (36 if precision == "fp32" else 56))},
        "gauss_residual": mom["gauss_residual"],
        "hot_kernel": {"name": kname, "ms_per_launch": kms, "particle_steps_per_s": hot_rate},
        "phase_ms_per_launch": prof,
        "phase_ms_per_step": phase_per_step(prof, cfg.get("sort_interval", 20)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": (tr * live) if tr else None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_particle_step": alg},
        "clocks": ck,
        "gpu_launches": launches,
    }
    sim.close()
    del sim
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_fp64 and precision == "fp32":
        out["fp64_path"] = fp64_run(cfg, dev, stream, args)
        if out["fp64_path"].get("value"):
            out["speedup_vs_fp64_path"] = value / out["fp64_path"]["value"]
    if not args.no_e2e:
        try:
            out["e2e"] = e2e_run(cfg, dev, stream, args)
        except Exception as exc:  # e.g. not enough pinned host memory for the state
            out["e2e"] = {"value": None, "unit": UNIT, "error": repr(exc)[:200]}
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(cfg)
    if world == 1 and not args.no_ensemble and args.workload == DEFAULT_WORKLOAD:
        # the batched ensemble (64 uneven plasmas), 200 steps, on this GPU
        ens = ensemble_measure(args, rank, world, local, steps=200, warmup=5)
        out["ensemble_64"] = {k: ens[k] for k in ("value", "unit", "ms_per_step", "steps", "config",
                                                   "sequential_pic_step", "autotune", "clocks", "gpu_launches")}
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def fp64_run(cfg, dev, stream, args):
    """The plain FP64 path on the same workload, timed; both paths run the
    same `compare_steps` steps from one FP32-rounded state and their plasma
    fields are compared on the whole grid (relative L2 and per-component
    max-norm).  The FP32 run goes first and logs its axis-crossing ties
    (|u_ph| <= 2^-13 |u|, where rounding sets the sign of the swept azimuth);
    the FP64 run follows those branches."""
    import numpy as np
    import torch

    ntot = cfg["nr"] * cfg["nth"] * cfg["pairs_per_cell"] * 2
    nsteps = max(args.compare_steps, 2 + args.fp64_steps)
    sim, qw, _, _ = W.make_sim(cfg, "fp32", stream.cuda_stream, ntot + (1 << 20))
    W.load_plasma(sim, cfg, qw, dev, stream, fp32_state=True)
    sim.step(nsteps)
    f32, m32, ties = sim.fields(), sim.moments(), sim.axis_ties()
    sim.close()
    del sim
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    sim, qw, _, _ = W.make_sim(cfg, "fp64", stream.cuda_stream, ntot + (1 << 20))
    W.load_plasma(sim, cfg, qw, dev, stream, fp32_state=True)
    sim.set_axis_hints(ties)
    sim.step(2)
    sim.profile(True)
    ms, units, _ = time_steps(sim, args.fp64_steps, stream)
    prof, _ = sim.get_profile()  # before profile(False), which clears the counters
    sim.profile(False)
    live = sim.live()
    kms = prof["particles"]
    res = {"value": units / (ms * 1e-3), "steps": args.fp64_steps, "ms_per_step": ms / args.fp64_steps,
           "hot_kernel": {"name": "k_particles64", "ms_per_launch": kms,
                          "achieved_GBps": ALG_BYTES_FP64 * live / (kms * 1e-3) / 1e9 if kms else None}}
    sim.step(nsteps - 2 - args.fp64_steps)
    f64, m64 = sim.fields(), sim.moments()
    sim.close()
    del sim
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    band = slice(32, cfg["nth"] + 1 - 32)  # 32 cells clear of each pole
    d = f32 - f64
    mx = max(float(np.max(np.abs(d[c])) / max(np.max(np.abs(f64[c])), 1e-300)) for c in range(6))
    res["fp32_vs_fp64_fields"] = {
        "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(f64)),
        "max_rel_per_component": mx,
        "rel_l2_away_from_axis": (float(np.linalg.norm(d[:, :, band]) / np.linalg.norm(f64[:, :, band]))
                                  if cfg["nth"] > 64 else None),
        "steps": nsteps, "start": "one FP32-rounded state", "fp64_gauss_residual": m64["gauss_residual"],
        "fp32_gauss_residual": m32["gauss_residual"], "live": [m32["live"], m64["live"]],
        "axis_ties": {"fp32": m32["axis_ties"], "fp64": m64["axis_ties"],
                      "per_particle_step": m32["axis_ties"] / max(1.0, ntot * nsteps),
                      "note": "axis crossings with |u_ph| <= 2^-13 |u|: the FP64 run takes the FP32 run's branch"}}
    return res


def e2e_run(cfg, dev, stream, args):
    """Same metric through the C-ABI with host buffers: the particle state is
    read from pinned host memory by pic_load_particles inside the timed region
    (in place, over the host link), then K steps, then the moments are read
    back to the host."""
    import torch

    from paper_1407_1810_gb300 import synthetic

    ntot = cfg["nr"] * cfg["nth"] * cfg["pairs_per_cell"] * 2
    sim, qw, _, _ = W.make_sim(cfg, stream=stream.cuda_stream, capacity=ntot + (1 << 20))
    host = {k: torch.empty(ntot, dtype=torch.float64, pin_memory=True) for k in ("x1", "x2", "ur", "uth", "uph", "qw")}
    off = 0
    with torch.cuda.stream(stream):
        for ch in synthetic.pair_plasma_torch(cfg["nr"], cfg["nth"], cfg["pairs_per_cell"], cfg["T"], qw,
                                              cfg["seed"], dev, rows_per_chunk=128):
            m = ch["x1"].numel()
            for k in host:
                host[k][off:off + m].copy_(ch[k])
            off += m
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.load(*(host[k] for k in ("x1", "x2", "ur", "uth", "uph", "qw")))
    t_load = time.perf_counter() - t0
    sim.step(args.steps)
    mom = sim.moments()  # device -> host read of the step's result (Gauss residual, energies, counts)
    t1 = time.perf_counter()
    units = 0.5 * (ntot + mom["live"]) * args.steps
    sim.close()
    del sim, host
    torch.cuda.empty_cache()
    import ctypes

    from paper_1407_1810_gb300 import picsar as P

    return {"value": units / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": 48 * ntot / args.steps,
            "d2h_bytes_per_step": ctypes.sizeof(P.pic_moments) / args.steps, "seconds": t1 - t0,
            "load_seconds": t_load}


SAMPLE_SIDE = 96


def oracle_sample(cfg, worker=0):
    """A bounded sample of the workload for the FP64 CPU oracle: the same r
    range and plasma (pairs per cell, temperature, omega_c dt, omega_p dt) on a
    SAMPLE_SIDE x SAMPLE_SIDE grid; worker w draws its plasma with seed
    seed + 1000 w, so concurrent workers run disjoint samples."""
    import oracle as O
    from paper_1407_1810_gb300 import configs, synthetic

    small = dict(cfg, nr=SAMPLE_SIDE, nth=SAMPLE_SIDE)
    dt = configs.courant_dt(small)
    b0, qw = configs.physics(small, dt)
    o = O.Oracle(O.params(**configs.oracle_kwargs(small, dt, b0)))
    d = synthetic.pair_plasma(SAMPLE_SIDE, SAMPLE_SIDE, small["pairs_per_cell"], small["T"], qw,
                              small["seed"] + 1000 * worker)
    o.load(d["x1"], d["x2"], d["ur"], d["uth"], d["uph"], d["qw"])
    desc = (f"{SAMPLE_SIDE}x{SAMPLE_SIDE} grid, same r range, {small['pairs_per_cell']} pairs/cell "
            f"({o.num_particles()} particles), FP64 C oracle")
    return o, desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(cfg, worker, warmup, steps, budget_s, barrier, results):
    """One oracle process: its own sample, W untimed steps, then either
    `steps` timed steps or as many as fit in budget_s (steps = 0)."""
    o, desc = oracle_sample(cfg, worker)
    if warmup:
        o.step(warmup)
    barrier.wait()
    units, t, n = 0.0, 0.0, 0
    while (steps and n < steps) or (not steps and t < budget_s and n < 200):
        u, dt = time_oracle(o, 1)
        units += u
        t += dt
        n += 1
    results.put((worker, units, t, n, desc))


def oracle_parallel(cfg, workers, warmup=0, steps=0, budget_s=10.0):
    """The oracle, unchanged and single-threaded, run as `workers` spawned
    processes at once on disjoint samples (a spawned pool: the parent may
    already hold a CUDA context).  Returns (sum of particle-steps, the
    slowest worker's seconds, steps per worker, sample description)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(workers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(cfg, w, warmup, steps, budget_s, barrier, results))
             for w in range(workers)]
    for p in procs:
        p.start()
    out = [results.get() for _ in procs]
    for p in procs:
        p.join()
    units = sum(r[1] for r in out)
    t = max(r[2] for r in out)
    return units, t, min(r[3] for r in out), out[0][4]


def time_oracle(o, nsteps):
    n0 = o.num_particles()
    t0 = time.perf_counter()
    o.step(nsteps)
    t = time.perf_counter() - t0
    return 0.5 * (n0 + o.num_particles()) * nsteps, t


def cpu_baseline(cfg, budget_s=10.0):
    """The oracle on all host cores (one process per core, disjoint samples,
    started together) and, beside it, on one core."""
    cores = host_cores()
    u1, t1, n1, desc = oracle_parallel(cfg, 1, budget_s=budget_s)
    un, tn, nn, _ = oracle_parallel(cfg, cores, budget_s=budget_s)
    return {"value": un / tn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{desc}; {cores} processes at once, one sample each (seeds differ), "
                      f"{nn}+ steps each, the slowest process's time",
            "single_core": {"value": u1 / t1, "cores": 1, "steps": n1}}


def reference_arm(args):
    """The oracle as the reference arm: one spawned process per host core,
    each with its own bounded sample, W untimed steps, then K timed steps;
    the value is all processes' particle-steps over the slowest one's time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1407_1810_gb300 import configs

    cfg = configs.CONFIGS[args.workload]
    cores = host_cores()
    units, t, _, desc = oracle_parallel(cfg, cores, warmup=args.warmup, steps=args.steps)
    v = units / t
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "path": "oracle"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{desc}; {cores} processes at once, one sample each, "
                                      f"{args.steps} steps each, the slowest process's time"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def ensemble_plasma(cfg, qw):
    """~cfg['particles'] particles of the member's recipe: whole pairs per cell
    where there are enough, else one pair in each of a random set of cells."""
    import numpy as np

    from paper_1407_1810_gb300 import synthetic

    ncell = cfg["nr"] * cfg["nth"]
    npairs = max(1, cfg["particles"] // 2)
    if npairs >= ncell:
        return synthetic.pair_plasma(cfg["nr"], cfg["nth"], npairs // ncell, cfg["T"], qw, cfg["seed"])
    cells = np.random.default_rng(cfg["seed"] + 7).choice(ncell, npairs, replace=False)
    return synthetic.pair_plasma_cells(cfg["nr"], cfg["nth"], np.sort(cells), 1, cfg["T"], qw, cfg["seed"])


def ensemble_members(n_members, rank, world):
    """The members one rank holds: the members are independent simulations,
    so N GPUs split them (member m on rank m mod N) with no collective in the
    data path; only the timing is combined."""
    return list(range(rank, n_members, world))


def ensemble_measure(args, rank, world, local, n_members=64, steps=None, warmup=None):
    """64 independent monopole plasmas with uneven grids and particle counts
    (this rank's share of them): the members autotuned together
    (pic_autotune_ensemble), then advanced by the batched, graph-captured
    pic_ensemble_step; the same members advanced one after another by
    pic_step are timed for comparison.  Returns the result line."""
    import torch

    from paper_1407_1810_gb300 import configs
    from paper_1407_1810_gb300 import picsar as P

    steps = steps or args.steps
    warmup = warmup or args.warmup
    stream = torch.cuda.Stream()
    sims, total = [], 0
    mine = ensemble_members(n_members, rank, world)
    for m in mine:
        cfg = configs.ensemble_member_config(m)
        dt = configs.courant_dt(cfg)
        b0, qw = configs.physics(cfg, dt)
        s = P.Simulation(P.make_desc(**configs.desc_kwargs(cfg, dt, b0)), stream=stream.cuda_stream)
        d = ensemble_plasma(cfg, qw)
        s.load(*(d[k] for k in ("x1", "x2", "ur", "uth", "uph", "qw")))
        total += len(d["x1"])
        sims.append(s)
    t0 = time.perf_counter()
    choice = P.autotune_ensemble(sims, trial_steps=40)
    t_tune = time.perf_counter() - t0
    P.ensemble_step(sims, warmup)
    torch.cuda.synchronize()
    live0 = sum(s.live() for s in sims)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler keep to the timed launches
    launches = P.ensemble_step(sims, steps)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    torch.cuda.nvtx.range_pop()
    ck = clocks.stop()
    live1 = sum(s.live() for s in sims)
    units = 0.5 * (live0 + live1) * steps
    ms_max, units_all = combine_ranks(1e3 * (t1 - t0), units, torch.device("cuda", local))
    value = units_all / (ms_max * 1e-3)
    # the same members stepped one after another
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for s in sims:
        s.step(steps)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    seq_ms, seq_units = combine_ranks(1e3 * (t3 - t2), units, torch.device("cuda", local))
    seq = seq_units / (seq_ms * 1e-3)
    total_all = combine_ranks(0.0, float(total), torch.device("cuda", local))[1]
    for s in sims:
        s.close()
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ensemble-64", "members": n_members, "members_per_rank": len(mine),
                       "split": "member m on rank m mod N", "particles": int(total_all), "path": "fp32",
                       "timing": "host clock around pic_ensemble_step (one launch per phase for all members, "
                                 "one graph per sort interval)"},
            "sequential_pic_step": {"value": seq, "speedup_of_ensemble": value / seq},
            "autotune": {"seconds": t_tune, "choice": choice,
                         "how": "one tile shape and sort interval for all members, timed on clones through "
                                "pic_ensemble_step"},
            "clocks": ck, "gpu_launches": launches}


def ensemble_arm(args, n_members=64):
    """`--workload ensemble-64`: the batched ensemble on its own line."""
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    out = ensemble_measure(args, rank, world, local, n_members)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def slabs_arm(args):
    """The workload split into args.slabs equal radial slabs on this GPU
    (pic_slabs_*: field and flux halos and particle migration every step)
    beside the same workload on one context: the cost of the decomposition's
    exchanges.  Host clock around the steps (a slab step reads its migration
    counts on the host)."""
    import torch

    from paper_1407_1810_gb300 import configs
    from paper_1407_1810_gb300 import picsar as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    cfg = dict(configs.CONFIGS[args.workload])
    if args.precision:
        cfg["precision"] = args.precision
    out = {}
    for split in (True, False):
        if split:
            dt = configs.courant_dt(cfg)
            b0, qw = configs.physics(cfg, dt)
            sim = P.Slabs(P.make_desc(**configs.desc_kwargs(cfg, dt, b0)), args.slabs, stream=stream.cuda_stream)
        else:
            sim, qw, _, _ = W.make_sim(cfg, stream=stream.cuda_stream)
        W.load_plasma(sim, cfg, qw, dev, stream)
        sim.step(args.warmup)
        live0 = sim.moments()["live"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(args.steps)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        live1 = sim.moments()["live"]
        out[split] = (0.5 * (live0 + live1) * args.steps / (ms * 1e-3), ms / args.steps)
        sim.close()
        del sim
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": out[True][0], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out[True][1], "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32" if cfg["precision"] == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "slabs": args.slabs, "path": cfg["precision"],
                       "timing": "host clock around pic_slabs_step / pic_step"},
            "one_context": {"value": out[False][0], "ms_per_step": out[False][1]},
            "exchange_ms_per_step": out[True][1] - out[False][1]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def steady_arm(args):
    """The Table 1 monopole rotator run to its steady state (two rotation
    periods from an empty domain): throughput over the run and its physics
    against the force-free solution."""
    import math

    import numpy as np
    import torch

    from paper_1407_1810_gb300 import steady

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    res = steady.run()
    r, L = res["r"], res["L_over_L0"]
    sel = (r >= 1.5) & (r <= 25.0)
    bphi, r2jr = {}, {}
    for name, p in res["bphi"].items():
        mid = (p["theta"] > 0.3) & (p["theta"] < math.pi - 0.3)
        bphi[f"r={p['r']:.2f}"] = float(np.median(p["bphi_over_br"][mid] / p["michel"][mid]))
        c = np.cos(p["theta_j"])
        r2jr[f"r={p['r']:.2f}"] = float(-(p["r2jr"] @ c) / (c @ c))
    out = {"metric": METRIC, "value": res["particle_steps_per_s"], "unit": UNIT, "n_gpus": world,
           "steps": res["steps"], "warmup": 0, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "rotator-steady", "grid": "1024x512", "periods": 2, "particles_at_end": res["particles"],
                      "timing": "host clock over the whole run, from an empty domain"},
           "physics": {"L_over_L0_r1.5_to_25": {"mean": float(L[sel].mean()), "min": float(L[sel].min()),
                                                 "max": float(L[sel].max())},
                       "bphi_over_br_to_michel": bphi, "r2jr_scale_to_michel": r2jr,
                       "poynting_plus_particle_flux_over_L0": {
                           f"r={x:g}": round(float(L[np.argmin(np.abs(r - x))] + lp), 4)
                           for x, lp in zip(res["lp_radii"], res["Lp_over_L0"])},
                       "gamma_median": res["gamma_median"],
                       "positive_charge_share_beyond_2r0": res["positive_share"],
                       "gauss_residual": res["gauss_residual"]}}
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "ensemble-64":
        ensemble_arm(args)
        return
    if args.slabs:
        slabs_arm(args)
        return
    if args.workload == "rotator-steady":
        steady_arm(args)
        return
    gpu_arm(args)


if __name__ == "__main__":
    main()
