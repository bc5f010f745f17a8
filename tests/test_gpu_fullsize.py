"""Parity at the workloads' full sizes, in the launch configuration the benchmark times.

The oracle cannot step 1e8-1e9 particles, so at full size each test lets the
GPU run a few steps, exports its state, and has the oracle replay one step of
a sample of the particles (every STRIDE-th id) on the GPU's own fields; the
GPU's step of the same particles must match that replay to the bars of the
small-size replay tests.  Gauss's law, which a charge-conserving deposit keeps
at any size, is checked on the whole grid, and the particle count is checked
against the removals the GPU reports.

  - 4096 x 4096 monopole, 1e9 particles, FP32 path (the benchmark's workload);
  - 512 x 512 monopole rotator with injection, 2e7 particles, FP64 path;
  - 1024 x 1024 rotator, 1e8 particles: FP32 path against the FP64 GPU path
    after 100 steps (the FP64 path itself being held to the oracle above and
    in the small-size tests), plus a sampled FP32 replay.
"""
import numpy as np
import pytest

import oracle as O
from paper_1407_1810_gb300 import configs, synthetic, workload

from gpu_common import KEYS, by_id, rel_l2, replay_compare_fp32

pytestmark = pytest.mark.gpu
TAU = 2e-6
GAUSS_FP32 = 1e-6
GAUSS_FP64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()
    O.build_oracle()
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _sample(sim, stride, keep=None):
    """Live particles whose id is a multiple of stride (and in keep, if given), on the host."""
    import torch

    d = sim.particles(device="cuda")
    m = d["id"] % stride == 0
    out = {k: v[m].cpu().numpy() for k, v in d.items()}
    del d, m
    torch.cuda.empty_cache()
    if keep is not None:
        sel = np.isin(out["id"], keep)
        out = {k: v[sel] for k, v in out.items()}
    return out


def _replay(cfg, dt, b0, fields, sample, step):
    """The oracle's step of a sample of particles in given fields."""
    p = O.params(**configs.oracle_kwargs(cfg, dt, b0))
    o = O.Oracle(p)
    o.set_fields(fields)
    o.load(*(sample[k] for k in KEYS), ids=sample["id"])
    o.set_clock(step, int(sample["id"].max()) + 1)
    assert o.particles_only() == 0
    return o.particles()


def _run(cfg, warm, stride, precision=None):
    """GPU simulation of a config at full size: warm steps, then a sampled
    one-step replay; returns (sim, gpu sample after, oracle replay, moments)."""
    import torch

    sim, qw, dt, b0 = workload.make_sim(cfg, precision)
    n = workload.load_plasma(sim, cfg, qw, "cuda")
    assert n == cfg["nr"] * cfg["nth"] * cfg["pairs_per_cell"] * 2
    torch.cuda.synchronize()
    sim.step(warm)
    m0 = sim.moments()
    before = _sample(sim, stride)
    fields = sim.fields()
    sim.step(1)
    m1 = sim.moments()
    after = _sample(sim, stride, keep=before["id"])
    replay = _replay(cfg, dt, b0, fields, before, warm)
    return sim, after, replay, m0, m1, len(before["id"])


def _counts_consistent(m0, m1):
    assert m1["live"] == m0["live"] - (m1["deleted"] - m0["deleted"]) + (m1["injected"] - m0["injected"])


def test_monopole_4096_fp32_sampled_replay_and_gauss():
    cfg = dict(configs.CONFIGS["monopole-4096x4096"])
    sim, g, r, m0, m1, ns = _run(cfg, warm=3, stride=50000)
    assert ns > 15000
    replay_compare_fp32(g, r, TAU)
    _counts_consistent(m0, m1)
    assert m1["gauss_residual"] <= GAUSS_FP32, m1["gauss_residual"]
    sim.close()


def test_rotator_512_fp64_sampled_replay_and_gauss():
    cfg = dict(configs.CONFIGS["rotator-512x512"])
    sim, g, r, m0, m1, ns = _run(cfg, warm=15, stride=1000)
    assert ns > 15000
    g, r = by_id(g), by_id(r)
    # FP64 path: removals exact, positions and momenta to rounding
    assert np.array_equal(g["id"], r["id"])
    assert np.max(np.abs(g["x1"] - r["x1"])) < 1e-10
    assert np.max(np.abs(g["x2"] - r["x2"])) < 1e-10
    assert np.array_equal(np.floor(g["x1"]), np.floor(r["x1"]))
    assert np.array_equal(np.floor(g["x2"]), np.floor(r["x2"]))
    umag = np.sqrt(r["ur"] ** 2 + r["uth"] ** 2 + r["uph"] ** 2) + 1e-3
    for k in ("ur", "uth", "uph"):
        assert np.max(np.abs(g[k] - r[k]) / umag) < 1e-11, k
    assert np.array_equal(g["qw"], r["qw"])
    _counts_consistent(m0, m1)
    assert m1["injected"] > m0["injected"]
    assert m1["gauss_residual"] <= GAUSS_FP64, m1["gauss_residual"]
    sim.close()


def _load_fp32_state(sim, cfg, qw):
    """The config's plasma rounded to the FP32 path's state (cell + FP32
    offset, FP32 momenta and charge), so both paths start from one state."""
    import torch

    for ch in synthetic.pair_plasma_torch(cfg["nr"], cfg["nth"], cfg["pairs_per_cell"], cfg["T"], qw,
                                          cfg["seed"], "cuda", rows_per_chunk=128):
        for k in ("x1", "x2"):
            c = torch.floor(ch[k])
            ch[k] = c + (ch[k] - c).float().double()
        for k in ("ur", "uth", "uph", "qw"):
            ch[k] = ch[k].float().double()
        sim.load(ch["x1"], ch["x2"], ch["ur"], ch["uth"], ch["uph"], ch["qw"])


def test_rotator_1024_fp32_against_fp64_100_steps():
    import torch

    cfg = dict(configs.CONFIGS["rotator-1024x1024"])
    s32, qw, _, _ = workload.make_sim(cfg, "fp32")
    s64, _, _, _ = workload.make_sim(cfg, "fp64")
    _load_fp32_state(s32, cfg, qw)
    _load_fp32_state(s64, cfg, qw)
    torch.cuda.synchronize()
    s32.step(100)
    s64.step(100)
    m32, m64 = s32.moments(), s64.moments()
    assert m32["gauss_residual"] <= GAUSS_FP32, m32["gauss_residual"]
    assert m64["gauss_residual"] <= GAUSS_FP64, m64["gauss_residual"]
    e = rel_l2(s32.fields(), s64.fields())
    assert e < 1e-5, e
    fx = rel_l2(s32.flux(), s64.flux())
    assert fx < 1e-5, fx
    assert abs(m32["live"] - m64["live"]) <= 1e-5 * m64["live"]
    s64.close()
    s32.close()


def test_rotator_1024_fp32_sampled_replay():
    cfg = dict(configs.CONFIGS["rotator-1024x1024"])
    sim, g, r, m0, m1, ns = _run(cfg, warm=10, stride=5000)
    assert ns > 15000
    replay_compare_fp32(g, r, TAU)
    _counts_consistent(m0, m1)
    assert m1["gauss_residual"] <= GAUSS_FP32, m1["gauss_residual"]
    sim.close()
