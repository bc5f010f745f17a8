"""Batched ensemble (pic_ensemble_step) and the tile/sort autotuner (pic_autotune).

Members are independent simulations with uneven grids and particle counts
(the ensemble workload's recipe).  The FP32 path's deposit sums are exact
integers, so neither the batching (graph capture, parallel branches) nor the
tile shape or sort interval may change a single bit of any member's result;
FP64 members agree to rounding (atomic summation order).
"""
import numpy as np
import pytest

from paper_1407_1810_gb300 import configs, synthetic

from gpu_common import setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_1810_gb300 import build

    build.build()


def _member_cfg(m, precision="fp32", scale=8):
    r = synthetic.ensemble_member(m)
    # the workload's grid shapes scaled down so the test stays small
    nr, nth = max(16, r["nr"] // scale), max(16, r["nth"] // scale)
    ppc = max(1, min(6, r["particles"] // (2 * nr * nth)))
    return dict(configs.CONFIGS["monopole-64x64"], nr=nr, nth=nth, pairs_per_cell=ppc, T=r["T"],
                seed=r["seed"], precision=precision)


def _pairs(n, precision):
    a, b = [], []
    for m in range(n):
        cfg = _member_cfg(m, precision)
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        a.append(s1)
        b.append(s2)
    return a, b


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ensemble_equals_independent_steps(precision):
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = _pairs(6, precision)
    P.ensemble_step(ens, 45)  # crosses two sort intervals (20)
    for s in ref:
        s.step(45)
    for k, (a, b) in enumerate(zip(ens, ref)):
        fa, fb = a.fields(), b.fields()
        if precision == "fp32":
            assert np.array_equal(fa, fb), k
        else:
            assert np.max(np.abs(fa - fb)) <= 1e-13 * max(np.max(np.abs(fb)), 1e-300), k
        assert a.moments()["live"] == b.moments()["live"], k


def test_ensemble_with_variable_count_injection():
    """Variable-count injection keys its rounding on the step number; the
    ensemble captures each member's steps into CUDA graphs, and every
    captured step must carry its own key: the members' injected ids, counts
    and fields equal those of independent steps bit for bit."""
    from paper_1407_1810_gb300 import picsar as P

    base = dict(configs.CONFIGS["rotator-1024x1024"], nr=24, nth=16, pairs_per_cell=1, absorb_cells=4, t_spin=0.0,
                inject=2, inject_pairs=6, inject_smooth=1)
    cfgs = [dict(base, inject_q=q, inject_seed=sd) for q, sd in ((2.0, 11), (0.7, 12))]
    ens, ref = [], []
    for cfg in cfgs:
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    P.ensemble_step(ens, 50)
    for s in ref:
        s.step(50)
    for k, (a, b) in enumerate(zip(ens, ref)):
        ma, mb = a.moments(), b.moments()
        assert ma["injected"] == mb["injected"] > 0 and ma["inject_capped"] == mb["inject_capped"], k
        assert np.array_equal(a.fields(), b.fields()), k
        ia, ib = np.sort(a.particles()["id"]), np.sort(b.particles()["id"])
        assert np.array_equal(ia, ib), k


def test_ensemble_with_injection_member():
    from paper_1407_1810_gb300 import picsar as P

    cfgs = [dict(configs.CONFIGS["rotator-1024x1024"], nr=24, nth=16, pairs_per_cell=1, absorb_cells=4, t_spin=0.5),
            _member_cfg(3)]
    ens, ref = [], []
    for cfg in cfgs:
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    P.ensemble_step(ens, 70)
    for s in ref:
        s.step(70)
    for a, b in zip(ens, ref):
        assert np.array_equal(a.fields(), b.fields())
        ma, mb = a.moments(), b.moments()
        assert ma["injected"] == mb["injected"] and ma["live"] == mb["live"]


def test_autotune_keeps_the_physics_bit_exact():
    cfg = dict(_member_cfg(5), T=0.8)
    s1, _, plasma, _ = setup(cfg)
    s2, _, _, _ = setup(cfg, plasma=plasma)
    s1.step(5)
    s2.step(5)
    choice = s1.autotune(trial_steps=20)
    assert choice["sort_interval"] in (5, 10, 20, 40) and choice["tile_shape"] in (0, 1, 2)
    # autotuning ran on clones: s1 has not advanced
    assert s1.moments()["step"] == 5
    s1.step(30)
    s2.step(30)
    assert np.array_equal(s1.fields(), s2.fields())
    assert np.array_equal(s1.flux(), s2.flux())


@pytest.mark.parametrize("shape", [1, 2])
def test_tile_shapes_agree(shape):
    cfg = _member_cfg(7)
    s1, _, plasma, _ = setup(cfg)
    s2, _, _, _ = setup(cfg, plasma=plasma, tile_shape=shape)
    s1.step(25)
    s2.step(25)
    assert np.array_equal(s1.fields(), s2.fields())


def test_members_keep_their_own_sort_intervals():
    """Members with sort intervals 5, 13 and 40 in one ensemble: each runs its
    own schedule (the same kernels as its independent run, counted launch by
    launch) and its result is bit-identical."""
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = [], []
    for m, S in ((0, 5), (1, 13), (2, 40)):
        cfg = dict(_member_cfg(m), sort_interval=S)
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    l0 = [s.launches() for s in ens]
    P.ensemble_step(ens, 60)
    for s in ref:
        s.step(60)
    for k, (a, b) in enumerate(zip(ens, ref)):
        assert a.launches() - l0[k] == b.launches() - l0[k], k
        assert np.array_equal(a.fields(), b.fields()), k
        assert a.moments()["step"] == 60


def test_one_launch_per_phase_for_all_members():
    """FP32 members on all three tile shapes: each phase of a step is one
    kernel launch for every member (one per tile shape for the tile kernel),
    so the call enqueues a few launches per step however many members there
    are, while each member's own count advances as in its pic_step run; every
    member's result equals that run's bit for bit."""
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = [], []
    for m, shape in ((0, 0), (1, 1), (2, 2), (3, 0), (4, 1), (6, 2)):
        cfg = _member_cfg(m)
        s1, _, plasma, _ = setup(cfg, tile_shape=shape)
        s2, _, _, _ = setup(cfg, plasma=plasma, tile_shape=shape)
        ens.append(s1)
        ref.append(s2)
    l0 = [s.launches() for s in ens]
    r0 = [s.launches() for s in ref]
    kernels = P.ensemble_step(ens, 30)
    for s in ref:
        s.step(30)
    member_launches = sum(s.launches() for s in ens) - sum(l0)
    assert member_launches == sum(s.launches() for s in ref) - sum(r0)
    # 3 tile shapes + flux + 3 Yee sub-steps + lossy + ghosts + copies per
    # step; between graphs the sorts of the members (10 kernels each) and
    # each member's Gauss-law snapshot before its first step (3 at most)
    sorts = sum(30 // s.desc.sort_interval + 1 for s in ens)
    assert kernels <= 30 * 10 + 10 * sorts + 3 * len(ens)
    assert kernels < member_launches / 2
    for k, (a, b) in enumerate(zip(ens, ref)):
        assert np.array_equal(a.fields(), b.fields()), k
        assert np.array_equal(a.flux(), b.flux()), k
        pa, pb = a.particles(), b.particles()
        oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
        for key in ("x1", "x2", "ur", "uth", "uph", "qw"):
            assert np.array_equal(pa[key][oa], pb[key][ob]), (k, key)


def test_mixed_precision_ensemble_takes_the_branch_form():
    """Any FP64 member sends the ensemble to the per-member graph branches:
    FP32 members stay bit-identical to their own runs, FP64 members agree to
    the rounding of their atomic sums."""
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = [], []
    for m, prec in ((0, "fp32"), (1, "fp64"), (2, "fp32")):
        cfg = _member_cfg(m, prec)
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    P.ensemble_step(ens, 30)
    for s in ref:
        s.step(30)
    for k, (a, b) in enumerate(zip(ens, ref)):
        fa, fb = a.fields(), b.fields()
        if k != 1:
            assert np.array_equal(fa, fb), k
        else:
            assert np.max(np.abs(fa - fb)) <= 1e-13 * np.max(np.abs(fb)), k
        assert a.moments()["live"] == b.moments()["live"], k


def test_members_without_particles():
    """An empty member (no tile launch, its grid phases still run), one that
    starts empty and fills by surface injection during the batched steps, and
    a plasma member: each equals its own run bit for bit."""
    from paper_1407_1810_gb300 import picsar as P

    cfgs = [dict(_member_cfg(0), pairs_per_cell=0),
            dict(configs.CONFIGS["rotator-1024x1024"], nr=24, nth=16, pairs_per_cell=0, absorb_cells=4, t_spin=0.5),
            _member_cfg(1)]
    ens, ref = [], []
    for cfg in cfgs:
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    P.ensemble_step(ens, 30)
    for s in ref:
        s.step(30)
    for k, (a, b) in enumerate(zip(ens, ref)):
        assert np.array_equal(a.fields(), b.fields()), k
        ma, mb = a.moments(), b.moments()
        assert ma["live"] == mb["live"] and ma["injected"] == mb["injected"], k
    assert ens[0].moments()["live"] == 0 and ens[1].moments()["injected"] > 0


def test_long_blocks_and_single_steps():
    """Sort interval 1000: 150 steps are three graphs (64, 64 and 22 steps,
    the last one re-instantiated for its shorter length) with no sort between
    them; then 10 calls of one step each.  Every member stays bit-identical to
    its own run."""
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = [], []
    for m in range(4):
        cfg = dict(_member_cfg(m), sort_interval=1000)
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    P.ensemble_step(ens, 150)
    for _ in range(10):
        P.ensemble_step(ens, 1)
    for s in ref:
        s.step(160)
    for k, (a, b) in enumerate(zip(ens, ref)):
        assert np.array_equal(a.fields(), b.fields()), k
        assert a.moments()["live"] == b.moments()["live"] and a.moments()["step"] == 160, k


def test_more_members_than_one_tile_launch_holds():
    """52 members of one tile kind: the tile kernel takes its members'
    arguments as kernel parameters, at most 48 per launch, so each step's
    tile phase is two launches; every member stays bit-identical to its own
    run."""
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = [], []
    for m in range(52):
        cfg = dict(configs.CONFIGS["monopole-64x64"], nr=16, nth=16, pairs_per_cell=1, T=0.05 + 0.01 * m,
                   seed=100 + m, precision="fp32")
        s1, _, plasma, _ = setup(cfg)
        s2, _, _, _ = setup(cfg, plasma=plasma)
        ens.append(s1)
        ref.append(s2)
    kernels = P.ensemble_step(ens, 25)
    for s in ref:
        s.step(25)
    # per step: 2 tile launches + flux + 3 Yee sub-steps + lossy + ghosts + copies
    assert kernels >= 25 * 9
    for k, (a, b) in enumerate(zip(ens, ref)):
        assert np.array_equal(a.fields(), b.fields()), k
        assert a.moments()["live"] == b.moments()["live"], k


def test_ensemble_autotune_applies_one_choice_and_keeps_results():
    """pic_autotune_ensemble times the batched step on clones: the members do
    not advance, every member takes the chosen shape and interval, and the
    results stay bit-identical to independent steps (the deposit sums are
    exact whatever the tiles and sorts)."""
    from paper_1407_1810_gb300 import picsar as P

    ens, ref = _pairs(4, "fp32")
    P.ensemble_step(ens, 3)
    for s in ref:
        s.step(3)
    choice = P.autotune_ensemble(ens, trial_steps=10)
    assert choice["sort_interval"] in (10, 20, 40) and choice["tile_shape"] in (0, 1, 2)
    assert all(s.moments()["step"] == 3 for s in ens)
    P.ensemble_step(ens, 45)
    for s in ref:
        s.step(45)
    for k, (a, b) in enumerate(zip(ens, ref)):
        assert np.array_equal(a.fields(), b.fields()), k
        assert a.moments()["live"] == b.moments()["live"], k


def test_ensemble_member_against_the_oracle():
    """One member of a batched FP32 ensemble, 100 steps, against the FP64
    oracle run from the same state (following the member's branches at
    axis-crossing ties): fields within the FP32 bar of 1e-5, live count within
    the near-ties."""
    import oracle as O

    from paper_1407_1810_gb300 import picsar as P

    from gpu_common import maxnorm_rel, rel_l2

    O.build_oracle()
    ens, oracles = [], []
    for m in (4, 8, 9):
        s, o, _, _ = setup(_member_cfg(m))
        ens.append(s)
        oracles.append(o)
    P.ensemble_step(ens, 100)
    s, o = ens[1], oracles[1]
    o.set_axis_hints(s.axis_ties())
    o.step(100)
    fs, fo = s.fields(), o.fields()
    assert rel_l2(fs, fo) < 1e-5
    assert maxnorm_rel(fs, fo) < 1e-4
    n = o.num_particles()
    assert abs(s.moments()["live"] - n) <= max(1, 1e-4 * n)


def test_benchmark_ensemble_members_against_the_oracle():
    """The benchmark's own ensemble (`bench.py --workload ensemble-64`: 64
    members, grids 64-256 x 64-512, 1e4-2e6 particles), autotuned and advanced
    20 steps by the batched step; two of its members -- member 8 (256 x 256,
    2.6e5 particles) and member 36 (64 x 64, 1.26e6: 300 per cell, many work
    units per tile) -- against the oracle from the same FP32 state, following
    their axis ties: fields within the FP32 bar, live counts within the
    near-ties."""
    import bench
    import oracle as O

    from paper_1407_1810_gb300 import picsar as P

    from gpu_common import KEYS, MAX_FP32_SPHERICAL, close, follow_ties, fp32_state

    O.build_oracle()
    sims, states = [], {}
    for m in range(64):
        cfg = configs.ensemble_member_config(m)
        dt = configs.courant_dt(cfg)
        b0, qw = configs.physics(cfg, dt)
        s = P.Simulation(P.make_desc(**configs.desc_kwargs(cfg, dt, b0)))
        d = bench.ensemble_plasma(cfg, qw)
        s.load(*(d[k] for k in KEYS))
        sims.append(s)
        if m in (8, 36):
            states[m] = (cfg, dt, b0, fp32_state(d))
    P.autotune_ensemble(sims, trial_steps=10)
    P.ensemble_step(sims, 20)
    for m, (cfg, dt, b0, d) in states.items():
        o = O.Oracle(O.params(**configs.oracle_kwargs(cfg, dt, b0)))
        o.load(*(d[k] for k in KEYS))
        follow_ties(sims[m], o)
        o.step(20)
        close(sims[m].fields(), o.fields(), 1e-5, MAX_FP32_SPHERICAL)
        n = o.num_particles()
        assert abs(sims[m].moments()["live"] - n) <= max(1, 1e-4 * n), m

