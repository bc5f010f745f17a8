"""The benchmark's multi-rank logic on CPU: two gloo ranks (the same code runs
over NCCL with one rank per GPU).  A run of N independent replicas reports
the slowest rank's time and the particle-steps of all ranks; the reference
arm runs on rank 0 alone."""
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, local = bench.dist_env()
    ms, units = bench.combine_ranks(10.0 + 5.0 * rank, 100.0 * (rank + 1), "cpu")
    q.put((r, w, local, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_max_time_and_total_work():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    for o in out:
        assert o[3] == 15.0 and o[4] == 300.0  # max of 10 and 15 ms; 100 + 200 particle-steps


def test_single_process_combines_to_its_own_values():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.combine_ranks(12.5, 7.0, "cpu") == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.reference_arm(bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"]))
    assert capsys.readouterr().out == ""


def test_ensemble_members_split_across_ranks():
    """The ensemble's members are independent: N ranks hold disjoint sets of
    them that together are the whole ensemble, within one member of even."""
    sys.path.insert(0, ROOT)
    import bench

    for world in (1, 2, 3, 4, 8):
        parts = [bench.ensemble_members(64, r, world) for r in range(world)]
        flat = sorted(m for p in parts for m in p)
        assert flat == list(range(64))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
