"""Multi-process host logic of the benchmark, on CPU.

A solve does not shard: with N ranks every rank solves its own problem
(replicas, no collective on the data path), the job's step time is the
slowest rank's, and the whole-job throughput counts every rank's solve.
Two gloo ranks check the max-over-ranks reduction and the throughput; a
non-zero rank of the reference arm (the CPU oracle runs on rank 0 only)
must exit at once without output.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench.dist_env()
        ms = bench.rank_max(10.0 + 3.0 * rank, world, "cpu")
        q.put((rank, env, ms, bench.job_value(world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_solve():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, env, ms, value in got:
        assert env == (rank, 2, rank)
        assert ms == 13.0                                 # rank 1's 13 ms, on both ranks
        assert value == pytest.approx(2 * 1000.0 / 13.0)  # two solves per 13 ms step


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(5.0, 1) == 5.0
    assert bench.job_value(1, 20.0) == pytest.approx(50.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_each_rank_draws_its_own_problem(monkeypatch):
    """Replicas: every rank solves an independent problem of the same shape
    (seed offset by rank), so the job's throughput counts N distinct solves."""
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "M_", 64)
    monkeypatch.setattr(bench, "N_", 32)
    monkeypatch.setattr(bench, "P_", 4)
    g0, g1 = bench.make_inputs(0, "cpu"), bench.make_inputs(1, "cpu")
    assert g0["A"].shape == g1["A"].shape == (64, 32) and g0["B"].shape == (4, 32)
    assert not (g0["A"] == g1["A"]).all()
    assert (bench.make_inputs(1, "cpu")["d"] == g1["d"]).all()
    assert bench.config("fp32") == bench.config("fp32") and bench.config()["workload"] == bench.WORKLOAD
