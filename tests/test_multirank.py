"""The multi-rank path of bench.py, on the CPU (gloo, world size 2).

Probes are independent within a frame, so N GPUs run N full replicas of the update with no
collective on the data path (weak scaling). What is shared between the ranks is host
logic: each timing becomes the slowest rank's, the whole-job rate counts every rank's
units over that time, rank 0 alone prints the line, and in the reference arm (the oracle)
only rank 0 works while the other ranks exit at once. These tests run that logic as two
gloo ranks; nothing here needs a GPU.
"""
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        times = bench.max_over_ranks([10.0 + rank, 7.0 - 2 * rank, 3.5], world)
        rate = bench.whole_job_rate(world, 1000.0, 4, times[0])
        q.put((rank, times, rate))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, times, rate in got:
        assert times == [11.0, 7.0, 3.5], (rank, times)  # the maximum of each value over the ranks
        assert rate == 2 * 1000.0 * 4 / (11.0 / 1e3)     # both ranks' units over the slowest time


def test_single_rank_values_pass_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1, 2.5], 1) == [1.0, 2.5]
    assert bench.whole_job_rate(1, 10.0, 3, 30.0) == 1000.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""  # rank 0 alone prints the line
