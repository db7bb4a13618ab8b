"""The N > 1 path of bench.py on CPU (gloo, world size 2): one independent replica per rank, no
data-path collective. The job's time is the max over ranks and its value counts the units of
every rank; under torchrun the reference arm runs on rank 0 only and the other ranks exit 0."""
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms = bench.job_time_ms(local_ms, dist, device="cpu")
    rate = bench.whole_job_rate(1000, 5, ms, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_ranks_take_the_max_time_and_count_both_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 150.0                               # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 1000 * 5 / 0.150)  # units of both replicas over that time


def test_single_rank_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(42.0, None) == 42.0
    assert bench.whole_job_rate(10, 3, 1000.0, 1) == pytest.approx(30.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "2", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
