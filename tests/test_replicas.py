"""The multi-GPU (replica) path on the CPU: two gloo ranks, each with its own volumes, agree on the
slowest rank's time and on the whole-job rate; the reference arm does its work on rank 0 only."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist

    from paper_1605_00133_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = 1.0 + rank  # rank 1 is the slow one
    tmax = replicas.max_over_ranks(local_seconds, dist, torch.device("cpu"))
    rate = replicas.whole_job_rate(3, world, tmax)
    seeds = replicas.volume_seeds(rank, 3)
    dist.destroy_process_group()
    q.put((rank, tmax, rate, seeds))


def test_two_gloo_ranks_agree_on_time_and_rate():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]          # the slowest rank's time on every rank
    assert [r[2] for r in res] == [3.0, 3.0]          # 3 units x 2 ranks / 2 s
    assert set(res[0][3]).isdisjoint(res[1][3])       # independent volumes


def test_single_process_needs_no_group():
    from paper_1605_00133_gb300 import replicas
    assert replicas.max_over_ranks(1.5) == 1.5
    assert replicas.whole_job_rate(10, 1, 2.0) == 5.0
    with pytest.raises(ValueError):
        replicas.volume_seeds(0, 101)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""
