"""The multi-rank host logic of bench.py on CPU: world-size-2 gloo ranks (the
GPU run uses NCCL with the same calls).  Each rank advances its own replica
(weak scaling, no data-path collective); the job time is the slowest rank's
and the value counts every rank's sites."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 17.25][rank]                 # the second rank is the slow one
    job = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (job, bench.job_value(1000, 10, world, job), bench.replica_seeds(1, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_sites():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 17.25
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000 * 10 / 17.25e-3 / 1e6)
    assert res[0][2] != res[1][2]            # independent replicas


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.job_value(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 2e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun only rank 0 times the checker; the other ranks exit at once
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
