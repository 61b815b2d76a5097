"""The multi-GPU benchmark's replica logic with two gloo ranks on the CPU:
the step time is the maximum over ranks, the throughput counts both ranks'
solves, each rank solves its own system, and the reference arm's extra ranks
exit without work (rank 0 alone times the oracle)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

from paper_2312_09376_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = replicas.env()
    ms = 10.0 + 5.0 * r                     # rank 1 is the slower replica
    m = replicas.max_over_ranks(ms, dist)
    v = replicas.aggregate_tflops(w, 2e12, m)
    dist.barrier()
    q.put((r, w, local, m, v, replicas.system_seed(r)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
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
    (r0, w0, l0, m0, v0, s0), (r1, w1, l1, m1, v1, s1) = out
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert m0 == m1 == 15.0                 # both ranks report the slowest time
    assert v0 == v1 == pytest.approx(2 * 2e12 / 15e-3 / 1e12)
    assert s0 != s1                         # each replica solves its own system


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate_tflops(1, 1e12, 1000.0) == pytest.approx(1.0)


def test_reference_arm_extra_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
