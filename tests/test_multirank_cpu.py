"""The multi-rank path of bench.py on CPU (gloo, world size 2).

Several GPUs run independent replicas (one lattice per rank, seed = rank);
the only exchanges are the timing barrier and the maximum of the ranks'
elapsed times.  These tests run that host logic over gloo without a GPU.
"""

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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1206_0675_gb300 import fields
    ms = [12.5, 20.0][rank]
    tdist.barrier()
    slowest = bench.max_over_ranks(ms, "cpu")
    rate = bench.whole_job_rate(10, world, slowest)
    U = fields.random_links((2, 2, 2, 2), bench.EPS, rank)   # each replica its own field
    sums = [None] * world
    tdist.all_gather_object(sums, complex(U.sum()))
    tdist.destroy_process_group()
    q.put((rank, slowest, rate, sums))


def test_two_gloo_ranks_take_the_slowest_time_and_own_fields():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, sums in out:
        assert slowest == 20.0                  # the max over ranks, on every rank
        assert rate == pytest.approx(1000.0)    # 2 ranks x 10 steps in 20 ms
        assert sums[0] != sums[1]               # independent replicas


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
