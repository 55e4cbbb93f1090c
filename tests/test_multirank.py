"""The multi-GPU path of bench.py on the host: two gloo ranks on the CPU.

The workload shards into independent replicas (each rank solves its own
problem, instance tag = rank; no data-path collective), and the job's time
is the slowest rank's.  These tests run the rank plumbing itself -- the
max-over-ranks reduction, the barrier, the replica assignment and the
whole-job throughput -- with the gloo backend, world size 2, and check that
the oracle-side noise of the two replicas differs (distinct tags, distinct
Philox streams).  The reference arm under torchrun prints only on rank 0.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import scenarios
    slowest = bench.max_over_ranks(torch, world, 10.0 + 5.0 * rank)
    bench.barrier(torch, world)
    inst = bench.replica_instance(scenarios.WORKLOADS["holo2d_n4"](), rank)
    q.put((rank, slowest, inst.tag, bench.job_throughput(1000.0, world, slowest)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
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
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 15.0 for o in out)            # the slowest rank's time on every rank
    assert [o[2] for o in out] == [0, 1]             # one replica (tag) per rank
    assert all(abs(o[3] - 2000.0 / 0.015) < 1e-6 for o in out)   # both ranks' units over the slowest time


def test_replicas_draw_distinct_noise(oracle_lib):
    """Tags 0 and 1 give different Philox streams for the same sample."""
    import scenarios
    from helpers import oracle_params, oracle_problem, round_instance
    a = round_instance(scenarios.WORKLOADS["holo2d_n4"]())
    b = round_instance(scenarios.WORKLOADS["holo2d_n4"]())
    b.tag = 1
    ea = oracle_lib.noise_block(oracle_problem(oracle_lib, a), oracle_params(oracle_lib, a), 0, 10, 0)
    eb = oracle_lib.noise_block(oracle_problem(oracle_lib, b), oracle_params(oracle_lib, b), 0, 10, 0)
    assert not np.allclose(ea, eb)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
