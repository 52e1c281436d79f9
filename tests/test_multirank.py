"""The multi-rank logic of bench.py on CPU with two gloo ranks (127.0.0.1):
every rank solves its own seeded problem (replicas, weak scaling, no
data-path collective), the job time is the slowest rank's, the job rate
counts every rank's units, and the reference arm runs on rank 0 only."""
import argparse
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + 2.0 * rank, world, device="cpu")
    args = argparse.Namespace(workload="uniform_small", d=None, n=None, k=None, train=None)
    p = bench.generate(bench.workload(args), rank)
    q.put((rank, t, bench.job_rate(3, 4, world, t), float(np.asarray(p.A, np.float64).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        r, t, rate, asum = q.get(timeout=120)
        out[r] = (t, rate, asum)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the slowest rank's time (3 s) on both ranks, and 2 ranks × 4 steps × 3 units / 3 s
    assert out[0][0] == out[1][0] == 3.0
    assert out[0][1] == out[1][1] == 2 * 4 * 3 / 3.0
    # each rank its own problem: rank r draws from seed + r
    sys.path.insert(0, ROOT)
    import bench
    from paper_1502_01645_gb300 import workloads as W
    w = bench.WORKLOADS["uniform_small"]
    for r in range(2):
        ref = W.uniform_small(d=w["d"], n=w["n"], seed=w["seed"] + r)
        assert out[r][2] == float(np.asarray(ref.A, np.float64).sum())
    assert out[0][2] != out[1][2]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(10, 5, 1, 2.0) == 25.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="uniform_small", d=None, n=None, k=None, train=None,
                              algorithm="antilop", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
