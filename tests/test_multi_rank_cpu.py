"""World-size-2 gloo test of the multi-GPU host logic on CPU.

Each rank solves its own runs (the FP64 oracle stands in for the device
path here), seeds are distinct per rank, and the global best is reduced
with a single all-gather; the result must equal a single-process solve of
both ranks' runs."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_01050_gb300 import multi


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    import workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    J, _ = workloads.sk_pm1(12, 3)
    pb = oracle.Problem.dense(J)
    beta, alpha = workloads.autotune_params(3, rank)
    res = oracle.run(pb, 150, 4, 3, multi.rank_seed(9, rank), beta, alpha)
    e, r, run, s = multi.reduce_best(res["best_energy"], res["best_spins"])
    t = multi.max_over_ranks(float(rank + 1))
    out[rank] = (e, r, run, s.tolist(), t, res["best_energy"].tolist())
    dist.destroy_process_group()


def test_two_rank_best_reduction_matches_single_process():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0][:4] == out[1][:4]            # every rank gets the same answer
    assert out[0][4] == out[1][4] == 2.0       # slowest rank's value
    allE = [(e, rk, i) for rk in range(world) for i, e in enumerate(out[rk][5])]
    best = min(allE)
    assert (out[0][0], out[0][1], out[0][2]) == best
    import oracle
    import workloads
    J, _ = workloads.sk_pm1(12, 3)
    assert oracle.energy(oracle.Problem.dense(J), np.array(out[0][3], dtype=np.int8)) == out[0][0]


def test_seed_and_split_helpers():
    assert multi.rank_seed(5, 0) == 5 and multi.rank_seed(5, 1) != multi.rank_seed(5, 2)
    parts = [multi.split_runs(10, 3, r) for r in range(3)]
    assert parts == [(0, 4), (4, 3), (7, 3)]
    assert sum(c for _, c in parts) == 10
    e, rk, run, s = multi.reduce_best([3.0, -1.0, -1.0], np.eye(3, dtype=np.int8))
    assert (e, rk, run) == (-1.0, 0, 1) and s.tolist() == [0, 1, 0]
