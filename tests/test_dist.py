"""Multi-process host logic (gloo, world size 2, CPU): sharding of independent
units, the global best-model all-gather (lowest MSE, lowest global index on
ties) and the max-over-ranks timing reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_00569_gb300 import dist as kd


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cases, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for local, offset in cases[rank]:
            res.append(kd.global_best(torch.tensor(local, dtype=torch.float64), offset))
        res.append(kd.max_over_ranks(float(rank) * 1.5 + 0.25))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_shard_covers_units_once():
    for units in (0, 1, 5, 96, 97, 1000):
        for world in (1, 2, 3, 8):
            spans = [kd.shard(units, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == units
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_global_best_and_max_over_two_gloo_ranks():
    # per rank: (local MSEs, global index of its first model)
    cases = {
        0: [([0.5, 0.2, 0.9], 0), ([0.3, 0.1], 0), ([], 0), ([0.7], 0)],
        1: [([0.4, 0.2, 0.3], 3), ([0.1, 0.1], 2), ([0.6], 1), ([0.7], 1)],
    }
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, port, cases, out), nprocs=2, join=True, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0 == r1  # every rank agrees
    best = r0[:4]
    assert best[0] == (1, 0.2)      # tie 0.2 at global 1 (rank 0) and 4 (rank 1): lowest index
    assert best[1] == (1, 0.1)      # tie across ranks at global 1, 2, 3
    assert best[2] == (1, 0.6)      # rank 0 has no models
    assert best[3] == (0, 0.7)      # equal MSE, lower global index wins
    assert r0[4] == pytest.approx(1.75)
