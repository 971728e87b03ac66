"""Multi-process host logic (gloo, world size 2, CPU): sharding of independent
units, LPT assignment of whole partitions, the K-means block-sum exchange
(sharded centres equal the one-process centres bit for bit), the score
all-gather and global best-model choice (lowest MSE, lowest global index on
ties) and the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
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


# ------------------------------------------------- sharded partitions (8(e))
def test_lpt_balances_cubic_costs_deterministically():
    sizes = [500, 16000, 1200, 7000, 7000, 300, 9000, 2500]
    parts = kd.lpt_assign([m ** 3 for m in sizes], 3)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    # decreasing cubes 1, 6, 3 = 4, 7, 2, 0, 5: the two largest each fill a
    # rank, the rest all fit under the second largest on the third rank
    assert parts == [[1], [6], [0, 2, 3, 4, 5, 7]]
    loads = [sum(sizes[i] ** 3 for i in p) for p in parts]
    assert max(loads) == 16000 ** 3 and loads[2] < 9000 ** 3
    assert kd.lpt_assign([1.0] * 5, 2) == [[0, 2, 4], [1, 3]]
    assert kd.lpt_assign([], 2) == [[], []]


def test_partition_subset_keeps_partition_order():
    perm = torch.arange(10, dtype=torch.int64).flip(0)
    sub, off = kd.partition_subset(perm, [0, 3, 3, 7, 10], [1, 3])
    assert sub.tolist() == [2, 1, 0] and off.tolist() == [0, 0, 3]  # partition 1 is empty
    sub, off = kd.partition_subset(perm, [0, 3, 3, 7, 10], [2, 3])
    assert sub.tolist() == [6, 5, 4, 3, 2, 1, 0] and off.tolist() == [0, 4, 7]


class _OracleKmeansOps:
    """The three Alg. 2 steps from the CPU oracle, as torch tensors."""

    def assign(self, X, C):
        import oracle
        return torch.from_numpy(oracle.assign(X.numpy(), C.numpy()))

    def block_sums(self, X, a, k):
        import oracle
        s, c = oracle.block_sums(X.numpy(), a.numpy(), k)
        return torch.from_numpy(s), torch.from_numpy(c)

    def combine(self, S, Cn, C):
        import oracle
        return torch.from_numpy(oracle.tree_combine(S.numpy(), Cn.numpy(), C.numpy()))


def _kmeans_worker(rank, world, port, X, init, iters, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Xt = torch.from_numpy(X)
        C0 = Xt[torch.from_numpy(init)].clone()
        C, a = kd.kmeans_sharded(_OracleKmeansOps(), Xt, C0, iters)
        # per-model scores of the partitions this rank owns (LPT on m^3),
        # gathered and reduced to the best model in model-index order
        sizes = torch.bincount(a.long(), minlength=C.shape[0]).tolist()
        owned = kd.lpt_assign([m ** 3 for m in sizes], world)[rank]
        G = 2
        gidx = [j * G + g for j in owned for g in range(G)]
        local = torch.tensor([((j * 7 + g * 3) % 5) / 4.0 for j in owned for g in range(G)], dtype=torch.float64)
        scores = kd.gather_scores(local, gidx, C.shape[0] * G)
        out[rank] = (C.numpy().copy(), a.numpy().copy(), kd.best_of(scores), owned)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n,d,k,iters", [(5000, 7, 6, 5), (2048, 3, 4, 3), (3000, 12, 9, 0)])
def test_sharded_kmeans_and_global_best_match_one_process(n, d, k, iters):
    """Two gloo ranks, each owning a contiguous range of the 1024-row blocks:
    the centres and every assignment equal the one-process Alg. 2 bit for bit
    (the block sums are exchanged and combined in the canonical tree), the
    LPT split covers every partition once, and the best model from the
    gathered scores is the one-process best."""
    import oracle
    rng = np.random.default_rng(n + d)
    Cc = 3.0 * rng.standard_normal((k, d))
    X = Cc[rng.integers(0, k, n)] + rng.standard_normal((n, d))
    init = rng.choice(n, k, replace=False).astype(np.int64)
    oC, oc, _ = oracle.kmeans(X, k, init, iters)
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_kmeans_worker, args=(2, port, X, init, iters, out), nprocs=2, join=True,
                           start_method="spawn")
        res = [out[0], out[1]]
    for C, a, _, _ in res:
        assert np.array_equal(C.view(np.uint64), oC.view(np.uint64))
        assert np.array_equal(a, oc)
    assert res[0][2] == res[1][2]
    assert sorted(res[0][3] + res[1][3]) == list(range(k))
    scores = torch.tensor([((j * 7 + g * 3) % 5) / 4.0 for j in range(k) for g in range(2)], dtype=torch.float64)
    assert res[0][2] == kd.best_of(scores)
