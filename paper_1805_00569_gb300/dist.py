"""Multi-process form of the partitioned hot path.

Partitions are independent problems (Alg. BKRR2: no communication during
training), so ranks own whole partitions and exchange only

* the model scores at the end -- the single reduction of Alg. BKRR2's model
  choice: one all-gather of the p * G MSEs, the best model taken in
  model-index order (lowest MSE, lowest index on ties); and
* for K-means partitions (Alg. 2, KKRR2 Sec. 4.2), once per round, the
  per-block centre sums: every rank holds a contiguous range of 1024-row
  blocks, computes their sums for its rows, and after one all-gather every
  rank combines all blocks in the same canonical tree, so the centres (and
  hence every assignment) are the same bits at any number of ranks.

Whole partitions go to ranks by LPT (longest processing time first) on the
Cholesky cost m_i^3.  Test rows are replicated.  Each rank is one process on
one GPU; the exchanges go through torch.distributed (NCCL on GPUs, gloo on
CPU).  The K-means driver takes its three steps as callables, so the same
exchange runs over the GPU library (``gpu_kmeans_ops``) or over any other
implementation of the steps.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

BLOCK = 1024  # rows per canonical centre-sum block


def _world():
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def _comm_device():
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def shard(units: int, rank: int, world: int):
    """Contiguous, balanced share [lo, hi) of `units` for `rank`."""
    base, extra = divmod(units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def lpt_assign(costs, world: int):
    """Longest processing time first: units in decreasing cost (ties: lower
    index first) each go to the rank with the least load so far (ties: lower
    rank).  Returns each rank's unit indices in ascending order."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def partition_subset(perm: torch.Tensor, offsets, owned):
    """perm / offsets restricted to the partitions in `owned` (ascending):
    the rank's own rows in partition order, for krr_fit_batch on the full X."""
    off = [int(v) for v in (offsets.tolist() if hasattr(offsets, "tolist") else offsets)]
    pieces = [perm[off[j]:off[j + 1]] for j in owned]
    sub = torch.cat(pieces) if pieces else perm[:0]
    so = [0]
    for j in owned:
        so.append(so[-1] + off[j + 1] - off[j])
    return sub, torch.tensor(so, dtype=torch.int64, device=perm.device)


def all_gather_uneven(local: torch.Tensor, counts):
    """Concatenation over ranks (rank order) of tensors whose first dimension
    is counts[rank]; equal-size buffers on the wire, trimmed on arrival."""
    rank, world = _world()
    if world == 1:
        return local
    dev = _comm_device()
    width = max(counts)
    shape = (width,) + tuple(local.shape[1:])
    buf = torch.zeros(shape, dtype=local.dtype, device=dev)
    if local.shape[0]:
        buf[:local.shape[0]] = local.to(dev)
    out = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(out, buf)
    return torch.cat([o[:c] for o, c in zip(out, counts)]).to(local.device)


def kmeans_sharded(ops, X, C0, iters: int):
    """Alg. 2 over ranks that each own a contiguous range of the 1024-row
    blocks of X (the full training set, replicated).  Per round: assignment
    of the own rows, block sums of the own blocks, one all-gather of every
    block's sums and counts, the canonical combine on every rank.  After the
    rounds, a final assignment with the final centres and one all-gather of
    the assignment.  Returns (centres, assignment of all n rows).

    ops: assign(X_rows, C) -> int32 [rows]; block_sums(X_rows, a, k) ->
    (sums [nb, k, d] float64, counts [nb, k] int64); combine(sums, counts,
    C) -> C."""
    rank, world = _world()
    n = X.shape[0]
    k = C0.shape[0]
    nblk = -(-n // BLOCK)
    spans = [shard(nblk, r, world) for r in range(world)]
    b0, b1 = spans[rank]
    r0, r1 = b0 * BLOCK, min(b1 * BLOCK, n)
    Xl = X[r0:r1]
    bcounts = [hi - lo for lo, hi in spans]
    rcounts = [min(hi * BLOCK, n) - min(lo * BLOCK, n) for lo, hi in spans]
    C = C0
    for _ in range(iters):
        a = ops.assign(Xl, C)
        s, c = ops.block_sums(Xl, a, k)
        S = all_gather_uneven(s, bcounts)
        Cn = all_gather_uneven(c, bcounts)
        C = ops.combine(S, Cn, C)
    a = ops.assign(Xl, C)
    return C, all_gather_uneven(a, rcounts)


class gpu_kmeans_ops:
    """The three K-means steps on the GPU library (one context)."""

    def __init__(self, ctx):
        self.ctx = ctx

    def assign(self, X, C):
        from . import krr_kmeans_assign
        return krr_kmeans_assign(self.ctx, X, C)

    def block_sums(self, X, a, k):
        from . import krr_kmeans_block_sums
        return krr_kmeans_block_sums(self.ctx, X, a, k)

    def combine(self, S, Cn, C):
        from . import krr_kmeans_combine
        return krr_kmeans_combine(self.ctx, S, Cn, C)


def gather_scores(local_mse: torch.Tensor, global_index, total: int):
    """Every model's score on every rank: one all-gather of (index, mse)
    pairs; returns the [total] float64 vector in model-index order."""
    rank, world = _world()
    idx = torch.as_tensor(list(global_index), dtype=torch.float64)
    mine = torch.stack([idx, local_mse.detach().to("cpu", torch.float64).flatten()], 1)
    if world == 1:
        allp = mine
    else:
        cnt = torch.tensor([mine.shape[0]], dtype=torch.int64, device=_comm_device())
        got = [torch.zeros_like(cnt) for _ in range(world)]
        dist.all_gather(got, cnt)
        counts = [int(g.item()) for g in got]
        allp = all_gather_uneven(mine, counts)
    out = torch.full((total,), float("inf"), dtype=torch.float64)
    out[allp[:, 0].long()] = allp[:, 1]
    return out


def best_of(scores: torch.Tensor):
    """Lowest score, lowest index on ties (strict <, model-index order)."""
    best = 0
    for i in range(1, scores.shape[0]):
        if scores[i] < scores[best]:
            best = i
    return best, float(scores[best])


def global_best(local_mse: torch.Tensor, local_offset: int):
    """Lowest MSE over all ranks' models (ties: lowest global model index).

    local_mse: this rank's per-model MSE (any device); local_offset: global
    index of its first model.  Returns (global index, mse) on every rank."""
    mse = local_mse.detach().to(torch.float64).flatten()
    if mse.numel() > 0:
        i = int(torch.argmin(mse).item())  # first minimum = lowest index
        mine = torch.tensor([float(mse[i].item()), float(local_offset + i)], dtype=torch.float64)
    else:
        mine = torch.tensor([float("inf"), float("inf")], dtype=torch.float64)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(mine[1].item()), float(mine[0].item())
    dev = _comm_device()
    buf = [torch.zeros(2, dtype=torch.float64, device=dev) for _ in range(dist.get_world_size())]
    dist.all_gather(buf, mine.to(dev))
    best = None
    for b in buf:
        v, idx = float(b[0].item()), float(b[1].item())
        if best is None or v < best[0] or (v == best[0] and idx < best[1]):
            best = (v, idx)
    return int(best[1]), best[0]


def sum_over_ranks(t: torch.Tensor) -> torch.Tensor:
    """Element-wise sum of a tensor over ranks (a copy; the input at one rank)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t.clone()
    buf = t.detach().to(_comm_device()).clone()
    dist.all_reduce(buf)
    return buf.to(t.device)


def max_over_ranks(x: float) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_comm_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
