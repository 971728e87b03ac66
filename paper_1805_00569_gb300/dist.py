"""Multi-process form of the partitioned hot path.

Partitions are independent problems (Alg. BKRR2: no communication during
training), so ranks shard whole units of work and exchange only the model
scores at the end -- the single reduction of Alg. BKRR2's model choice / the argmin of
the best model.  Each rank is one process on one GPU; the exchange is one
all-gather of a few doubles through torch.distributed (NCCL on GPUs, gloo on
CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(units: int, rank: int, world: int):
    """Contiguous, balanced share [lo, hi) of `units` for `rank`."""
    base, extra = divmod(units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


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
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    buf = [torch.zeros(2, dtype=torch.float64, device=dev) for _ in range(dist.get_world_size())]
    dist.all_gather(buf, mine.to(dev))
    best = None
    for b in buf:
        v, idx = float(b[0].item()), float(b[1].item())
        if best is None or v < best[0] or (v == best[0] and idx < best[1]):
            best = (v, idx)
    return int(best[1]), best[0]


def max_over_ranks(x: float) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
