"""Host-side bookkeeping of an ensemble sharded over ranks (one GPU each).

Trajectories are independent, so rank r of W runs trajectories
[offset(r), offset(r) + M_r) with that offset as `traj_offset` of its context;
the Philox counter then reproduces exactly the rows an unsharded run would
produce. The only exchange is at the end: the per-trajectory window means
(M_r x 5 doubles per rank) are gathered in rank order and reduced once
(twa_reduce_moments). Nothing is exchanged during the steps.
"""
import numpy as np


def shard(M_total, world, rank):
    """(offset, count) of rank's contiguous share of M_total trajectories."""
    base, extra = divmod(int(M_total), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def gather_means(local, group=None):
    """All-gather per-trajectory window means [M_r][5] from every rank and return
    them concatenated in rank order ([sum M_r][5], float64 numpy)."""
    import torch
    import torch.distributed as dist
    local = np.ascontiguousarray(local, dtype=np.float64)
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    n = torch.tensor([local.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    width = max(counts)
    buf = torch.zeros((width, 5), dtype=torch.float64, device=dev)
    buf[: local.shape[0]] = torch.from_numpy(local).to(dev)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([p[:c].cpu().numpy() for p, c in zip(parts, counts)], axis=0)
