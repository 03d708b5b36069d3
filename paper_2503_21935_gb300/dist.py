"""Multi-GPU data parallelism for the matrix-element path.

Events are independent (Sec. 2: event-level data parallelism), so N GPUs run N
replicas of the process, each on its own contiguous range of events; the only
communication is the timing reduction (max over ranks).  There is no data-path
collective.
"""


def event_range(rank, world, nevt_per_rank):
    """(first, count) of the events rank `rank` evaluates under weak scaling."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank * nevt_per_rank, nevt_per_rank


def split_range(rank, world, nevt_total):
    """(first, count) for strong scaling: nevt_total events split into contiguous ranges."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, rem = divmod(nevt_total, world)
    first = rank * base + min(rank, rem)
    return first, base + (1 if rank < rem else 0)


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks of the default process group (value if not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
