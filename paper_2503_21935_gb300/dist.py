"""Multi-GPU data parallelism for the matrix-element path and the learned unweighting.

Events are independent (Sec. 2: event-level data parallelism), so N GPUs run N
replicas of the process, each on its own contiguous range of events; |M|^2 needs
no communication at all.  Two steps around it do exchange data:

  * unweighting: the ranks agree on the weight statistics before accept/reject,
    one collective of (max w, sum w, N) per batch (and, for quantile maxima, one
    gather of the calibration weights), so that every rank uses the same maxima
    and the union of the ranks' unweighted events is the sample one rank would
    draw from all the events;
  * surrogate training: data-parallel replicas of the network average their
    gradients (weighted by batch size) with one all-reduce per step and apply
    the same Adam step, so the replicas stay identical.

Each collective has a pure combination function beside it (the reduction over a
list of per-rank values in rank order), which is what the collective computes
and what a single process uses to emulate several ranks.
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


def _initialised():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def rank_world():
    """(rank, world size) of the default process group, (0, 1) without one."""
    import torch.distributed as dist
    if not _initialised():
        return 0, 1
    return dist.get_rank(), dist.get_world_size()


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks of the default process group (value if not initialised)."""
    import torch
    import torch.distributed as dist
    if not _initialised():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ weight statistics
def combine_weight_stats(stats):
    """(max w, sum w, N) over ranks from the per-rank triples in rank order: the maximum, the sum
    of the per-rank sums taken in rank order (so every rank gets the same bits), the event count."""
    mx, sw, n = float("-inf"), 0.0, 0
    for m, s, k in stats:
        mx = max(mx, float(m))
        sw += float(s)
        n += int(k)
    return mx, sw, n


def allreduce_weight_stats(max_w, sum_w, n, device=None):
    """The global (max w, sum w, N) of one batch: one all-gather of the three scalars, combined in
    rank order by combine_weight_stats (identical on every rank)."""
    import torch
    import torch.distributed as dist
    if not _initialised():
        return combine_weight_stats([(max_w, sum_w, n)])
    mine = torch.tensor([float(max_w), float(sum_w), float(n)], dtype=torch.float64, device=device)
    parts = [torch.empty_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, mine)
    return combine_weight_stats([tuple(p.tolist()) for p in parts])


def combine_sums(parts):
    """Element-wise sums over ranks of per-rank vectors of sums, taken in rank order."""
    acc = [0.0] * len(parts[0])
    for p in parts:
        acc = [a + float(v) for a, v in zip(acc, p)]
    return acc


def allreduce_sums(values, device=None):
    """Global sums of a short vector of per-rank sums (moments, counts): one all-gather, combined
    in rank order by combine_sums (identical on every rank)."""
    import torch
    import torch.distributed as dist
    if not _initialised():
        return combine_sums([values])
    mine = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    parts = [torch.empty_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, mine)
    return combine_sums([p.tolist() for p in parts])


def gather_samples(x):
    """All ranks' 1-D tensors concatenated in rank order (every rank gets the whole union): the
    calibration weights from which quantile maxima are taken.  Lengths may differ by rank."""
    import torch
    import torch.distributed as dist
    if not _initialised():
        return x
    world = dist.get_world_size()
    n = torch.tensor([x.numel()], dtype=torch.int64, device=x.device)
    sizes = [torch.empty_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(s.item()) for s in sizes]
    top = max(sizes)
    pad = torch.zeros(top, dtype=x.dtype, device=x.device)
    pad[: x.numel()] = x
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:k] for p, k in zip(parts, sizes)])


# ------------------------------------------------------------------ gradients
def combine_gradients(grads, counts):
    """Gradient of the mean loss over the union of the ranks' batches from each rank's gradient of
    its own mean loss: sum_r n_r g_r / sum_r n_r (rank order)."""
    total = sum(int(c) for c in counts)
    acc = None
    for g, c in zip(grads, counts):
        term = g * (float(c) / total)
        acc = term if acc is None else acc + term
    return acc


def allreduce_gradients(grad, n):
    """In-place average of a replica's gradient over all ranks, weighted by the ranks' batch sizes
    n: one all-reduce of (n g, n); returns the total batch size."""
    import torch
    import torch.distributed as dist
    if not _initialised():
        return int(n)
    buf = torch.empty(grad.numel() + 1, dtype=torch.float64 if grad.dtype == torch.float64 else torch.float32,
                      device=grad.device)
    buf[:-1] = grad.reshape(-1) * float(n)
    buf[-1] = float(n)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    total = float(buf[-1].item())
    grad.copy_((buf[:-1] / total).reshape(grad.shape))
    return int(round(total))
