"""Running independent enforcements on several GPUs, one process per GPU.

Enforcement items (a network with one domain state) are independent
problems, so ranks share nothing on the data path: each rank takes a
contiguous, balanced share of the items, and only timings and counts are
reduced across ranks (for reporting).  No collective runs inside an
enforcement."""


def shard_range(n_items, rank, world):
    """Contiguous share [start, stop) of rank `rank` among `world` ranks; the
    shares partition [0, n_items) and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world: %d/%d" % (rank, world))
    base, extra = divmod(int(n_items), world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _reduce(value, op_name):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    backend = dist.get_backend()
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(value):
    """Largest value over all ranks (the slowest rank's time)."""
    return _reduce(value, "MAX")


def sum_over_ranks(value):
    """Sum over all ranks (units processed by the whole job)."""
    return _reduce(value, "SUM")
