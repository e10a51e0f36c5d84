"""Multi-process helpers (one process per GPU, torch.distributed).

The worm-LBM grid of one run does not shard without a halo exchange; the library runs
independent problems per rank instead: replicas of one grid, or disjoint shares of a
batch of instances.  Nothing here touches the data path: ranks only agree on their share
of the work and on the slowest rank's time.
"""


def shard(n_items, rank, world):
    """Indices of the items rank `rank` of `world` owns: a contiguous, balanced block."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def shard_by_cost(costs, rank, world):
    """Greedy longest-processing-time assignment of weighted items (e.g. Q * cells of
    each instance) to ranks; every rank computes the same assignment."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    owner = [0] * len(costs)
    for k in order:
        r = min(range(world), key=lambda j: (load[j], j))
        owner[k] = r
        load[r] += costs[k]
    return [k for k in range(len(costs)) if owner[k] == rank]


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks (the job's time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
