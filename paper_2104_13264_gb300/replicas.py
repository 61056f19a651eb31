"""Replica sharding across ranks (one process per GPU; no data-path collective).

The proposals are independent draws indexed by their Philox sample index, so N
ranks draw disjoint index ranges and together produce exactly what one process
drawing all of them would: rank i takes, at step k, the B indices starting at
sample_offset(i, k).  The only collectives are the timing and the count of
accepted samples at the end (max of the ranks' times, sum of their counts).
"""


def sample_offset(rank, world, step, B):
    """First sample index of rank `rank` at step `step` (B proposals per rank and step)."""
    return (step * world + rank) * B


def mh_step_offset(rank, world, step, T):
    """First MH step index of the rank's chains at step `step` (T proposals per chain)."""
    return (step * world + rank) * T


def reduce_timing(ms, n_accepted, dist=None, device=None):
    """(max over ranks of ms, sum over ranks of n_accepted); identity without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), int(n_accepted)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(n_accepted)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))
