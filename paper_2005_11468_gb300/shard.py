"""Reactors over ranks (one process per GPU).

Reactors are independent (the paper's batch of PSRs, Sec. 6). For weak scaling each rank
solves its own seeded shard and nothing on the data path is exchanged; ranks only combine
the step's timing (the slowest rank's time) and their converged counts (summed) to report
the job's throughput. A caller's own batch is split into contiguous reactor ranges of
nearly equal expected cost (`split_ranges`, with `reactor_cost` weights for batches that
mix mechanisms); each rank solves its range and the results are gathered once at the end.
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
SHARD_STRIDE = 1000   # seed offset between ranks' shards


def reactor_cost(K: int, I: int) -> float:
    """Expected relative cost of one reactor of a K-species, I-reaction mechanism, per Newton
    iteration: the LU of the (K+1)-square Jacobian (2/3 n^3 flops) plus the rate and Jacobian
    passes over the reactions (a few dozen operations and two exponentials per reaction,
    counted as 64). A balancing weight only: measured per-reactor times can replace it."""
    n = K + 1
    return (2.0 / 3.0) * n ** 3 + 64.0 * I


def split_ranges(costs, world: int):
    """Contiguous [lo, hi) ranges of a caller's batch, one per rank, whose summed expected
    costs are as equal as contiguous cuts allow: the cut between ranks r - 1 and r sits at
    the reactor boundary nearest to r / world of the total cost, so no rank's share exceeds
    total / world by more than its largest reactor. Ranks may get empty ranges."""
    import numpy as np
    c = np.asarray(costs, dtype=np.float64)
    if c.ndim != 1 or np.any(c < 0) or not np.all(np.isfinite(c)):
        raise ValueError("costs must be a 1-D array of finite non-negative numbers")
    if world < 1:
        raise ValueError("world must be >= 1")
    B = len(c)
    prefix = np.concatenate([[0.0], np.cumsum(c)])
    total = prefix[-1]
    cuts = [0]
    for r in range(1, world):
        k = int(np.searchsorted(prefix, total * r / world, side="left")) if total > 0 else (B * r) // world
        # the cut that leaves the two neighbouring ranks closer to their share
        if 0 < k <= B and abs(prefix[k - 1] - total * r / world) < abs(prefix[k] - total * r / world):
            k -= 1
        cuts.append(min(max(k, cuts[-1]), B))
    cuts.append(B)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gather_ranges(pg, local, ranges):
    """Every rank's result rows for its range of `split_ranges`, concatenated in the caller's
    reactor order (on every rank): one all_gather of equal-length padded pieces. `local` is
    this rank's [hi - lo, ...] tensor; `pg` the torch.distributed module or None (one rank)."""
    if pg is None:
        return local
    import torch
    m = max(hi - lo for lo, hi in ranges)
    pad = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.zeros_like(pad) for _ in ranges]
    pg.all_gather(parts, pad)
    return torch.cat([p[:hi - lo] for p, (lo, hi) in zip(parts, ranges)])


def shard_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s shard of a workload whose single-GPU batch uses base_seed."""
    return base_seed + SHARD_STRIDE * rank


def reduce_max(pg, values, device="cpu"):
    """Element-wise maximum over ranks of a list of floats (identity without a group)."""
    if pg is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return t.tolist()


def reduce_sum(pg, values, device="cpu"):
    """Element-wise sum over ranks of a list of floats (identity without a group)."""
    if pg is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return t.tolist()


def job_throughput(units_summed: float, slowest_seconds: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return units_summed / slowest_seconds if slowest_seconds > 0 else 0.0
