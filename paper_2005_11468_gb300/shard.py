"""Weak-scaling shards of independent reactors over ranks (one process per GPU).

Reactors are independent (the paper's batch of PSRs, Sec. 6), so each rank solves its own
seeded shard and nothing on the data path is exchanged; ranks only combine the step's
timing (the slowest rank's time) and their converged counts (summed) to report the job's
throughput. Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
SHARD_STRIDE = 1000   # seed offset between ranks' shards


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
