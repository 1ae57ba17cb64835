"""The multi-GPU path's host logic on CPU: two gloo ranks, each solving its own seeded
shard of independent reactors (here with the oracle, no GPU), combine the step's timing
(slowest rank) and converged counts (sum) the way bench.py does; shards are distinct."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port):
    import time

    import torch
    import torch.distributed as dist

    from oracle import psr_oracle as O
    from paper_2005_11468_gb300 import shard, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = synth.workload_mechanism("k10_b64")
        mech = O.Mechanism(synth.mechanism_text(spec))
        w = synth.WORKLOADS["k10_b64"]
        batch = synth.make_batch(spec, 6, seed=shard.shard_seed(synth.MECH_SEED_BASE + 10 * w["tag"] + 1, rank))
        t0 = time.perf_counter()
        res = O.solve_batch(mech, batch, indices=[0, 1])
        dt = time.perf_counter() - t0 + 0.01 * rank          # ranks take different times
        conv = float(np.sum(res["status"] == O.CONVERGED))
        # what every rank contributed, for the checks
        mine = torch.tensor([dt, conv, float(batch.Y_in.sum()), float(batch.T_in[0])], dtype=torch.float64)
        allv = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allv, mine)
        slowest = shard.reduce_max(dist, [dt])[0]
        total = shard.reduce_sum(dist, [conv])[0]
        assert slowest == max(v[0].item() for v in allv)
        assert total == sum(v[1].item() for v in allv)
        assert allv[0][3].item() != allv[1][3].item()          # distinct shards
        rate = shard.job_throughput(total, slowest)
        assert abs(rate - total / slowest) <= 1e-12 * rate
        assert total == 2.0 * world                            # every sampled reactor converged
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_rank_main, args=(2, _free_port()), nprocs=2, join=True)


def test_single_process_identity():
    from paper_2005_11468_gb300 import shard
    assert shard.reduce_max(None, [1.0, 2.0]) == [1.0, 2.0]
    assert shard.reduce_sum(None, [3.0]) == [3.0]
    assert shard.shard_seed(100, 0) == 100 and shard.shard_seed(100, 3) == 100 + 3 * shard.SHARD_STRIDE
    assert shard.job_throughput(10.0, 0.0) == 0.0
