"""The multi-GPU path's host logic on CPU: two gloo ranks, each solving its own seeded
shard of independent reactors (here with the oracle, no GPU), combine the step's timing
(slowest rank) and converged counts (sum) the way bench.py does; shards are distinct. A
caller's batch split into cost-balanced contiguous ranges and gathered back equals the
one-process solve."""
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


def _split_main(rank, world, port):
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
        batch = synth.make_batch(spec, 5, seed=77)            # the caller's batch, the same on every rank
        costs = [1.0, 3.0, 1.0, 1.0, 2.0]                      # e.g. from an earlier solve's iteration counts
        ranges = shard.split_ranges(costs, world)
        lo, hi = ranges[rank]
        res = O.solve_batch(mech, batch, indices=list(range(lo, hi)))
        local = torch.tensor(np.c_[res["Y"], res["T"]] if hi > lo else np.zeros((0, spec.K + 1)))
        got = shard.gather_ranges(dist, local, ranges).numpy()
        ref = O.solve_batch(mech, batch, indices=list(range(5)))
        assert got.shape == (5, spec.K + 1)
        assert np.array_equal(got, np.c_[ref["Y"], ref["T"]])   # the same oracle on the same reactors
    finally:
        dist.destroy_process_group()


def test_caller_batch_split_and_gathered():
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_split_main, args=(2, _free_port()), nprocs=2, join=True)


def test_split_ranges_balance_and_edges():
    from paper_2005_11468_gb300 import shard
    rng = np.random.Generator(np.random.PCG64(3))
    for world in (1, 2, 3, 8):
        for B in (0, 1, 5, 64, 1000):
            c = rng.uniform(0.0, 10.0, B)
            r = shard.split_ranges(c, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == B
            assert all(a[1] == b[0] for a, b in zip(r, r[1:])) and all(lo <= hi for lo, hi in r)
            if B:
                share = [c[lo:hi].sum() for lo, hi in r]
                assert max(share) <= c.sum() / world + c.max() + 1e-9
    # the uneven mix: 50/35/15 % of K = 10/53/200 reactors, weighted by mechanism cost; the
    # K = 200 block at the end gets ranks of its own
    K = np.r_[[10] * 50, [53] * 35, [200] * 15]
    I = np.where(K == 10, 30, np.where(K == 53, 325, 1500))
    w = np.array([shard.reactor_cost(k, i) for k, i in zip(K, I)])
    assert shard.reactor_cost(200, 1500) > shard.reactor_cost(53, 325) > shard.reactor_cost(10, 30)
    r = shard.split_ranges(w, 4)
    assert r[0][1] > 85            # ranks 1-3 share the 15 costly reactors
    assert shard.split_ranges(np.zeros(8), 4) == [(0, 2), (2, 4), (4, 6), (6, 8)]
    with pytest.raises(ValueError):
        shard.split_ranges([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        shard.split_ranges([1.0], 0)
