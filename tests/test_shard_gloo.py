"""Multi-rank host logic on CPU (gloo, world size 2).

* One fit split by histograms over two ranks, each evaluated by the oracle, summed in
  rank order through all_gather, equals the single-rank cost and gradient.
* The benchmark's multi-rank bookkeeping: ranks draw different seeded fits, and the
  job's throughput is the units of all ranks over the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import musr_inputs as mi


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1509_07685_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = mi.cfg2(nhist=5, nbins=2000, bin_width_ns=6.0, seed=51)
    x = mi.start_point(p, 2)

    def evaluate(sub, xx):
        v, g, _, _ = oracle.cost(sub, xx, 1)
        return np.concatenate([[v], g])

    tot = shard.distributed_eval(p, x, rank, world, evaluate)
    # bench bookkeeping: per-rank units and the max-over-ranks time
    t_local = torch.tensor([0.5 + rank], dtype=torch.float64)
    dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    q.put((rank, tot, float(t_local.item())))
    dist.destroy_process_group()


def test_histogram_split_over_two_gloo_ranks_matches_single_rank():
    import oracle
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = mi.cfg2(nhist=5, nbins=2000, bin_width_ns=6.0, seed=51)
    x = mi.start_point(p, 2)
    v, g, gs, _ = oracle.cost(p, x, 1)
    tots = {r: t for r, t, _ in out}
    assert np.array_equal(tots[0], tots[1])  # every rank sees the same bits
    assert abs(tots[0][0] - v) <= 1e-12 * abs(v)
    assert np.all(np.abs(tots[0][1:] - g) <= 1e-12 * gs)
    assert all(tmax == 1.5 for _, _, tmax in out)


def test_partition_follows_the_bins_in_the_fit():
    """A histogram whose fit window holds few bins counts for those bins only."""
    import dataclasses
    from paper_1509_07685_gb300 import shard
    p = mi.cfg2(nhist=4, nbins=1000, bin_width_ns=10.0, seed=52)
    q = dataclasses.replace(p, t0=np.array([0.0, 0.0, 0.0, 900.0]))  # the last starts 900 bins late
    bins = shard.bins_in_fit(q)
    assert bins[:3] == [bins[0]] * 3 and bins[3] < bins[0] // 5
    parts = shard.partition_histograms(bins, 2)
    loads = sorted(sum(bins[h] for h in part) for part in parts)
    assert loads[1] - loads[0] <= max(bins)


def test_partition_is_balanced_and_complete():
    from paper_1509_07685_gb300 import shard
    bins = [100, 90, 80, 10, 10, 10, 5]
    parts = shard.partition_histograms(bins, 3)
    assert sorted(h for p in parts for h in p) == list(range(len(bins)))
    loads = [sum(bins[h] for h in p) for p in parts]
    assert max(loads) - min(loads) <= max(bins)
    assert shard.partition_histograms([5], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.partition_histograms([1], 0)
