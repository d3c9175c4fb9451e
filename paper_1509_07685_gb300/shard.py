"""Splitting one fit's histograms over ranks (one GPU per rank).

The cost of Section 4.1 is a sum over histograms, so a fit whose histograms do
not fit one device -- or that should finish sooner -- can be split by histogram:
each rank evaluates the cost and gradient of its own histograms with the full
parameter vector, and one exchange of (1 + P) doubles per evaluation adds the
ranks' results.  The sum runs in rank order on every rank (an all-gather, not a
reduction whose order the library chooses), so every rank sees the same
bit-identical total.  Independent fits need no exchange at all: those are
spread over ranks as whole fits (see bench.py).
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np


def partition_histograms(bins_per_hist: Sequence[int], world: int) -> List[List[int]]:
    """Histogram indices per rank, balanced by bins in the fit (largest first, each to
    the least loaded rank; ties to the lowest rank).  Every rank gets a list (maybe empty)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(bins_per_hist)), key=lambda h: (-int(bins_per_hist[h]), h))
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for h in order:
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].append(h)
        load[r] += int(bins_per_hist[h])
    return [sorted(p) for p in parts]


def sub_problem(problem, hists: Sequence[int]):
    """The same fit restricted to some histograms: same parameters, same map rows."""
    import dataclasses
    idx = np.asarray(list(hists), dtype=np.int64)
    return dataclasses.replace(problem, counts=np.ascontiguousarray(problem.counts[idx]),
                               t0=np.asarray(problem.t0)[idx], map=np.ascontiguousarray(problem.map[idx]))


def combine(rank_results: Sequence[np.ndarray]) -> np.ndarray:
    """(1 + P) vectors of all ranks summed in rank order."""
    out = np.zeros_like(np.asarray(rank_results[0], dtype=np.float64))
    for r in rank_results:
        out = out + np.asarray(r, dtype=np.float64)
    return out


def bins_in_fit(problem) -> List[int]:
    """Bins of each histogram inside the fit range: those with lo <= (n - t0) dt <= hi."""
    dt = problem.bin_width_ns / 1000.0
    lo, hi = problem.fit_range_us
    n = np.arange(problem.B, dtype=np.float64)
    out = []
    for h in range(problem.H):
        t = (n - float(problem.t0[h])) * dt
        out.append(int(np.count_nonzero((t >= lo) & (t <= hi))))
    return out


def distributed_eval(problem, x, rank: int, world: int, evaluate: Callable, group=None) -> np.ndarray:
    """Cost and gradient of the whole fit on every rank.

    Histograms go to ranks balanced by their bins in the fit.  ``evaluate(sub_problem, x)``
    returns this rank's (1 + P) vector (value, gradient); the vectors are all-gathered --
    on the current CUDA device for an NCCL group, on the host otherwise -- and summed in
    rank order.  A rank without histograms contributes zeros."""
    import torch
    import torch.distributed as dist
    parts = partition_histograms(bins_in_fit(problem), world)
    P = int(problem.nparams)
    mine = parts[rank]
    local = np.zeros(1 + P) if not mine else np.asarray(evaluate(sub_problem(problem, mine), x), np.float64)
    device = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(local, dtype=torch.float64, device=device)
    gathered = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(gathered, t, group=group)
    return combine([g.cpu().numpy() for g in gathered])
