#!/usr/bin/env python
"""Benchmark of the muSR fused value+gradient cost (arXiv 1509.07685, Section 4).

Workload of the contract line (one GPU): the large single fit -- 64 histograms x 2^20
bins (12.8 us at 12.2 ps per bin), FP32 counts from the seeded event-level Monte Carlo
(256 MiB, N0 = 2 counts per bin: the maximum-likelihood regime), two precession terms
plus a static Gaussian Kubo-Toyabe term, 197 parameters -- evaluated with the fused
value+analytic-gradient kernel in the FP32/FP64-split precision.  One step is one launch
that evaluates a batch of 64 parameter vectors (the trial points a fitter or a
multi-start scan hands over at once): params in, 64 x (1 + 197) doubles out.  The counts
(256 MiB) are larger than the L2; the L2 is also flushed (a 512 MiB write) between
timed steps.

Printed JSON line (rank 0): value = (histogram, bin) pairs x vectors per second of
device time (Gbins/s), measured with CUDA events on the launching stream; e2e = the same
through the C ABI with host buffers (params H2D and results D2H inside the timed
region); roofline of the fused kernel against the SM instruction-issue rate; the plain
FP64 path on the same workload; the global TF fit (8 x 65536 bins) as a second workload;
BFGS fits/s of both precisions; the serving loop (SPLIT and FP64); the oracle timed on
the host cores.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
Multi-GPU (torchrun): each rank evaluates its own independent fits (weak scaling, no
collective on the data path); timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NVEC = 64
LOAD_S = 1.5  # seconds of untimed back-to-back steps under the clock sampler before the timed ones
# Roofline of the fused SPLIT kernel.  It is bound by instruction issue (one warp
# instruction per SM sub-partition per clock: 152 SMs x 4 x 32 lanes x clock), not by HBM
# (the counts are read once per launch, 4 bytes per (histogram, bin) against ~40 lane
# operations).  Algorithmic lane operations per (histogram, bin) of the basis form,
# value+gradient, with 8 histograms of a chunk sharing each bin's time-only work:
#   per (histogram, bin): 1 shared-memory load, 3 FMA for N (M = 3 basis functions),
#     cost (-2lnL: reciprocal, residual, u, degree-6 polynomial and its two products 8, log
#     branch 4, 5 compares and selects = 20; chi^2: max, reciprocal, residual, u, value = 5),
#     1 value add,
#     7 gradient accumulations (G_m 3, W 1, V_m 3);
#   per bin / 8: time 2, E 2, per cosine term 17 (exponent 4, phase 9, sin and cos 2,
#     cosine and sine parts 2), basis sums (one per term merged into a basis function),
#     value compensation 2, shared channels (3 + 7 per cosine term + 4 per other term);
#     the Kubo-Toyabe term: exponent 4, KT factor 12 (t^2, its exponential 2, u, the
#     derivative factor 4, the factor itself 4).
# Two cosine terms (the global TF fit, merged shape M = 3): 32 + 59/8 = 39 (-2lnL), 24 (chi^2).
# Two cosine terms + Kubo-Toyabe (the large single fit): 32 + 80/8 = 42 (-2lnL), 27 (chi^2).
ALGO_INST = {"cfg5": {0: 27.0, 1: 42.0}, "cfg2": {0: 24.0, 1: 39.0}}
LANES_PER_SMSP, SMSP_PER_SM = 32, 4
# DRAM bytes of one launch of the timed kernel from an ncu capture of the workload
# (dram__bytes_read.sum + dram__bytes_write.sum, one -2lnL value+grad launch of 64 vectors),
# valid for the kernel source and cost they were taken on (None: not captured for it).
TRAFFIC = {
    "cfg5": {"kernel_sha256": "d960d5283de95a209a39d8d66265e9f0bc80fee96da6b9abeaa94caebdebfc76",
             "mode": 1, "bytes": 12062285808},
    "cfg2": {"kernel_sha256": "879a6dcc0875abf094e81477de516b460f85ebc596798c2d0855cec008222c43",
             "mode": 1, "bytes": 2231808},
}


def _kernel_sha():
    import hashlib
    src = os.path.join(ROOT, "paper_1509_07685_gb300", "csrc", "musr_kernels.cuh")
    try:
        return hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None


def _traffic(name, mode):
    """Per-launch DRAM bytes of the timed kernel (ncu), or None when the kernel source or
    the cost has changed since the capture."""
    t = TRAFFIC[name]
    return t["bytes"] if t["kernel_sha256"] == _kernel_sha() and t["mode"] == mode else None


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", type=int, default=1, help="0 chi^2, 1 -2lnL")
    ap.add_argument("--no-fits", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000,
                    help="fit requests of the serving measurement (0: skip)")
    ap.add_argument("--poisson-only", action="store_true",
                    help="run only the particle-mesh Poisson leg and print its JSON")
    ap.add_argument("--poisson-meshes", default="64x64x32,128x128x64,256x256x128,512x512x256",
                    help="comma-separated mx x my x mz meshes of the Poisson leg")
    ap.add_argument("--config-sweep", action="store_true",
                    help="instead of the contract line: SPLIT and FP64 Gbins/s of every config at 1, 8 "
                         "and 64 parameter vectors, both costs, with the oracle on one host thread")
    ap.add_argument("--sweep-configs", default="cfg1,cfg2,cfg3,cfg5,paper_tf16",
                    help="configs of --config-sweep")
    ap.add_argument("--sweep-vectors", default="1,8,64", help="parameter vectors per launch of --config-sweep")
    ap.add_argument("--sweep-modes", default="0,1", help="costs of --config-sweep (0 chi^2, 1 -2lnL)")
    ap.add_argument("--sweep-split-only", action="store_true",
                    help="--config-sweep: the SPLIT launches only (no FP64 path, cfg1 scan or oracle)")
    ap.add_argument("--precision-report", action="store_true",
                    help="instead of timing: the SPLIT path's error against FP64 for every config "
                         "(cost value, gradient, fitted parameters in units of sigma)")
    return ap.parse_args()


WORKLOADS = {
    "cfg5": "large single fit {H}x{B} FP32 counts (256 MiB), two TF terms + Kubo-Toyabe, {P} params, "
            "fused value+grad, {V} param vectors per step",
    "cfg2": "global TF fit {H}x{B} FP32 counts, two TF terms, {P} params, fused value+grad, "
            "{V} param vectors per step",
}


def _problem(name: str, rank: int = 0):
    """The seeded workload (a rank draws its own histograms) and its 64 parameter vectors."""
    import musr_inputs as mi
    if name == "cfg5":
        p = mi.cfg5(seed=5 + 1000 * rank)
    else:
        p = mi.cfg2(seed=2 + 1000 * rank)
    X = mi.jitter(p.truth, NVEC, seed=1 + rank, lo=0.9, hi=1.1)
    return p, X


def _workload(rank: int):
    return _problem("cfg5", rank)


def _workload_desc(p, mode, name="cfg5"):
    return {"workload": WORKLOADS[name].format(H=p.H, B=p.B, P=p.nparams, V=NVEC),
            "mode": "chi2" if mode == 0 else "mle", "nhist": p.H, "nbins": p.B,
            "params": p.nparams, "vectors_per_step": NVEC,
            "l2": "counts larger than L2; flushed between steps (512 MiB write)"}


# ---------------------------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(ROOT, ".clocks", f"clocks_bench_{os.getpid()}.csv")  # git-ignored

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------------------------

# The reference arm's step: value+grad of REF_VECTORS of the 64 vectors over all 64
# histograms, split over the host cores by (vector, group of REF_GROUP histograms); the cost
# and its gradient are sums over histograms, so the groups' results add up to the whole.
REF_VECTORS = 4
REF_GROUP = 16


def run_reference(args, rank, world):
    if rank != 0:
        return
    import multiprocessing as mp

    p, X = _workload(0)
    groups = [list(range(g, min(g + REF_GROUP, p.H))) for g in range(0, p.H, REF_GROUP)]
    tasks = [(k, g, args.mode) for k in range(REF_VECTORS) for g in range(len(groups))]
    bins_per_step = _bins_in_fit(p) * REF_VECTORS
    ncores = os.cpu_count() or 1
    with _SharedCounts(p) as shm:
        with mp.get_context("spawn").Pool(ncores, initializer=_pool_init,
                                          initargs=(shm.spec(), p, X, groups)) as pool:
            for w in range(max(args.warmup, 1)):
                pool.map(_oracle_task, tasks, chunksize=1)
            t = time.perf_counter()
            for s_ in range(args.steps):
                pool.map(_oracle_task, tasks, chunksize=1)
            dt = (time.perf_counter() - t) / max(args.steps, 1)
    val = bins_per_step / dt / 1e9
    sample = (f"each step: value+grad of {REF_VECTORS} of the {NVEC} parameter vectors over all {p.H} "
              f"histograms ({bins_per_step} (histogram, bin) pairs), {len(tasks)} tasks (vector x group of "
              f"{REF_GROUP} histograms) over {ncores} processes")
    line = {"metric": "value+grad Gbins/s", "value": val, "unit": "Gbins/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": _workload_desc(p, args.mode),
            "cpu_baseline": {"value": val, "unit": "Gbins/s", "cores": ncores, "kind": "oracle",
                             "cpu_model": _cpu_model()["model"], "sample": sample},
            "e2e": {"value": val, "unit": "Gbins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class _SharedCounts:
    """The workload's counts in a shared-memory block, so that spawned oracle processes map
    them instead of each receiving a pickled copy."""

    def __init__(self, p):
        from multiprocessing import shared_memory
        c = np.ascontiguousarray(p.counts)
        self.shape, self.dtype = c.shape, c.dtype.str
        self.shm = shared_memory.SharedMemory(create=True, size=max(c.nbytes, 1))
        np.ndarray(c.shape, c.dtype, buffer=self.shm.buf)[...] = c

    def spec(self):
        return (self.shm.name, self.shape, self.dtype)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.shm.close()
        self.shm.unlink()


_POOL_WORK = {}


def _pool_init(spec, p, X, groups):
    """Spawned oracle worker: map the shared counts, keep the vectors, load the library."""
    import dataclasses
    from multiprocessing import shared_memory
    import oracle
    name, shape, dtype = spec
    shm = shared_memory.SharedMemory(name=name)
    counts = np.ndarray(shape, np.dtype(dtype), buffer=shm.buf)
    _POOL_WORK["shm"] = shm
    _POOL_WORK["X"] = X
    _POOL_WORK["sub"] = [dataclasses.replace(p, counts=counts[g], t0=p.t0[g], map=p.map[g]) for g in groups]
    oracle.build()


def _oracle_task(args):
    """One oracle value+grad evaluation of vector k on histogram group g (in a pool worker)."""
    import oracle
    k, g, mode = args
    oracle.cost(_POOL_WORK["sub"][g], _POOL_WORK["X"][k % len(_POOL_WORK["X"])], mode)


def _bins_in_fit(p):
    dt = p.bin_width_ns / 1000.0
    lo, hi = p.fit_range_us
    n = np.arange(p.B)
    tot = 0
    for h in range(p.H):
        t = (n - p.t0[h]) * dt
        tot += int(np.count_nonzero((t >= lo) & (t <= hi)))
    return tot


def _oracle_worker(args):
    """One process of the all-cores oracle timing: evaluate vectors until the deadline."""
    p, X, mode, seconds = args
    import oracle
    oracle.cost(p, X[0], mode)  # load the library before the clock starts
    n = 0
    t = time.perf_counter()
    while time.perf_counter() - t < seconds:
        oracle.cost(p, X[n % len(X)], mode)
        n += 1
    return n, time.perf_counter() - t


def _oracle_all_cores(p, X, mode, seconds):
    """(evaluations, seconds, processes): the oracle as it stands, one process per host core
    (spawned, so no process inherits a CUDA context), each on its own vectors."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(ncores) as pool:
        res = pool.map(_oracle_worker, [(p, X[k::ncores] if len(X) > k else X, mode, seconds)
                                        for k in range(ncores)])
    return sum(n for n, _ in res), max(t for _, t in res), ncores


def cpu_baseline(p, X, mode, budget_s=6.0, nhist=4):
    """The oracle as it stands on a bounded sample of the same workload -- its first `nhist`
    histograms, value+grad of the 64 vectors in turn -- on one thread, then one process per
    host core (the figure reported)."""
    import dataclasses
    import oracle
    q = dataclasses.replace(p, counts=np.ascontiguousarray(p.counts[:nhist]), t0=p.t0[:nhist], map=p.map[:nhist])
    bins = _bins_in_fit(q)
    oracle.cost(q, X[0], mode)
    n = 0
    t = time.perf_counter()
    while True:
        oracle.cost(q, X[n % len(X)], mode)
        n += 1
        if time.perf_counter() - t > budget_s or n >= 200:
            break
    single = bins * n / (time.perf_counter() - t) / 1e9
    n_all, t_all, ncores = _oracle_all_cores(q, X, mode, budget_s)
    return {"value": bins * n_all / t_all / 1e9, "unit": "Gbins/s", "cores": ncores, "kind": "oracle",
            "single_thread_value": single, "cpu_model": _cpu_model()["model"],
            "sample": f"value+grad evaluations of the workload's first {nhist} histograms ({bins} bins each) for "
                      f"{budget_s:.0f} s: {n} on one thread, {n_all} over {ncores} processes"}


# ---------------------------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------------------------

def _timed(B, ctx, d_x, nvec, mode, prec, d_out, flush, stream, steps, warmup, world=1):
    """CUDA-event seconds of `steps` launches of nvec evaluations (L2 flushed before each)."""
    import torch

    def step():
        B.musr_eval_device(ctx.ctx, d_x.data_ptr(), nvec, mode, prec, True, d_out.data_ptr())

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s_ in range(steps):
        flush.zero_()
        ev[s_][0].record(stream)
        step()
        ev[s_][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    return [a_.elapsed_time(b_) * 1e-3 for a_, b_ in ev]


def _roofline(name, p, bins, mode, t_kernel, peaks, nsm):
    """Roofline of one launch of the fused kernel: algorithmic lane operations per (histogram,
    bin) x pairs per launch / CUDA-event time, against the SM instruction-issue rate."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_inst = nsm * SMSP_PER_SM * LANES_PER_SMSP * sm_max * 1e6
    ach_inst = ALGO_INST[name][mode] * bins * NVEC / t_kernel
    algo_bytes = 4 * p.H * p.B + 8 * NVEC * (p.nparams + 1 + p.nparams)  # counts once, params in, value+grad out
    shape = "two TF terms + KT merged (M = 3)" if name == "cfg5" else "two TF terms merged (M = 3)"
    return {"bound": "alu", "achieved": ach_inst / 1e12, "peak": peak_inst / 1e12, "unit": "Tinst/s",
            "frac": ach_inst / peak_inst, "traffic": _traffic(name, mode),
            "kernel": f"eval_kernel<SPLIT, {shape}, {'MLE' if mode else 'chi2'}, grad>",
            "measure": "lane operations of the algorithm per (histogram, bin) x (histogram, bin) pairs "
                       "per launch / CUDA-event time of the launch",
            "instructions_per_hist_bin": ALGO_INST[name][mode],
            "peak_source": f"instruction issue: {nsm} SMs x {SMSP_PER_SM} sub-partitions x "
                           f"{LANES_PER_SMSP} lanes x {sm_max:.0f} MHz (max SM clock of MEASURED_PEAKS.json)",
            "algorithmic_bytes": algo_bytes,
            "hbm_frac": algo_bytes / t_kernel / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
            "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0))}


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1509_07685_gb300 import binding as B

    B.load()
    p, X = _workload(rank)
    mode = args.mode
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = B.Context(p, device=local_rank, cuda_stream=stream.cuda_stream)
    bins = ctx.bins_in_fit()
    P = p.nparams
    d_x = torch.tensor(X, dtype=torch.float64, device="cuda")
    d_out = torch.empty((NVEC, 1 + P), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    launches0 = B.musr_launches_per_eval(ctx.ctx)

    # Main measurement (SPLIT).  The sampler also covers LOAD_S seconds of the same steps
    # run back to back just before the timed ones (untimed): the clocks they start from.
    with ClockSampler(local_rank) as clk:
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < LOAD_S:
            for _ in range(10):
                flush.zero_()
                B.musr_eval_device(ctx.ctx, d_x.data_ptr(), NVEC, mode, B.MUSR_SPLIT, True, d_out.data_ptr())
            torch.cuda.synchronize()
        t_wall = time.perf_counter()
        times = _timed(B, ctx, d_x, NVEC, mode, B.MUSR_SPLIT, d_out, flush, stream, args.steps,
                       max(args.warmup, 3), world)
        t_wall = time.perf_counter() - t_wall
    mean_t = float(np.mean(times))
    t_kernel = mean_t
    if world > 1:
        tt = torch.tensor([mean_t], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        mean_t = float(tt.item())
    value = bins * NVEC * world / mean_t / 1e9
    out_split = d_out.cpu().numpy().copy()

    # Plain FP64 path on the same workload: the first 8 vectors (it is ~300x slower).
    n64 = 8
    d_o64 = torch.empty((n64, 1 + P), dtype=torch.float64, device="cuda")
    t64 = _timed(B, ctx, d_x[:n64].contiguous(), n64, mode, B.MUSR_FP64, d_o64, flush, stream, 2, 1)
    fp64_gbins = bins * n64 / float(np.mean(t64)) / 1e9
    out_fp64 = d_o64.cpu().numpy()
    rel_err = float(np.max(np.abs(out_split[:n64, 0] - out_fp64[:, 0]) / np.abs(out_fp64[:, 0])))

    # End to end through the C ABI with host buffers.
    Xh = np.ascontiguousarray(X)
    for _ in range(2):
        ctx.eval_batch(Xh, mode, B.MUSR_SPLIT)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        ctx.eval_batch(Xh, mode, B.MUSR_SPLIT)
    e2e_t = (time.perf_counter() - t) / args.steps
    if world > 1:  # whole job: every rank's evaluations over the slowest rank's time
        tt = torch.tensor([e2e_t], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_t = float(tt.item())
    e2e = {"value": bins * NVEC * world / e2e_t / 1e9, "unit": "Gbins/s", "h2d_bytes_per_step": int(Xh.nbytes),
           "d2h_bytes_per_step": int(NVEC * (1 + P) * 8),
           "path": "musr_eval_batch (host params in, host value+grad out, synchronous)"}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    clocks = clk.summary() | {"window": f"{LOAD_S} s of back-to-back steps, then the timed steps"}
    nsm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    roofline = _roofline("cfg5", p, bins, mode, t_kernel, peaks, nsm)

    # The second workload (the global TF fit, 8 x 65536 bins): same measurement.
    q, Xq = _problem("cfg2", rank)
    with B.Context(q, device=local_rank, cuda_stream=stream.cuda_stream) as cq:
        bq = cq.bins_in_fit()
        dq = torch.tensor(Xq, dtype=torch.float64, device="cuda")
        doq = torch.empty((NVEC, 1 + q.nparams), dtype=torch.float64, device="cuda")
        tq = float(np.mean(_timed(B, cq, dq, NVEC, mode, B.MUSR_SPLIT, doq, flush, stream, args.steps,
                                  max(args.warmup, 3))))
        tq64 = float(np.mean(_timed(B, cq, dq, NVEC, mode, B.MUSR_FP64, doq, flush, stream, 2, 1)))
    second = {"config": _workload_desc(q, mode, "cfg2"), "value": bq * NVEC / tq / 1e9, "unit": "Gbins/s",
              "ms_per_step": tq * 1e3, "roofline": _roofline("cfg2", q, bq, mode, tq, peaks, nsm),
              "fp64_path": {"value": bq * NVEC / tq64 / 1e9, "unit": "Gbins/s", "split_speedup": tq64 / tq}}

    fits = asym = poisson = lists = dkt = None
    if not args.no_fits and rank == 0:
        fits = _fits(B, mode)
        asym = _asymmetry(B, flush, stream)
        lists = _term_lists(B, flush, stream)
        dkt = _dynamic_kt(B, flush, stream)
        poisson = _poisson(B, peaks, cpu=not args.no_cpu, meshes=_meshes(args))
    serving = None
    if args.serving_requests > 0 and rank == 0:
        serving = _serving(B, args.serving_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(p, X, mode)

    if rank == 0:
        line = {"metric": "value+grad Gbins/s", "value": value, "unit": "Gbins/s", "n_gpus": world,
                "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": mean_t * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64-split",
                "data": "synthetic (seeded event-level Monte Carlo muSR histograms)",
                "config": _workload_desc(p, mode),
                "e2e": e2e, "roofline": roofline, "clocks": clocks,
                "gpu_launches": args.steps * launches0, "wall_s_timed_region": t_wall,
                "parallelism": f"dp{world} (independent fits per rank)",
                "fp64_path": {"value": fp64_gbins, "unit": "Gbins/s", "vectors": n64,
                              "split_speedup": value / world / fp64_gbins,
                              "max_rel_value_diff_split_vs_fp64": rel_err},
                "global_tf_fit": second,
                "fits": fits, "asymmetry": asym, "term_lists": lists, "dynamic_kt": dkt, "poisson": poisson, "serving": serving,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _asymmetry(B, flush, stream, steps=10):
    """Asymmetry-form fit of the paper's 16 detectors as 8 forward / backward pairs (81920
    bins each): value+grad of the weighted chi^2 for 64 parameter vectors per launch,
    SPLIT and FP64 (CUDA events on the launching stream, L2 flushed between launches)."""
    import torch
    import musr_inputs as mi
    p = mi.asym_tf(npairs=8, nbins=81920, bin_width_ns=12800.0 / 81920, seed=31, n0=60.0)
    X = mi.jitter(p.truth, NVEC, seed=5, lo=0.97, hi=1.03)
    out = {"workload": "8 forward/backward pairs x 81920 bins (the 16 detectors of the paper's benchmark), "
                       "chi^2 of the asymmetry, fused value+grad, 64 parameter vectors per launch",
           "params": int(p.nparams)}
    with torch.cuda.stream(stream):
        with B.Context(p, cuda_stream=stream.cuda_stream) as ctx:
            bins = ctx.bins_in_fit()
            dx = torch.tensor(X, dtype=torch.float64, device="cuda")
            do = torch.empty((NVEC, 1 + p.nparams), dtype=torch.float64, device="cuda")
            res = {}
            for prec, name in ((B.MUSR_SPLIT, "split"), (B.MUSR_FP64, "fp64")):
                for _ in range(3):
                    B.musr_eval_device(ctx.ctx, dx.data_ptr(), NVEC, 0, prec, True, do.data_ptr())
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps if prec == B.MUSR_SPLIT else 3)]
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    B.musr_eval_device(ctx.ctx, dx.data_ptr(), NVEC, 0, prec, True, do.data_ptr())
                    b.record(stream)
                torch.cuda.synchronize()
                t = float(np.mean([a.elapsed_time(b) * 1e-3 for a, b in ev]))
                out[f"{name}_gbins_per_s"] = bins * NVEC / t / 1e9
                res[name] = do.cpu().numpy().copy()
    out["split_speedup"] = out["split_gbins_per_s"] / out["fp64_gbins_per_s"]
    out["max_rel_value_diff_split_vs_fp64"] = float(np.max(np.abs(res["split"][:, 0] - res["fp64"][:, 0]) /
                                                           np.abs(res["fp64"][:, 0])))
    return out


def _term_lists(B, flush, stream, steps=10):
    """Theories without a basis form on the paper's benchmark workload (16 x 81920 bins): its
    model with the cosine replaced by a Bessel precession, and with the Gaussian replaced by a
    stretched exponential (exponent shared); SPLIT (the term list per bin in FP32) and FP64,
    chi^2 value+grad of 64 parameter vectors per launch (CUDA events, L2 flushed)."""
    import dataclasses
    import torch
    import musr_inputs as mi
    base = mi.paper_tf16(seed=33, n0=60.0)
    P = base.nparams
    theories = {
        "bessel": dataclasses.replace(base, terms=[[("AMP", (2,)), ("GAUSS", (3,)), ("BESSEL", (4, 5))]]),
        "stretched_exponential": dataclasses.replace(
            base, terms=[[("AMP", (2,)), ("STREXP", (3, 6)), ("TFCOS", (4, 5))]],
            map=np.hstack([base.map, np.full((base.H, 1), P, np.int32)]), nparams=P + 1,
            truth=np.append(base.truth, 1.5), names=base.names + ["beta"]),
    }
    out = {"workload": "paper benchmark (16 x 81920 bins) with a Bessel precession or a stretched exponential, "
                       "chi^2, fused value+grad, 64 parameter vectors per launch"}
    for name, p in theories.items():
        X = mi.jitter(p.truth, NVEC, seed=8, lo=0.97, hi=1.03)
        with torch.cuda.stream(stream):
            with B.Context(p, cuda_stream=stream.cuda_stream) as ctx:
                bins = ctx.bins_in_fit()
                dx = torch.tensor(X, dtype=torch.float64, device="cuda")
                do = torch.empty((NVEC, 1 + p.nparams), dtype=torch.float64, device="cuda")
                res, rate = {}, {}
                for prec, pn in ((B.MUSR_SPLIT, "split"), (B.MUSR_FP64, "fp64")):
                    for _ in range(2):
                        B.musr_eval_device(ctx.ctx, dx.data_ptr(), NVEC, 0, prec, True, do.data_ptr())
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(steps if prec == B.MUSR_SPLIT else 2)]
                    for a, b in ev:
                        flush.zero_()
                        a.record(stream)
                        B.musr_eval_device(ctx.ctx, dx.data_ptr(), NVEC, 0, prec, True, do.data_ptr())
                        b.record(stream)
                    torch.cuda.synchronize()
                    rate[pn] = bins * NVEC / float(np.mean([a.elapsed_time(b) * 1e-3 for a, b in ev])) / 1e9
                    res[pn] = do.cpu().numpy().copy()
        out[name] = {"split_gbins_per_s": rate["split"], "fp64_gbins_per_s": rate["fp64"],
                     "split_speedup": rate["split"] / rate["fp64"],
                     "max_rel_value_diff_split_vs_fp64": float(np.max(np.abs(res["split"][:, 0] - res["fp64"][:, 0]) /
                                                                      np.abs(res["fp64"][:, 0])))}
    return out


def _dynamic_kt(B, flush, stream, steps=10):
    """Zero-field fit in fluctuating fields at the paper benchmark's size (16 x 81920 bins,
    12.8 us): A0 DKT(Delta, nu) per detector, -2lnL value+grad of 64 parameter vectors per
    launch, SPLIT (FP32 tables, term-list kernel) and FP64; each launch first solves one
    table per vector (CUDA events on the launching stream, L2 flushed)."""
    import torch
    import musr_inputs as mi
    p = mi.dkt_zf(nhist=16, nbins=81920, bin_width_ns=12800.0 / 81920, seed=35, n0=60.0)
    X = mi.jitter(p.truth, NVEC, seed=9, lo=0.97, hi=1.03)
    out = {"workload": "zero-field fit, 16 x 81920 bins, A0 DKT(Delta, nu), -2lnL, fused value+grad, "
                       "64 parameter vectors per launch (one renewal-equation table per vector)",
           "params": int(p.nparams)}
    with torch.cuda.stream(stream):
        with B.Context(p, cuda_stream=stream.cuda_stream) as ctx:
            bins = ctx.bins_in_fit()
            dx = torch.tensor(X, dtype=torch.float64, device="cuda")
            do = torch.empty((NVEC, 1 + p.nparams), dtype=torch.float64, device="cuda")
            res = {}
            for prec, pn in ((B.MUSR_SPLIT, "split"), (B.MUSR_FP64, "fp64")):
                for _ in range(3):
                    B.musr_eval_device(ctx.ctx, dx.data_ptr(), NVEC, 1, prec, True, do.data_ptr())
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(steps if prec == B.MUSR_SPLIT else 3)]
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    B.musr_eval_device(ctx.ctx, dx.data_ptr(), NVEC, 1, prec, True, do.data_ptr())
                    b.record(stream)
                torch.cuda.synchronize()
                t = float(np.mean([a.elapsed_time(b) * 1e-3 for a, b in ev]))
                out[f"{pn}_gbins_per_s"] = bins * NVEC / t / 1e9
                out[f"{pn}_ms_per_launch"] = t * 1e3
                res[pn] = do.cpu().numpy().copy()
            out["launches_per_eval"] = int(B.musr_launches_per_eval(ctx.ctx))
    out["split_speedup"] = out["split_gbins_per_s"] / out["fp64_gbins_per_s"]
    out["max_rel_value_diff_split_vs_fp64"] = float(np.max(np.abs(res["split"][:, 0] - res["fp64"][:, 0]) /
                                                           np.abs(res["fp64"][:, 0])))
    return out


# Algorithmic bytes of one particle-mesh Poisson solve per mesh point (M points, doubled mesh
# N = 8 M with N/2 complex points, r bytes per real of the transforms, FP64 density in and
# potential out): pad (read 8 M, write r M: the zeros stay), forward FFT (read r N, write r N),
# Hadamard product (read r N + r N / 2, write r N), inverse FFT (read r N, write r N),
# extraction (read r M, write 8 M), each array touched once: (16 + 54 r) M, i.e. 448 bytes per
# mesh point with FP64 transforms and 232 with FP32 ones.
POISSON_BYTES_PER_POINT = {0: 448, 1: 232}
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal FP64 (not measured on this machine)


def _poisson(B, peaks, cpu=True, meshes=((64, 64, 32), (128, 128, 64), (256, 256, 128), (512, 512, 256))):
    """The particle-mesh Poisson solve of Section 3 on the meshes of the paper's benchmark
    table, FP64 and FP32 transforms: device time per solve (CUDA events on the solver's
    stream, median of 7), end to end through the host-array call, achieved GB/s of the
    algorithmic bytes (and, for FP64, the transforms' FLOP rate, 2 x 2.5 N log2 N, against the
    nominal FP64 peak); the oracle's direct sum timed on sampled points of the smallest mesh."""
    import torch
    import oracle
    out = {"workload": "open-boundary Poisson solve (Hockney, doubled mesh) of a Gaussian bunch",
           "bytes_per_mesh_point": {"fp64": 448, "fp32_transforms": 232}, "meshes": []}
    stream = torch.cuda.Stream()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    for shape in meshes:
        shape = tuple(shape)
        M = int(np.prod(shape))
        N = 8 * M
        x, y, z = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij", sparse=True)
        rho = np.exp(-0.5 * (((x - 0.45 * shape[0]) / (0.1 * shape[0])) ** 2 +
                             ((y - 0.5 * shape[1]) / (0.1 * shape[1])) ** 2 +
                             ((z - 0.55 * shape[2]) / (0.1 * shape[2])) ** 2))
        rho = np.ascontiguousarray(rho)
        h = (1.0 / shape[0], 1.0 / shape[1], 2.0 / shape[2])
        entry = {"mesh": list(shape), "e2e_h2d_d2h_bytes": 16 * M}
        phis = {}
        for prec, name in ((B.MUSR_SPLIT, "fp32_transforms"), (B.MUSR_FP64, "fp64")):
            with B.Poisson(shape, h, prec, cuda_stream=stream.cuda_stream) as ps:
                d_rho = torch.tensor(rho, device="cuda")
                d_phi = torch.empty_like(d_rho)
                for _ in range(2):
                    ps.solve_device(d_rho.data_ptr(), d_phi.data_ptr())
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(7)]
                for a, b in ev:
                    a.record(stream)
                    ps.solve_device(d_rho.data_ptr(), d_phi.data_ptr())
                    b.record(stream)
                torch.cuda.synchronize()
                t = float(np.median([a.elapsed_time(b) * 1e-3 for a, b in ev]))
                phis[name] = ps.solve(rho)
                t0 = time.perf_counter()
                for _ in range(3):
                    ps.solve(rho)
                t_e2e = (time.perf_counter() - t0) / 3
                del d_rho, d_phi
            gbs = POISSON_BYTES_PER_POINT[prec] * M / t / 1e9
            r = {"ms_per_solve": t * 1e3, "e2e_ms_per_solve": t_e2e * 1e3, "achieved_gbs": gbs, "hbm_frac": gbs / hbm}
            if prec == B.MUSR_FP64:
                tf = 2 * 2.5 * N * math.log2(N) / t / 1e12
                r |= {"fft_tflops": tf, "fp64_nominal_frac": tf / FP64_NOMINAL_TFLOPS}
            entry[name] = r
        entry["max_rel_diff_fp32_vs_fp64"] = float(np.max(np.abs(phis["fp32_transforms"] - phis["fp64"])) /
                                                   np.max(np.abs(phis["fp64"])))
        entry["fp32_speedup"] = entry["fp64"]["ms_per_solve"] / entry["fp32_transforms"]["ms_per_solve"]
        out["meshes"].append(entry)
        if cpu and shape == (64, 64, 32):
            ijk = np.stack([np.random.default_rng(6).integers(0, n, 24) for n in shape], axis=1)
            t0 = time.perf_counter()
            oracle.poisson_points(rho, h, ijk)
            per_point = (time.perf_counter() - t0) / len(ijk)
            out["cpu_baseline"] = {"kind": "oracle", "cores": 1, "mesh": list(shape),
                                   "direct_sum_s_per_solve": per_point * M,
                                   "sample": f"{len(ijk)} mesh points by direct summation, scaled to the {M} points"}
    out["peak_hbm_gbs"] = hbm
    out["fp64_nominal_tflops"] = FP64_NOMINAL_TFLOPS
    return out


def _fits(B, mode, nfits=8):
    """fits/s of both precisions on the global TF fit (8 x 65536 bins, 28 parameters): BFGS
    fits one after another through the C ABI's native fit (musr_fit: C++ BFGS driving the
    fused kernel) from the same 8 start points, SPLIT and FP64; the Python BFGS of fit.py;
    the agreement of the SPLIT fit with the FP64 fit; parameter errors."""
    try:
        from paper_1509_07685_gb300 import fit as F
    except Exception:
        return None
    import musr_inputs as mi
    p = mi.cfg2()
    out = {"workload": f"global TF fit {p.H}x{p.B}, {p.nparams} params, {'MLE' if mode else 'chi2'}, "
                       f"{nfits} fits from the same start points per precision"}
    with B.Context(p) as ctx:
        res = {}
        for prec, name in ((B.MUSR_SPLIT, "split"), (B.MUSR_FP64, "fp64")):
            B.musr_fit(ctx.ctx, mi.start_point(p, 99), mode, prec)  # warm-up: tables, buffers
            lat, nfev, xs = [], [], []
            for s_ in range(nfits):
                x0 = mi.start_point(p, 100 + s_)
                t = time.perf_counter()
                r = B.musr_fit(ctx.ctx, x0, mode, prec)
                lat.append(time.perf_counter() - t)
                nfev.append(r["nfev"])
                xs.append(r["x"])
            res[name] = xs
            out[name] = {"fits_per_s": len(lat) / sum(lat), "latency_ms_p50": 1e3 * float(np.median(lat)),
                         "latency_ms_max": 1e3 * float(np.max(lat)), "evals_per_fit": float(np.mean(nfev))}
        out["split_speedup_fits_per_s"] = out["split"]["fits_per_s"] / out["fp64"]["fits_per_s"]
        out["path"] = "musr_fit (C++ BFGS through the C ABI)"
        lat_py = []
        for s_ in range(4):
            t = time.perf_counter()
            F.fit_context(ctx, mi.start_point(p, 100 + s_), mode, B.MUSR_SPLIT)
            lat_py.append(time.perf_counter() - t)
        out["python_bfgs_split_fits_per_s"] = len(lat_py) / sum(lat_py)
        x64 = res["fp64"][0]
        t = time.perf_counter()
        sig = F.sigmas_context(ctx, x64, mode)  # central differences of FP64 gradients (2P)
        t_fd = time.perf_counter() - t
        out["max_param_dev_split_vs_fp64_sigma"] = float(max(np.max(np.abs(a_ - b_) / sig)
                                                             for a_, b_ in zip(res["split"], res["fp64"])))
        for _ in range(2):
            F.sigmas_gauss_newton(ctx, x64, mode, B.MUSR_SPLIT)
        t = time.perf_counter()
        sig_gn = F.sigmas_gauss_newton(ctx, x64, mode, B.MUSR_SPLIT)
        t_gn = time.perf_counter() - t
        t = time.perf_counter()
        sig_gn64 = F.sigmas_gauss_newton(ctx, x64, mode, B.MUSR_FP64)
        t_gn64 = time.perf_counter() - t
    out["parameter_errors"] = {"gauss_newton_split_ms": 1e3 * t_gn, "gauss_newton_fp64_ms": 1e3 * t_gn64,
                               "central_differences_fp64_ms": 1e3 * t_fd,
                               "max_rel_diff_sigma_gn_vs_fd": float(np.max(np.abs(sig_gn / sig - 1.0))),
                               "max_rel_diff_sigma_gn_split_vs_fp64": float(np.max(np.abs(sig_gn / sig_gn64 - 1.0)))}
    return out


def _saturation(B, reqs, precision, budget, window=1024):
    """Closed loop (at most `window` fits in flight): fits/s, converged count, stats."""
    with B.Server(hbm_budget_bytes=budget, max_active=1024) as srv:
        t = time.perf_counter()
        pending, statuses = [], []
        i = 0
        while i < len(reqs) or pending:
            while i < len(reqs) and len(pending) < window:
                r = reqs[i]
                pending.append(srv.submit(r.problem, r.x0, r.mode, precision))
                i += 1
            res = srv.wait(pending.pop(0))
            statuses.append(res["status"])
        wall = time.perf_counter() - t
        st = srv.stats()
    return len(reqs) / wall, wall, int(sum(s_ == 0 for s_ in statuses)), st


def _serving(B, n_requests, window=1024, seed=4, pool_size=256):
    """Serving: fits/s at saturation (closed loop, at most `window` in flight), then
    Poisson arrivals at 0.5x and 0.9x that rate with p50/p99 latency (server clock,
    submission to completion); the same saturation run for the FP64 path against SPLIT on
    the first 1000 requests; saturation at smaller HBM budgets.  Requests draw from a pool
    of 256 seeded fits (H, B log-uniform, theory from cfg1/cfg2/cfg3, truths jittered, each
    fit its own event-level Monte Carlo), each request with its own start point and cost."""
    import threading

    import musr_inputs as mi
    pool = mi.serving_pool(pool_size, seed=seed, workers=os.cpu_count() or 1)
    out = {"requests": n_requests, "pool": len(pool), "precision": "split", "hbm_budget_gib": 8, "max_active": 1024}
    reqs = mi.request_stream(pool, n_requests, 0.0, seed=seed)
    # Warm-up (untimed): one pass over the pool's fits, so that the timed runs do not include
    # the first touch of the pool's host memory and the helper threads' first copies.
    _saturation(B, mi.request_stream(pool, len(pool) + 64, 0.0, seed=seed + 99), B.MUSR_SPLIT, 2 << 30, window)
    rate, wall, conv, st = _saturation(B, reqs, B.MUSR_SPLIT, 8 << 30, window)
    out["saturation"] = {"fits_per_s": rate, "wall_s": wall, "converged": conv,
                         "gbins_per_s": st["bin_evals"] / wall / 1e9, "steps": st["steps"],
                         "launches": st["launches"], "evals": st["evals"],
                         "worker_s": {"busy": st["busy_s"], "minimizer": st["minimizer_s"],
                                      "admit": st["admit_s"], "device_wait": st["wait_s"]},
                         "configure_thread_s": {"context": st["cfg_create_s"], "upload": st["cfg_upload_s"],
                                                "plan": st["cfg_plan_s"], "buffers": st["cfg_buffers_s"]}}
    for frac in (0.5, 0.9):
        rq = mi.request_stream(pool, n_requests, frac * rate, seed=seed + 10)
        with B.Server(hbm_budget_bytes=8 << 30, max_active=1024) as srv:
            ids = [None] * len(rq)
            t0 = time.perf_counter()

            def submitter():
                for k, r in enumerate(rq):
                    delay = r.arrival_s - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                    ids[k] = srv.submit(r.problem, r.x0, r.mode, B.MUSR_SPLIT)

            th = threading.Thread(target=submitter)
            th.start()
            lat = []
            for k in range(len(rq)):
                while ids[k] is None:
                    time.sleep(0.0005)
                res = srv.wait(ids[k])
                lat.append(res["t_done"] - res["t_submit"])
            th.join()
            wall = time.perf_counter() - t0
        lat = np.array(lat)
        out[f"load_{frac}"] = {"rate_fits_per_s": frac * rate, "fits_per_s": n_requests / wall,
                               "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                               "latency_ms_p99": 1e3 * float(np.percentile(lat, 99))}
    # SPLIT against the plain FP64 path on the same 1000 requests (the FP64 path is far
    # slower per evaluation, so the whole stream would take minutes)
    sub = reqs[:min(1000, len(reqs))]
    r32, w32, c32, _ = _saturation(B, sub, B.MUSR_SPLIT, 8 << 30, window)
    r64, w64, c64, _ = _saturation(B, sub, B.MUSR_FP64, 8 << 30, window)
    out["split_vs_fp64"] = {"requests": len(sub), "split_fits_per_s": r32, "fp64_fits_per_s": r64,
                            "split_speedup": r32 / r64, "converged": [c32, c64]}
    sweep = {}
    for gib in (1, 2, 4):
        rate_b, wall_b, conv_b, st_b = _saturation(B, reqs[:min(3000, len(reqs))], B.MUSR_SPLIT, gib << 30, window)
        sweep[f"{gib}GiB"] = {"fits_per_s": rate_b, "converged": conv_b, "arena_bytes": int(st_b["arena_bytes"])}
    out["hbm_budget_sweep"] = {"requests": min(3000, len(reqs)), **sweep}
    return out


def precision_report(args):
    """Error of the FP32/FP64-split path against FP64, per configuration and mode: the cost
    value (relative), the gradient (|dg_i| / gradient scale_i, the scale from the oracle),
    and BFGS fits from the same start point (|x_split - x_fp64| / sigma_i, sigma from the
    FP64 Hessian at the FP64 optimum).  The plain FP64 GPU path is the reference for values
    and fits (it matches the oracle to 1e-12; checked here on the value)."""
    import torch
    import musr_inputs as mi
    import oracle
    from paper_1509_07685_gb300 import binding as B
    from paper_1509_07685_gb300 import fit as F
    torch.cuda.set_device(0)
    B.load()
    cfgs = {"cfg1": mi.cfg1(), "cfg2": mi.cfg2(), "cfg3": mi.cfg3(), "cfg5": mi.cfg5(), "paper_tf16": mi.paper_tf16()}
    out = {}
    for name, p in cfgs.items():
        with B.Context(p) as ctx:
            for mode in (0, 1):
                x = mi.start_point(p, 100)
                ref = oracle.cost(p, x, mode)
                v64, g64, _ = ctx.eval(x, mode, B.MUSR_FP64)
                v32, g32, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
                r64 = F.fit_context(ctx, x, mode, B.MUSR_FP64)
                r32 = F.fit_context(ctx, x, mode, B.MUSR_SPLIT)
                with np.errstate(invalid="ignore"):
                    sig = F.sigmas_context(ctx, r64["x"], mode)
                ok = np.isfinite(sig)  # sigma needs a positive-definite FP64 Hessian at the optimum
                dev = np.where(ok, np.abs(r32["x"] - r64["x"]) / np.where(ok, sig, 1.0), np.nan)
                vf64, _, _ = ctx.eval(r64["x"], mode, B.MUSR_FP64)
                vf32, _, _ = ctx.eval(r64["x"], mode, B.MUSR_SPLIT)
                out[f"{name}/{'mle' if mode else 'chi2'}"] = {
                    "fp64_value_rel_err_vs_oracle": abs(v64 - ref[0]) / abs(ref[0]),
                    "split_value_rel_err": abs(v32 - v64) / abs(v64),
                    "split_value_rel_err_at_optimum": abs(vf32 - vf64) / abs(vf64),
                    "split_grad_err_over_scale": float(np.max(np.abs(g32 - g64) / ref[2])),
                    "fit_max_dev_sigma": float(np.nanmax(dev)) if ok.any() else None,
                    "params_without_sigma": int((~ok).sum()),
                    "fit_dev_sigma_by_param": {n: float(d) for n, d in zip(p.names, dev)} if p.nparams <= 32 else None,
                    "fit_status": [int(r64["status"]), int(r32["status"])],
                    "params": p.nparams}
                print(name, mode, json.dumps(out[f"{name}/{'mle' if mode else 'chi2'}"])[:300], flush=True)
    print(json.dumps({"precision_report": out}), flush=True)


def _sweep_time(B, ctx, dx, nvec, mode, prec, grad, do, flush, stream, reps):
    """Mean CUDA-event seconds of one musr_eval_device launch (L2 flushed before each)."""
    import torch
    for _ in range(2):
        B.musr_eval_device(ctx.ctx, dx.data_ptr(), nvec, mode, prec, grad, do.data_ptr())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        B.musr_eval_device(ctx.ctx, dx.data_ptr(), nvec, mode, prec, grad, do.data_ptr())
        b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) * 1e-3 for a, b in ev]))


def config_sweep(args):
    """Throughput of every configuration: the SPLIT path at 1, 8 and 64 parameter vectors per
    launch and the plain FP64 path at 8 (value+grad, chi^2 and -2lnL), the value-only scan of
    cfg1 (1000 random vectors, FP64 and SPLIT), and the oracle on one host thread (value+grad;
    for cfg5 on its first 4 histograms, 4 x 2^20 bins).  CUDA events on the launching stream,
    L2 flushed before every launch.  One JSON line.  ``--sweep-configs``, ``--sweep-vectors``
    and ``--sweep-modes`` narrow it; ``--sweep-split-only`` keeps the SPLIT launches alone
    (per config: 2 untimed, then 10 timed launches per vector count and cost)."""
    import dataclasses
    import torch
    import musr_inputs as mi
    from paper_1509_07685_gb300 import binding as B
    full = not args.sweep_split_only
    torch.cuda.set_device(0)
    B.load()
    if full:
        import oracle
        oracle.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    make = {"cfg1": mi.cfg1, "cfg2": mi.cfg2, "cfg3": mi.cfg3, "cfg5": mi.cfg5, "paper_tf16": mi.paper_tf16}
    names = [n for n in args.sweep_configs.split(",") if n]
    vectors = [int(v) for v in args.sweep_vectors.split(",") if v]
    modes = [int(m) for m in args.sweep_modes.split(",") if m]
    out = {}
    for name in names:
        p = make[name]()
        row = {"nhist": p.H, "nbins": p.B, "params": p.nparams}
        with torch.cuda.stream(stream):
            with B.Context(p, cuda_stream=stream.cuda_stream) as ctx:
                bins = ctx.bins_in_fit()
                row["bins_in_fit"] = bins
                for mode in modes:
                    mname = "mle" if mode else "chi2"
                    for nvec in vectors:
                        X = mi.jitter(p.truth, nvec, seed=1, lo=0.95, hi=1.05)
                        dx = torch.tensor(X, dtype=torch.float64, device="cuda")
                        do = torch.empty((nvec, 1 + p.nparams), dtype=torch.float64, device="cuda")
                        t = _sweep_time(B, ctx, dx, nvec, mode, B.MUSR_SPLIT, True, do, flush, stream, 10)
                        row[f"split_{mname}_{nvec}v_gbins_per_s"] = bins * nvec / t / 1e9
                        if nvec == 8 and full:
                            t = _sweep_time(B, ctx, dx, nvec, mode, B.MUSR_FP64, True, do, flush, stream, 2)
                            row[f"fp64_{mname}_8v_gbins_per_s"] = bins * nvec / t / 1e9
                    if name == "cfg1" and full:  # value-only scan of 1000 random vectors (truth x U(0.8, 1.2))
                        X = mi.jitter(p.truth, 1000, seed=1, lo=0.8, hi=1.2)
                        dx = torch.tensor(X, dtype=torch.float64, device="cuda")
                        do = torch.empty((1000, 1 + p.nparams), dtype=torch.float64, device="cuda")
                        for prec, pname in ((B.MUSR_SPLIT, "split"), (B.MUSR_FP64, "fp64")):
                            t = _sweep_time(B, ctx, dx, 1000, mode, prec, False, do, flush, stream, 5)
                            row[f"{pname}_{mname}_scan1000_value_only_gbins_per_s"] = bins * 1000 / t / 1e9
                            row[f"{pname}_{mname}_scan1000_value_only_ms"] = t * 1e3
        if not full:
            out[name] = row
            print(name, json.dumps(row), flush=True)
            continue
        q = p
        if p.H > 16:
            q = dataclasses.replace(p, counts=p.counts[:4], t0=p.t0[:4], map=p.map[:4])
            row["oracle_sample"] = "first 4 histograms"
        qbins = _bins_in_fit(q)
        x = mi.start_point(q, 100)
        for mode in modes:
            mname = "mle" if mode else "chi2"
            oracle.cost(q, x, mode)
            n, t = 0, time.perf_counter()
            while n < 3 or time.perf_counter() - t < 1.0:
                oracle.cost(q, x, mode)
                n += 1
            row[f"oracle_1thread_{mname}_gbins_per_s"] = qbins * n / (time.perf_counter() - t) / 1e9
        out[name] = row
        print(name, json.dumps(row), flush=True)
    print(json.dumps({"config_sweep": out, "cpu": _cpu_model(), "l2": "flushed before every launch"}), flush=True)


def _cpu_model():
    """Host CPU model name and core count (lscpu, else /proc/cpuinfo)."""
    name = None
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in txt.splitlines():
            if line.split(":")[0].strip() == "Model name":
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if name is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": name, "cores": os.cpu_count()}


def _meshes(args):
    return [tuple(int(v) for v in m.split("x")) for m in args.poisson_meshes.split(",") if m]


def poisson_only(args):
    """The particle-mesh Poisson leg alone (one GPU): its JSON object on one line."""
    import torch
    from paper_1509_07685_gb300 import binding as B
    torch.cuda.set_device(0)
    B.load()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    print(json.dumps({"poisson": _poisson(B, peaks, cpu=not args.no_cpu, meshes=_meshes(args))}), flush=True)


def main():
    args = _args()
    if args.precision_report:
        precision_report(args)
        return
    if args.config_sweep:
        config_sweep(args)
        return
    if args.poisson_only:
        poisson_only(args)
        return
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
