"""Host-only logic of the library, on the CPU: the BFGS state machine behind musr_fit and
the serving loop (musr_bfgs.h), the planning of the SPLIT kernels (musr_plan.h: canonical
terms, shape, merging, slot contributions) and the decomposition cost model (musr_dev.h).
tests/host_logic.cpp drives the headers; g++ builds it with the CUDA vector types only."""
import json
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_logic.cpp")
EXE = os.path.join(ROOT, "tests", "_build", "host_logic")  # git-ignored
CSRC = os.path.join(ROOT, "paper_1509_07685_gb300", "csrc")

# SPLIT shapes and term kinds as numbered in musr_dev.h
SHAPE = {"generic": 0, "T1": 1, "N1": 2, "T1N1": 3, "T2": 4, "T2N1": 5, "T2m": 6, "T2N1m": 7}
TERM = {"plain": 1, "tf": 2, "kt": 3, "lkt": 4, "dkt": 5}
C_AMP, C_PHI, C_DEL, C_LKT, C_DKT_D, C_DKT_N = 2, 3, 7, 8, 9, 10


def _cuda_include():
    for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include")):
        if os.path.exists(os.path.join(d, "vector_types.h")):
            return d
    pytest.skip("CUDA headers not found")


@pytest.fixture(scope="module")
def run():
    deps = [SRC] + [os.path.join(CSRC, f) for f in ("musr_bfgs.h", "musr_plan.h", "musr_dev.h", "musr_partition.h")] + \
        [os.path.join(ROOT, "include", "musr.h")]
    if not os.path.exists(EXE) or os.path.getmtime(EXE) < max(os.path.getmtime(d) for d in deps):
        os.makedirs(os.path.dirname(EXE), exist_ok=True)
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                               "-I", _cuda_include(), "-o", EXE, SRC])

    def _run(what):
        out = subprocess.run([EXE, what], capture_output=True, text=True, check=True).stdout
        return {d["name"] if d["name"] != "pick" else d["nvec"]: d for d in map(json.loads, out.splitlines())}
    return _run


def test_bfgs_state_machine_minimises(run):
    r = run("bfgs")
    q = r["quadratic"]
    assert q["status"] == 0
    assert np.allclose(q["x"], [1.5, -2.0, 0.25, 3.0], atol=1e-6)
    # the start point, then the P points of the diagonal curvature estimate, then single trials
    assert q["first_requests"][:3] == [1, 4, 1]
    rb = r["rosenbrock"]
    assert rb["status"] == 0 and np.allclose(rb["x"], [1.0, 1.0], atol=1e-6) and rb["f"] < 1e-12
    nf = r["nonfinite"]
    assert nf["status"] == 1 and nf["nfev"] == 1


def test_split_planning(run):
    r = run("plan")
    m = r["tf2_merged"]
    assert m["ok"] and m["shape"] == SHAPE["T2m"] and m["merged"] == 1
    assert m["bamp"] == pytest.approx([0.125, 0.1], rel=1e-7)
    kinds = [c[1] for c in m["contrib"]]
    assert kinds.count(C_PHI) == 1 and C_AMP not in kinds  # one shared phase, constant amplitudes
    for name in ("tf2_own_phases", "tf2_amp_per_hist"):
        assert r[name]["shape"] == SHAPE["T2"] and r[name]["merged"] == 0
    assert [c[1] for c in r["tf2_own_phases"]["contrib"]].count(C_PHI) == 2
    k = r["kt_then_tf"]  # the cosine term moves first
    assert k["shape"] == SHAPE["T1N1"] and k["kinds"] == [TERM["tf"], TERM["kt"]]
    assert [3, C_DEL, 1] in k["contrib"]
    lk = r["lkt"]
    assert lk["shape"] == SHAPE["N1"] and lk["kinds"] == [TERM["lkt"]] and [3, C_LKT, 0] in lk["contrib"]
    assert not r["two_cosines"]["ok"]
    g = r["generic4"]
    assert g["shape"] == SHAPE["generic"] and g["kinds"] == [TERM["tf"], TERM["plain"], TERM["plain"], TERM["kt"]]
    d = r["dkt_then_tf"]  # the cosine term moves first; the dynamic KT term keeps both its slots
    assert d["ok"] and d["shape"] == SHAPE["T1N1"] and d["kinds"] == [TERM["tf"], TERM["dkt"]]
    assert [3, C_DKT_D, 1] in d["contrib"] and [4, C_DKT_N, 1] in d["contrib"]
    assert not r["dkt_times_cosine"]["ok"]


def test_decomposition_cost_model(run):
    r = run("pick")
    for nvec, d in r.items():
        costs = d["costs"]
        assert d["v"] == int(np.argmin(costs))  # the first (smallest-tile) minimum
    assert r[1]["v"] == 0 and r[8]["v"] == 2 and r[64]["v"] == 5 and r[152]["v"] == 6


PARTITION_CASES = {  # name: chunk iterations, chunk loads, vectors, CTAs, largest piece, piece cost (host_logic.cpp)
    "paper_64": ([160, 160], [2.4, 2.4], 64, 304, 64, 1.3),
    "cfg2_64": ([128], [2.4], 64, 304, 64, 1.3),
    "uneven": ([7, 100, 33], [1.0, 2.0, 3.0], 5, 13, 16, 1.3),
    "long": ([2048, 2048, 2048], [2.4, 2.4, 2.4], 3, 7, 64, 1.3),
    "tiny": ([3, 5], [1.0, 2.0], 3, 4, 2, 0.5),
    "cfg2_64_chi2": ([128], [3.6], 64, 304, 64, 1.95),
    "paper_8": ([160, 160], [2.4, 2.4], 8, 304, 64, 1.3),
}


def _range_cost(iters, load, max_piece, piece, lo, hi):
    """Cost of the CTA range [lo, hi) of the batch order: its iterations, a piece cost per
    piece (cut at the largest piece from the range's start in each chunk) and a chunk load
    per chunk it starts on."""
    pre = np.concatenate([[0], np.cumsum(iters)])
    S = int(pre[-1])
    c, q = float(hi - lo), lo
    while q < hi:
        j, off = divmod(q, S)
        k = int(np.searchsorted(pre, off, side="right") - 1)
        n = min(hi - q, iters[k] - (off - int(pre[k])))
        c += load[k] + piece * -(-n // max_piece)
        q += n
    return c


def _check_partition(p, iters, load, nvec, G, max_piece, piece):
    """Invariants of one cut (see test_partition_invariants)."""
    pieces, cta, nck = p["pieces"], p["cta"], len(iters)
    pre = np.concatenate([[0], np.cumsum(iters)])
    S = int(pre[-1])
    I = S * nvec
    assert p["grid"] == G and len(cta) == G + 1 and cta[0] == 0 and cta[-1] == len(pieces)
    assert all(a <= b for a, b in zip(cta, cta[1:]))
    q, costs, counts = 0, [], []
    for b in range(G):
        lo, cost, prev = q, 0.0, None
        for j, k, it0, nit, row in pieces[cta[b]:cta[b + 1]]:
            assert 1 <= nit <= max_piece and 0 <= it0 and it0 + nit <= iters[k]
            assert j * S + pre[k] + it0 == q  # the next iteration of the batch order
            q += nit
            cost += nit + piece + (load[k] if prev != (j, k) else 0.0)
            prev = (j, k)
        assert cost == pytest.approx(_range_cost(iters, load, max_piece, piece, lo, q), abs=1e-9)
        costs.append(cost)
        counts.append(q - lo)
    assert q == I
    assert p["worst"] == pytest.approx(max(costs), rel=1e-12, abs=1e-12)
    equal = max(_range_cost(iters, load, max_piece, piece, I * b // G, I * (b + 1) // G) for b in range(G))
    assert p["equal"] == pytest.approx(equal, rel=1e-12, abs=1e-12)
    if counts != [I * (b + 1) // G - I * b // G for b in range(G)]:  # the cost-balanced cut
        assert p["worst"] <= 0.95 * equal + 1e-9
    rows = p["rows"]
    cr = np.array(p["chunk_rows"]).reshape(nvec, nck, 2)
    for j in range(nvec):
        own = [pc for pc in pieces if pc[0] == j]
        assert rows[j] == len(own) and sorted(pc[4] for pc in own) == list(range(rows[j]))
        for k in range(nck):
            ck = [pc for pc in own if pc[1] == k]
            first, count = cr[j, k]
            assert count == len(ck) and [pc[4] for pc in ck] == list(range(first, first + count))
            assert sum(pc[3] for pc in ck) == iters[k]


def test_partition_invariants(run):
    """The launch-level partition: each job's chunk iterations are covered exactly once, in
    order, by pieces of at most the largest piece; the CTAs take consecutive ranges of the
    batch order; a job's rows follow its pieces and each chunk's rows are contiguous; the
    returned cost is the busiest CTA's.  The ranges hold equal iteration counts (within one)
    unless ranges of equal cost lower the busiest CTA's cost by 5 % or more."""
    r = run("partition")
    for name, case in PARTITION_CASES.items():
        _check_partition(r[name], *case)
    # which cut each case takes (model costs: 34.4 -> 31.7, 38.1 -> 33.55, 75.4 -> 74.0)
    assert r["cfg2_64"]["worst"] == pytest.approx(31.7) and r["cfg2_64_chi2"]["worst"] == pytest.approx(33.55)
    assert r["paper_64"]["worst"] == pytest.approx(75.4) and r["paper_8"]["worst"] == pytest.approx(12.7)
    # the compiled decomposition's busiest CTA: ceil(640 / 304) = 3 items of 8 iterations, a
    # piece cost each and a chunk load at the start and after 5 items
    assert r["paper_64"]["items_cost"] == pytest.approx(3 * (8 + 1.3) + 2 * 2.4, rel=1e-12)


def test_partition_invariants_on_random_batches(run):  # run: the harness is built
    """The same invariants on 300 seeded random batches: 1-4 chunks of 1-60 iterations, loads
    0-5, 1-6 vectors, 1-40 CTAs (some batches smaller than the grid, leaving CTAs empty),
    pieces of 1-16 iterations, piece costs 0-2."""
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(300):
        nck = int(rng.integers(1, 5))
        cases.append(([int(v) for v in rng.integers(1, 61, nck)], [float(v) for v in np.round(rng.uniform(0, 5, nck), 3)],
                      int(rng.integers(1, 7)), int(rng.integers(1, 41)), int(rng.integers(1, 17)),
                      float(np.round(rng.uniform(0, 2), 3))))
    text = "".join(f"{len(it)} {' '.join(map(str, it))} {' '.join(map(str, ld))} {nv} {G} {mp} {pc}\n"
                   for it, ld, nv, G, mp, pc in cases) + "0\n"
    out = subprocess.run([EXE, "partition_stdin"], input=text, capture_output=True, text=True, check=True).stdout
    got = {d["name"]: d for d in map(json.loads, out.splitlines())}
    assert len(got) == len(cases)
    balanced = 0
    for i, case in enumerate(cases):
        _check_partition(got[str(i)], *case)
        balanced += got[str(i)]["worst"] < got[str(i)]["equal"] - 1e-9
    assert balanced > 0  # the cost-balanced cut is exercised


def test_partition_balanced_cut_is_optimal_on_a_tiny_batch(run):
    """Brute force: the smallest busiest-CTA cost over every cut of the 24 iterations of the
    tiny batch into 4 contiguous ranges (dynamic programming over the range ends) equals the
    cost-balanced cut's, to the bisection's tolerance."""
    iters, load, nvec, G, max_piece, piece = PARTITION_CASES["tiny"]
    I = sum(iters) * nvec
    best = {(0, 0): 0.0}  # (ranges used, iterations covered) -> smallest busiest cost
    for g in range(1, G + 1):
        for e in range(I + 1):
            cands = [max(best[(g - 1, s)], _range_cost(iters, load, max_piece, piece, s, e) if e > s else 0.0)
                     for s in range(e + 1) if (g - 1, s) in best]
            best[(g, e)] = min(cands)
    opt = best[(G, I)]
    w = run("partition")["tiny"]["worst"]
    assert opt - 1e-9 <= w <= opt + 1e-3
