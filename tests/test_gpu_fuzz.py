"""Randomised parity: seeded random theories against the oracle, both GPU paths.

Each case draws:
* 1 to 4 terms, each an amplitude times 0 to 3 more primitives of any kind (exponential,
  Gaussian, Gaussian or Lorentzian Kubo-Toyabe, TF cosine, stretched exponential, Bessel).
  Repeats are allowed, so some terms have the basis form and some do not (two cosines,
  a Bessel factor).
* For every slot: a parameter shared by the histograms, one per histogram, or a constant.
  Time-dependent slots are shared or constant in most cases, per histogram in some.
* 1 to 6 histograms of 700 to 3000 bins, with per-histogram time zeros (whole or fractional
  bins, or all equal), a random fit window and a random count dtype.

Amplitudes of at most 0.12 in at most 4 terms keep |A(t)| well below 1 (below 0.7 even at
the few negative times of a window that starts before time zero), so N > 0 and -2lnL is
defined.  The SPLIT planner then picks a basis shape, the generic shape or the term-list
kernel.  Tolerances are those of test_gpu_parity: FP64 1e-12, SPLIT 2^-16, relative to
the value and to the gradient scale; the Gauss-Newton matrices against sqrt(H_pp H_qq).
"""
import numpy as np
import pytest

import musr_inputs as mi
import oracle
from test_gpu_parity import SPLIT_EPS, _check_fp64, _check_split

pytestmark = pytest.mark.gpu

KINDS = ["EXP", "GAUSS", "KT", "LKT", "TFCOS", "STREXP", "BESSEL"]
NCASES = 40


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _value(rng, kind, q):
    """A plausible value for slot q of a primitive of this kind."""
    if kind == "AMP":
        return rng.uniform(0.02, 0.12)
    if kind == "EXP":
        return rng.uniform(0.05, 1.0)
    if kind == "GAUSS":
        return rng.uniform(0.05, 0.8)
    if kind in ("KT", "LKT"):
        return rng.uniform(0.1, 0.8)
    if kind in ("TFCOS", "BESSEL"):
        return rng.uniform(0.5, 8.0) if q == 0 else rng.uniform(0.0, 360.0)
    if kind == "STREXP":
        return rng.uniform(0.1, 1.0) if q == 0 else rng.uniform(0.5, 1.8)
    raise ValueError(kind)


def random_problem(seed):
    rng = np.random.default_rng(seed)
    H = int(rng.integers(1, 7))
    nbins = int(rng.integers(700, 3001))
    dt_ns = float(rng.choice([2.0, 4.0, 6.25, 10.0]))
    per_hist_time = rng.random() < 0.25  # time-dependent slots may differ between histograms
    terms, slot_info = [], [("N0", None, 0), ("NBKG", None, 0)]
    for _ in range(int(rng.integers(1, 5))):
        prims = [("AMP", 1)] + [(k, 2 if k in ("TFCOS", "STREXP", "BESSEL") else 1)
                                for k in rng.choice(KINDS, size=int(rng.integers(0, 4)))]
        term = []
        for kind, ns in prims:
            slots = tuple(range(len(slot_info), len(slot_info) + ns))
            slot_info += [(kind, None, q) for q in range(ns)]
            term.append((str(kind), slots))
        terms.append(term)
    nslots = len(slot_info)
    mp = np.zeros((H, nslots), np.int32)
    truth, consts = [], []
    for s, (kind, _, q) in enumerate(slot_info):
        if kind == "N0":
            how = "hist"
        elif kind == "NBKG":
            how = rng.choice(["hist", "shared"])
        elif kind == "AMP" or (kind in ("TFCOS", "BESSEL") and q == 1):  # amplitudes, phases
            how = rng.choice(["hist", "shared", "const"])
        else:
            how = rng.choice(["hist", "shared", "const"] if per_hist_time else ["shared", "shared", "const"])
        for h in range(H):
            if kind == "N0":
                v = rng.uniform(200.0, 600.0)
            elif kind == "NBKG":
                v = rng.uniform(1.0, 5.0)
            else:
                v = _value(rng, kind, q)
            if how == "hist" or (how == "shared" and h == 0):
                truth.append(v)
                mp[h, s] = len(truth) - 1
            elif how == "shared":
                mp[h, s] = mp[0, s]
            elif h == 0:
                consts.append(v)
                mp[h, s] = -len(consts)
            else:
                mp[h, s] = mp[0, s]
    t0_kind = rng.choice(["zero", "whole", "fraction"])
    t0 = np.zeros(H)
    if t0_kind == "whole":
        t0 = rng.integers(0, 12, H).astype(float)
    elif t0_kind == "fraction":
        t0 = rng.integers(0, 12, H) + rng.uniform(0.0, 1.0, H)
    span = nbins * dt_ns * 1e-3
    lo = float(rng.uniform(-0.02, 0.1) * span)
    hi = float(rng.uniform(0.6, 1.05) * span)
    t = (np.arange(nbins) * dt_ns * 1e-3)[None, :]
    counts = rng.poisson(400.0 * np.exp(-t / 2.197019) * np.ones((H, 1)) + 3.0)
    dtype = rng.choice(["int32", "float32", "float64"])
    counts = counts.astype(dtype)
    P = len(truth)
    return mi.Problem(counts, t0, dt_ns, (lo, hi), terms, mp, np.array(consts), P, np.array(truth),
                      [f"p{i}" for i in range(P)])


@pytest.mark.parametrize("seed", range(NCASES))
def test_random_theory_matches_oracle(B, seed):
    p = random_problem(1000 + seed)
    X = mi.jitter(p.truth, 2, seed=seed, lo=0.97, hi=1.03)
    with B.Context(p) as ctx:
        if ctx.bins_in_fit() == 0:
            pytest.skip("empty fit window")
        for mode in (0, 1):
            for prec, check in ((B.MUSR_FP64, _check_fp64), (B.MUSR_SPLIT, _check_split)):
                ref = oracle.cost(p, X[0], mode)
                assert ref[3] == 0
                v, g, st = ctx.eval(X[0], mode, prec)
                assert st == 0
                check(v, g, ref)
                vals, grads, st = ctx.eval_batch(X, mode, prec)
                assert st == 0
                check(vals[1], grads[1], oracle.cost(p, X[1], mode))


def _check_gn(H, ref, tol):
    scale = np.sqrt(np.outer(np.abs(np.diag(ref)), np.abs(np.diag(ref))))
    bad = np.abs(H - ref) > tol * scale + 1e-300
    assert not bad.any(), (np.argwhere(bad)[:5], float(np.max(np.abs(H - ref) / (scale + 1e-300))))


# J0 and J1 come from two libraries, CUDA's j0/j1 on the device and libstdc++'s
# std::cyl_bessel_j in the oracle.  At the arguments met here (up to 2 pi (8 MHz x 30 us + 1),
# about 1500 rad) they agree to ~5e-13 absolute; the oracle against scipy, a third library,
# differs by 4.4e-13 at most over [0, 2000].  There |J| has the envelope sqrt(2 / (pi x)), about
# 0.02, so the relative difference per bin is up to 5e-13 / 0.02 = 2.5e-11.  A Gauss-Newton
# diagonal squares a derivative carrying that factor: 2 x 2.5e-11 = 5e-11.  The cost and the
# gradient keep 1e-12: there the per-bin differences enter with the residual's changing sign.
BESSEL_GN_TOL = 5e-11


@pytest.mark.parametrize("seed", range(0, NCASES, 2))
def test_random_theory_gauss_newton_matches_oracle(B, seed):
    """Gauss-Newton matrices of the same random theories: the FP64 path for every theory
    (1e-12 of sqrt(H_pp H_qq); BESSEL_GN_TOL with a Bessel factor); SPLIT (2^-16) where the
    theory has a basis form, and MUSR_EINVAL where it has none."""
    p = random_problem(1000 + seed)
    x = mi.jitter(p.truth, 1, seed=seed, lo=0.97, hi=1.03)[0]
    bessel = any(k == "BESSEL" for term in p.terms for k, _ in term)
    with B.Context(p) as ctx:
        if ctx.bins_in_fit() == 0:
            pytest.skip("empty fit window")
        for mode in (0, 1):
            ref = oracle.gauss_newton(p, x, mode)
            _check_gn(ctx.gauss_newton(x, mode, B.MUSR_FP64), ref, BESSEL_GN_TOL if bessel else 1e-12)
            try:
                H = ctx.gauss_newton(x, mode, B.MUSR_SPLIT)
            except B.MusrError as e:  # no basis form: the term-list kernel has no products
                assert e.status == B.MUSR_EINVAL
                continue
            _check_gn(H, ref, SPLIT_EPS)
