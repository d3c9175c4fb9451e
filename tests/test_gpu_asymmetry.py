"""Asymmetry-form fits on the GPU (musr_upload_asymmetry) against the oracle.

* Parity: the FP64 path within 1e-12 (value relative; gradient against the oracle's
  gradient scale), SPLIT within 2^-16 -- for the transverse-field pair configuration, a
  two-term theory with the scale and the baseline fitted, per-pair time-zero offsets (the
  shifted upload) and every count dtype, single and batched evaluations.
* -2lnL is refused for asymmetry data; SPLIT Gauss-Newton products are refused, FP64 ones
  match the oracle's matrix.
* A count the store cannot hold in either histogram of a pair gives MUSR_EINVAL.
* Fits: the SPLIT fit lands within 0.01 sigma of the FP64 fit, which matches the oracle's.
"""
import dataclasses

import numpy as np
import pytest

import musr_inputs as mi
import oracle
from test_gpu_parity import SPLIT_EPS, _check_fp64, _check_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _two_term(p):
    """Cosine term plus an exponential term; scale, baseline, both amplitudes, rates and the
    frequency shared, a phase per pair."""
    terms = [[("AMP", (2,)), ("GAUSS", (3,)), ("TFCOS", (4, 5))], [("AMP", (6,)), ("EXP", (7,))]]
    rows = [[0, 1, 2, 3, 4, 7 + k, 5, 6] for k in range(p.H)]
    names = ["scale", "baseline", "A0", "sigma", "nu", "A1", "lam"] + [f"phi_{k}" for k in range(p.H)]
    truth = np.array([1.0, 0.0, 0.22, 0.4, 3.0, 0.03, 0.5] + list(p.truth[3:]))
    return dataclasses.replace(p, terms=terms, map=np.array(rows, np.int32), consts=np.zeros(0),
                               nparams=len(truth), truth=truth, names=names)


def _cases():
    base = mi.asym_tf(npairs=4, nbins=6000, bin_width_ns=2.0, seed=61)
    return {
        "tf_pairs": base,
        "two_terms": _two_term(base),
        "t0_offsets": dataclasses.replace(base, t0=np.array([0.0, 3.0, 5.5, 8.0]), fit_range_us=(0.02, 11.5)),
        "int32": dataclasses.replace(base, forward=base.forward.astype(np.int32),
                                     backward=base.backward.astype(np.int32)),
        "fp64": dataclasses.replace(base, forward=base.forward.astype(np.float64),
                                    backward=base.backward.astype(np.float64)),
        # a few counts per bin over a larger background: many bins with f + alpha b <= 0
        # (weight 0) and many with one count only
        "low_counts": mi.asym_tf(npairs=3, nbins=5000, bin_width_ns=2.0, seed=64, n0=3.0, nbkg=2.0),
    }


@pytest.mark.parametrize("name", ["tf_pairs", "two_terms", "t0_offsets", "int32", "fp64", "low_counts"])
def test_asymmetry_matches_oracle(B, name):
    p = _cases()[name]
    if name == "low_counts":  # the case does what it is there for
        _, w = oracle.asymmetry(p.forward, p.backward, p.alpha, p.bkg_f, p.bkg_b)
        assert 0.2 < np.mean(w == 0.0) < 0.9
    x = mi.start_point(p, 4)
    X = mi.jitter(x, 6, seed=9, lo=0.98, hi=1.02)
    ref = oracle.cost(p, x, 0)
    assert ref[3] == 0
    with B.Context(p) as ctx:
        assert ctx.bins_in_fit() > 0
        v, g, _ = ctx.eval(x, 0, B.MUSR_FP64)
        _check_fp64(v, g, ref)
        v, g, _ = ctx.eval(x, 0, B.MUSR_SPLIT)
        _check_split(v, g, ref)
        for prec, check in ((B.MUSR_FP64, _check_fp64), (B.MUSR_SPLIT, _check_split)):
            vals, grads, st = ctx.eval_batch(X, 0, prec)
            assert st == 0
            for i in (0, 5):
                check(vals[i], grads[i], oracle.cost(p, X[i], 0))


def test_asymmetry_cost_and_gauss_newton_modes(B):
    p = _cases()["two_terms"]
    x = mi.start_point(p, 5)
    with B.Context(p) as ctx:
        for prec in (B.MUSR_FP64, B.MUSR_SPLIT):
            with pytest.raises(B.MusrError) as e:
                ctx.eval(x, 1, prec)
            assert e.value.status == B.MUSR_EINVAL
        with pytest.raises(B.MusrError) as e:
            ctx.gauss_newton(x, 0, B.MUSR_SPLIT)
        assert e.value.status == B.MUSR_EINVAL
        H = ctx.gauss_newton(x, 0, B.MUSR_FP64)
    ref = oracle.gauss_newton(p, x, 0)
    scale = np.sqrt(np.outer(np.abs(np.diag(ref)), np.abs(np.diag(ref))))
    assert np.all(np.abs(H - ref) <= 1e-12 * scale + 1e-300)


def test_asymmetry_upload_checks_counts(B):
    p = mi.asym_tf(npairs=2, nbins=1000, bin_width_ns=8.0, seed=62)
    ctx = B.musr_ctx_create(0)
    try:
        for which in ("forward", "backward"):
            for dtype, bad in ((np.float32, np.nan), (np.float64, np.inf), (np.int32, 1 << 24)):
                F = np.ascontiguousarray(p.forward.astype(dtype))
                Bk = np.ascontiguousarray(p.backward.astype(dtype))
                (F if which == "forward" else Bk)[1, -1] = bad
                with pytest.raises(B.MusrError) as e:
                    B.musr_upload_asymmetry(ctx, F, Bk, p.t0, p.bin_width_ns, p.fit_range_us, p.alpha, p.bkg_f,
                                            p.bkg_b)
                assert e.value.status == B.MUSR_EINVAL, (which, dtype)
        with pytest.raises(B.MusrError) as e:
            B.musr_upload_asymmetry(ctx, p.forward, p.backward, p.t0, p.bin_width_ns, p.fit_range_us,
                                    -p.alpha, p.bkg_f, p.bkg_b)
        assert e.value.status == B.MUSR_EINVAL
    finally:
        B.musr_ctx_destroy(ctx)


def test_asymmetry_fits(B):
    """musr_fit on asymmetry data: the SPLIT fit within 0.01 sigma of the FP64 fit, and the
    FP64 fit at the oracle's optimum."""
    p = mi.asym_tf(npairs=2, nbins=4000, bin_width_ns=3.0, seed=63, n0=2000.0)
    x0 = mi.start_point(p, 6)
    with B.Context(p) as ctx:
        r64 = B.musr_fit(ctx.ctx, x0, 0, B.MUSR_FP64)
        r32 = B.musr_fit(ctx.ctx, x0, 0, B.MUSR_SPLIT)
    assert r64["status"] == 0 and r32["status"] == 0
    ro = oracle.fit(p, x0, 0)
    assert ro["status"] == 0
    sig = oracle.sigmas(p, ro["x"], 0)
    assert np.all(np.abs(r64["x"] - ro["x"]) / sig < 1e-3), (r64["x"] - ro["x"]) / sig
    assert np.all(np.abs(r32["x"] - r64["x"]) / sig < 0.01), (r32["x"] - r64["x"]) / sig
