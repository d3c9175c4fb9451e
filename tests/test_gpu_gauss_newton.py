"""GPU Gauss-Newton products and matrices (musr_gn_product, musr_gauss_newton) against the
oracle's Gauss-Newton matrix, element by element.

Tolerances, per element (p, q), against the scale sqrt(H_pp H_qq): the FP64 path 1e-12;
SPLIT 2^-16, the per-bin error bound of its FP32 evaluation with margin (the matrix is a
sum of per-bin products of those terms)."""
import numpy as np
import pytest

import musr_inputs as mi
import oracle

from test_gpu_parity import SPLIT_EPS, _build, _shape_cases, problems

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _check(H, ref, tol):
    scale = np.sqrt(np.outer(np.abs(np.diag(ref)), np.abs(np.diag(ref))))
    err = np.abs(H - ref)
    bad = err > tol * scale + 1e-300
    assert not bad.any(), (np.argwhere(bad)[:5], float(np.max(err / (scale + 1e-300))))


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg3", "cfg5", "paper_tf16"])
@pytest.mark.parametrize("mode", [0, 1])
def test_gauss_newton_matches_oracle(B, name, mode):
    p = problems()[name]
    x = mi.start_point(p, 5)
    ref = oracle.gauss_newton(p, x, mode)
    with B.Context(p) as ctx:
        _check(ctx.gauss_newton(x, mode, B.MUSR_FP64), ref, FP64_TOL)
        _check(ctx.gauss_newton(x, mode, B.MUSR_SPLIT), ref, SPLIT_EPS)


@pytest.mark.parametrize("name", sorted(_shape_cases()))
def test_gauss_newton_every_split_shape(B, name):
    terms, slots = _shape_cases()[name]
    p = _build(terms, slots, H=5, seed=sum(map(ord, name)))
    x = p.truth * np.random.default_rng(9).uniform(0.97, 1.03, p.nparams)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            ref = oracle.gauss_newton(p, x, mode)
            _check(ctx.gauss_newton(x, mode, B.MUSR_FP64), ref, FP64_TOL)
            _check(ctx.gauss_newton(x, mode, B.MUSR_SPLIT), ref, SPLIT_EPS)


def test_products_along_arbitrary_directions(B):
    """H v and v^T H v for random directions (several in one launch) match the oracle's
    matrix; the zero direction gives zeros."""
    p = problems()["cfg2"]
    x = mi.start_point(p, 6)
    rng = np.random.default_rng(12)
    V = rng.normal(size=(5, p.nparams))
    V[2] = 0.0
    with B.Context(p) as ctx:
        for mode in (0, 1):
            ref = oracle.gauss_newton(p, x, mode)
            for prec, tol in ((B.MUSR_FP64, FP64_TOL), (B.MUSR_SPLIT, SPLIT_EPS)):
                vhv, hv, st = ctx.gn_product(x, V, mode, prec)
                assert st == B.MUSR_OK
                for i in range(len(V)):
                    r = ref @ V[i]
                    scale = np.abs(ref) @ np.abs(V[i])  # sum |H_pq v_q| bounds the rounding
                    assert np.all(np.abs(hv[i] - r) <= tol * scale + 1e-300)
                    q = V[i] @ ref @ V[i]
                    assert abs(vhv[i] - q) <= tol * (np.abs(V[i]) @ np.abs(ref) @ np.abs(V[i])) + 1e-300
                assert not hv[2].any() and vhv[2] == 0.0


def test_gauss_newton_errors_agree_with_curvature_at_the_optimum(B):
    """At the -2lnL optimum of Poisson data the Gauss-Newton errors agree with those from
    central differences of the analytic gradient (the dropped term averages out)."""
    from paper_1509_07685_gb300 import fit as F
    p = mi.cfg3(nhist=4, nbins=8000, bin_width_ns=1.6, seed=41)
    with B.Context(p) as ctx:
        r = F.fit_context(ctx, mi.start_point(p, 2), 1, B.MUSR_FP64)
        assert r["status"] == 0
        s_fd = F.sigmas_context(ctx, r["x"], 1)
        s_gn = F.sigmas_gauss_newton(ctx, r["x"], 1, B.MUSR_SPLIT)
    assert np.all(np.abs(s_gn / s_fd - 1.0) < 0.05), s_gn / s_fd


def test_undefined_likelihood_is_nonfinite(B):
    p = mi.cfg1(nbins=2048, seed=3, dtype=np.float32)
    x = p.truth.copy()
    x[0], x[1] = -50.0, 0.0
    with B.Context(p) as ctx:
        for prec in (B.MUSR_FP64, B.MUSR_SPLIT):
            vhv, hv, st = ctx.gn_product(x, np.eye(p.nparams)[:2], 1, prec)
            assert st == B.MUSR_ENONFINITE and np.isinf(vhv).all() and not hv.any()
