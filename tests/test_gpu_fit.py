"""GPU fits: the host BFGS driven by the fused kernel.

* The FP32/FP64-split fit lands within 0.01 sigma of the plain FP64 fit (sigma from
  the FP64 Hessian at the FP64 optimum), on every parameter.
* The FP64 GPU fit agrees with the oracle's own fit (different minimiser code, same
  start) to far below a sigma.
* The autograd Function returns the kernel's gradient, which agrees with central
  finite differences of the value; a fit with a finite-difference gradient (2P + 1
  evaluations per gradient) reaches the same optimum as the analytic one.
"""
import numpy as np
import pytest

import musr_inputs as mi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _fit_pair(B, p, mode, seed=1):
    from paper_1509_07685_gb300 import fit as F
    x0 = mi.start_point(p, seed)
    with B.Context(p) as ctx:
        r64 = F.fit_context(ctx, x0, mode, B.MUSR_FP64)
        r32 = F.fit_context(ctx, x0, mode, B.MUSR_SPLIT)
        sig = F.sigmas_context(ctx, r64["x"], mode)
    return r64, r32, sig


@pytest.mark.parametrize("name,mode", [("cfg2", 1), ("cfg2", 0), ("cfg3", 1), ("cfg1", 0)])
def test_split_fit_within_hundredth_sigma_of_fp64(B, name, mode):
    p = {"cfg1": lambda: mi.cfg1(), "cfg2": lambda: mi.cfg2(), "cfg3": lambda: mi.cfg3()}[name]()
    r64, r32, sig = _fit_pair(B, p, mode)
    assert r64["status"] == 0 and r32["status"] == 0, (r64["status"], r32["status"])
    dev = np.abs(r32["x"] - r64["x"]) / sig
    assert np.all(dev < 0.01), dict(zip(p.names, np.round(dev, 4)))


def test_gpu_fit_matches_oracle_fit(B):
    from paper_1509_07685_gb300 import fit as F
    p = mi.cfg3(nhist=2, nbins=8192, bin_width_ns=1.5625, seed=31)
    x0 = mi.start_point(p, 2)
    with B.Context(p) as ctx:
        r = F.fit_context(ctx, x0, 1, B.MUSR_FP64)
        sig = F.sigmas_context(ctx, r["x"], 1)
    ro = oracle.fit(p, x0, 1)
    assert r["status"] == 0 and ro["status"] == 0
    so = oracle.sigmas(p, ro["x"], 1)
    assert np.allclose(sig, so, rtol=1e-3)
    assert np.all(np.abs(r["x"] - ro["x"]) / so < 1e-3)


def test_autograd_gradient_and_fit(B):
    import torch

    from paper_1509_07685_gb300 import autograd as AG
    from paper_1509_07685_gb300 import fit as F
    p = mi.cfg3(nhist=4, nbins=16384, bin_width_ns=0.78125, seed=41)
    x = mi.start_point(p, 5)
    stream = torch.cuda.current_stream().cuda_stream
    with B.Context(p, cuda_stream=stream) as ctx:
        t = torch.tensor(x, dtype=torch.float64, device="cuda", requires_grad=True)
        f = AG.cost(t, ctx, 1, B.MUSR_FP64)
        f.backward()
        g = t.grad.cpu().numpy()
        rv, rg, rgs, _ = oracle.cost(p, x, 1)
        assert abs(f.item() - rv) <= 1e-12 * rv
        assert np.all(np.abs(g - rg) <= 1e-12 * rgs)
        _, gfd = F.fd_gradient_batch(ctx, x, 1, B.MUSR_FP64)
        assert np.all(np.abs(gfd - g) <= 1e-6 * rgs)
        ra = AG.fit_autograd(ctx, x, 1, B.MUSR_SPLIT)
        rc = F.fit_context(ctx, x, 1, B.MUSR_SPLIT)
        sig = F.sigmas_context(ctx, rc["x"], 1)
        assert ra["status"] == 0 and rc["status"] == 0
        assert np.all(np.abs(ra["x"] - rc["x"]) / sig < 0.01)


def test_finite_difference_gradient_fit_reaches_same_optimum(B):
    """cfg3-shaped fit: BFGS with the analytic gradient kernel vs with central differences."""
    from paper_1509_07685_gb300 import fit as F
    p = mi.cfg3()
    x0 = mi.start_point(p, 7)
    with B.Context(p) as ctx:
        ra = F.fit_context(ctx, x0, 1, B.MUSR_FP64)
        fd_evals = [0]

        def fg(x):
            v, g = F.fd_gradient_batch(ctx, x, 1, B.MUSR_FP64)
            fd_evals[0] += 2 * x.size + 1
            return v, g

        rf = F.bfgs(fg, x0)
        sig = F.sigmas_context(ctx, ra["x"], 1)
    assert ra["status"] == 0 and rf["status"] == 0
    assert np.all(np.abs(ra["x"] - rf["x"]) / sig < 0.01)
    assert fd_evals[0] >= (2 * p.nparams + 1) * rf["nfev"] // 2


def test_cfg1_scan_of_1000_random_vectors_fp64(B):
    """The cfg1 workload: value only, FP64, chi^2 and -2lnL at 1000 random parameter vectors
    (truth x U(0.8, 1.2), seed 1), in one batched launch each, against the oracle."""
    p = mi.cfg1()
    X = mi.jitter(p.truth, 1000, seed=1)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            vals, _, st = ctx.eval_batch(X, mode, B.MUSR_FP64, grad=False)
            assert st == 0
            for i in range(0, 1000, 37):
                rv = oracle.cost(p, X[i], mode, grad=False)[0]
                assert abs(vals[i] - rv) <= 1e-12 * abs(rv)
            vs, _, _ = ctx.eval_batch(X, mode, B.MUSR_SPLIT, grad=False)
            assert np.all(np.abs(vs - vals) <= 2.0 ** -16 * np.abs(vals))


@pytest.mark.slow
def test_large_fit_split_vs_fp64(B):
    """64 x 2^20 bins, 197 parameters, -2lnL: SPLIT fit within 0.01 sigma of the FP64 fit."""
    p = mi.cfg5()
    r64, r32, sig = _fit_pair(B, p, 1)
    assert r64["status"] == 0 and r32["status"] == 0
    dev = np.abs(r32["x"] - r64["x"]) / sig
    assert np.all(dev < 0.01), float(dev.max())


@pytest.mark.parametrize("name", ["levy_lf", "inc_bessel"])
def test_split_fit_of_term_lists_without_basis_form(B, name):
    """Theories without a basis form (a stretched exponential, a Bessel precession): the SPLIT
    fit, through the term list kernel, lands within 0.01 sigma of the FP64 fit."""
    from paper_1509_07685_gb300 import fit as F
    p = mi.levy_lf(seed=109) if name == "levy_lf" else mi.inc_bessel(seed=108)
    x0 = mi.start_point(p, 1)
    with B.Context(p) as ctx:
        r64 = F.fit_context(ctx, x0, 1, B.MUSR_FP64)
        r32 = F.fit_context(ctx, x0, 1, B.MUSR_SPLIT)
        sig = F.sigmas_context(ctx, r64["x"], 1)
    assert r64["status"] == 0 and r32["status"] == 0
    dev = np.abs(r32["x"] - r64["x"]) / sig
    assert np.all(dev < 0.01), dict(zip(p.names, np.round(dev, 4)))
