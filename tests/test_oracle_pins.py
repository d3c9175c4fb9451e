"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's formulas: every expected value comes
from a closed form (geometric series of the decay and of the damped cosine), a
special value (Kubo-Toyabe at 0, at infinity and at its minimum), an exact
identity (data equal to the model), an optimum known in closed form (constant
model), an independent differentiation method (complex step, finite
differences) or an exactly rounded sum.  Each test names the mistake it is
there to catch.
"""
import math

import numpy as np
import pytest

import oracle
from musr_inputs import TAU_MU_US, Problem

CHI2, MLE = oracle.CHI2, oracle.MLE


def _problem(counts, terms, mp, nparams, bin_width_ns=0.5, t0=None, fit=(0.0, 1e9), consts=()):
    counts = np.atleast_2d(np.asarray(counts, dtype=np.float64))
    H = counts.shape[0]
    return Problem(counts, np.zeros(H) if t0 is None else np.asarray(t0, float), bin_width_ns,
                   fit, terms, np.atleast_2d(np.asarray(mp, np.int32)),
                   np.asarray(consts, dtype=np.float64), nparams, np.zeros(nparams),
                   [f"p{i}" for i in range(nparams)])


# ------------------------------------------------------------------------------------------
# Primitives (Eq. asymmetry and its generalisation)
# ------------------------------------------------------------------------------------------

def test_kubo_toyabe_special_values():
    """KT(0) = 1, KT(inf) = 1/3, minimum at t = sqrt(3)/Delta equal to 1/3 - (4/3) e^{-3/2}.

    Catches a wrong exponent factor, a wrong sign of the (1 - Delta^2 t^2) factor and
    wrong 1/3, 2/3 weights."""
    from scipy.optimize import minimize_scalar
    for delta in (0.1, 0.3, 1.7):
        assert oracle.primitive("KT", delta, 0.0, 0.0) == 1.0
        assert abs(oracle.primitive("KT", delta, 0.0, 60.0 / delta) - 1.0 / 3.0) < 1e-15
        res = minimize_scalar(lambda t: oracle.primitive("KT", delta, 0.0, t),
                              bounds=(0.5 / delta, 4.0 / delta), method="bounded",
                              options={"xatol": 1e-10})
        assert abs(res.x - math.sqrt(3.0) / delta) < 1e-4 / delta
        assert abs(res.fun - (1.0 / 3.0 - (4.0 / 3.0) * math.exp(-1.5))) < 1e-12


def test_lorentzian_kubo_toyabe_special_values():
    """LKT(0) = 1, LKT(inf) = 1/3, LKT(1/a) = 1/3 exactly (the factor 1 - a t vanishes), and the
    minimum at t = 2/a equal to 1/3 - (2/3) e^{-2}.  Catches a squared argument, a wrong sign of
    the (1 - a t) factor and wrong 1/3, 2/3 weights."""
    from scipy.optimize import minimize_scalar
    for a in (0.2, 0.6, 2.5):
        assert oracle.primitive("LKT", a, 0.0, 0.0) == 1.0
        assert abs(oracle.primitive("LKT", a, 0.0, 80.0 / a) - 1.0 / 3.0) < 1e-15
        assert abs(oracle.primitive("LKT", a, 0.0, 1.0 / a) - 1.0 / 3.0) < 1e-16
        res = minimize_scalar(lambda t: oracle.primitive("LKT", a, 0.0, t), bounds=(0.5 / a, 5.0 / a),
                              method="bounded", options={"xatol": 1e-10})
        assert abs(res.x - 2.0 / a) < 1e-4 / a
        assert abs(res.fun - (1.0 / 3.0 - (2.0 / 3.0) * math.exp(-2.0))) < 1e-12


def test_relaxation_primitives_special_values():
    """EXP at lambda t = 1 is 1/e; GAUSS at sigma t = sqrt(2) is 1/e (the factor 1/2 of
    Eq. asymmetry); both are even/odd as they must be."""
    assert abs(oracle.primitive("EXP", 0.5, 0.0, 2.0) - math.exp(-1.0)) < 4e-16
    assert abs(oracle.primitive("GAUSS", 0.3, 0.0, math.sqrt(2.0) / 0.3) - math.exp(-1.0)) < 4e-16
    assert oracle.primitive("GAUSS", -0.3, 0.0, 1.0) == oracle.primitive("GAUSS", 0.3, 0.0, 1.0)
    assert oracle.primitive("AMP", 0.125, 0.0, 3.0) == 0.125


def test_tf_cosine_units():
    """cos(2 pi (nu t + phi/360)): nu in MHz with t in us, phi in degrees.

    Catches radians/degrees, a missing 2 pi, and a sign error on the phase."""
    assert abs(oracle.primitive("TFCOS", 1.0, 0.0, 0.25)) < 1e-15  # quarter turn
    assert abs(oracle.primitive("TFCOS", 1.0, 90.0, 0.0)) < 1e-15
    assert oracle.primitive("TFCOS", 7.0, 180.0, 0.0) == -1.0
    assert abs(oracle.primitive("TFCOS", 2.0, 30.0, 0.125) + 0.5) < 1e-15  # cos(pi/2 + pi/6)
    assert abs(oracle.primitive("TFCOS", 5.0, 10.0, 0.0) - math.cos(math.radians(10.0))) < 1e-16


# ------------------------------------------------------------------------------------------
# Costs in closed form
# ------------------------------------------------------------------------------------------

def test_data_equal_model_gives_zero():
    """chi^2 = 0 and -2lnL = 0 when the data equal the model (Eq. chisq, Eq. log-likelihood).

    Catches a wrong sign or a dropped (N - d) term of the likelihood."""
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))], [("AMP", (6,)), ("KT", (7,))]]
    mp = [[0, 1, 2, 3, 4, 5, 6, 7]]
    x = np.array([250.0, 3.0, 0.2, 0.4, 3.0, 20.0, 0.1, 0.5])
    p = _problem(np.zeros((1, 700)), terms, mp, 8, bin_width_ns=10.0, fit=(0.0, 6.0))
    dt = p.bin_width_ns / 1000.0
    d = np.array([[oracle.model(p, x, 0, n * dt) for n in range(700)]])
    p = p.with_counts(d)
    for mode in (CHI2, MLE):
        v, g, gs, st = oracle.cost(p, x, mode)
        assert st == 0
        assert abs(v) < 1e-18 * 700 + 1e-20
        assert np.all(np.abs(g) <= 1e-12 * gs + 1e-300)


def test_constant_model_closed_forms():
    """Constant model N = c (N0 = 0, A = 0) on constant data k:
    chi^2 = n (k - c)^2 / max(k, 1);  -2lnL = 2 n [(c - k) + k ln(k / c)]  (k > 0), 2 n c (k = 0)."""
    n = 333
    for k, c in ((7.0, 5.5), (0.0, 2.5), (1.0, 0.25), (0.5, 3.0)):
        p = _problem(np.full((1, n), k), [], [[0, 1]], 2, fit=(0.0, 1e9))
        x = np.array([0.0, c])
        chi2, _, _, _ = oracle.cost(p, x, CHI2, grad=False)
        assert chi2 == pytest.approx(n * (k - c) ** 2 / max(k, 1.0), rel=1e-14)
        mle, _, _, _ = oracle.cost(p, x, MLE, grad=False)
        ref = 2 * n * ((c - k) + k * math.log(k / c)) if k > 0 else 2 * n * c
        assert mle == pytest.approx(ref, rel=1e-13)


def _geom(a, b, t0, c):
    """sum_{n=a}^{b} exp((n - t0) c) for real or complex c (closed form)."""
    m = b - a + 1
    return np.exp((a - t0) * c) * np.expm1(m * c) / np.expm1(c)


def test_exponential_decay_geometric_sum():
    """Pure decay N = N0 e^{-t/tau}, d = 0: -2lnL = 2 N0 sum r^(n - t0), chi^2 = N0^2 sum r^(2(n - t0)).

    The fit range and t0 are chosen so that the first and last bins are known by hand:
    dt = 0.5 ns, t0 = 10.25 bins, range [0.01, 1.0] us -> bins 31 .. 2010 (closed range).
    Catches tau_mu, the ns -> us conversion, the sign of t0 and an open/closed range."""
    N0 = 123.0
    p = _problem(np.zeros((1, 4096)), [], [[0, 1]], 2, bin_width_ns=0.5, t0=[10.25],
                 fit=(0.01, 1.0))
    x = np.array([N0, 0.0])
    dt = 0.5e-3
    S1 = _geom(31, 2010, 10.25, -dt / TAU_MU_US)
    S2 = _geom(31, 2010, 10.25, -2.0 * dt / TAU_MU_US)
    mle, _, _, _ = oracle.cost(p, x, MLE, grad=False)
    chi2, _, _, _ = oracle.cost(p, x, CHI2, grad=False)
    assert mle == pytest.approx(2.0 * N0 * S1, rel=1e-13)
    assert chi2 == pytest.approx(N0 * N0 * S2, rel=1e-13)


def test_fit_range_is_closed_at_both_ends():
    """A bin whose time equals lo or hi exactly is in the fit (the range is closed)."""
    # dt = 1 ns = 1e-3 us (exact products), t0 = 0; t_n = n * 1e-3.  lo = t_4, hi = t_9.
    p = _problem(np.zeros((1, 16)), [], [[0, 1]], 2, bin_width_ns=1.0, fit=(4 * 1e-3, 9 * 1e-3))
    mle, _, _, _ = oracle.cost(p, np.array([0.0, 1.0]), MLE, grad=False)
    assert mle == pytest.approx(2.0 * 6, rel=1e-15)  # bins 4..9, N = Nbkg = 1 each


def test_damped_cosine_geometric_sum():
    """N = N0 e^{-t/tau} [1 + A e^{-lambda t} cos(2 pi (nu t + phi/360))] + Nbkg with d = 0:
    -2lnL / 2 = N0 S(-dt/tau) + N0 A Re(e^{i phi} S(c)) + Nbkg n, c = (-1/tau - lambda + 2 pi i nu) dt.

    Catches the phase convention, the frequency unit, the sign of lambda, a dropped N0
    on the asymmetry term and a dropped background."""
    N0, Nbkg, A, lam, nu, phi = 80.0, 1.5, 0.3, 0.7, 13.0, 37.0
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))]]
    p = _problem(np.zeros((1, 5000)), terms, [[0, 1, 2, 3, 4, 5]], 6, bin_width_ns=0.8,
                 t0=[3.5], fit=(0.0002, 3.0))
    # t_n = (n - 3.5) * 8e-4 >= 2e-4 -> n >= 3.75 -> first 4; <= 3.0 -> n <= 3753.5 -> last 3753
    a, b, t0, dt = 4, 3753, 3.5, 0.8e-3
    c = complex(-1.0 / TAU_MU_US - lam, 2.0 * math.pi * nu) * dt
    S0 = _geom(a, b, t0, -dt / TAU_MU_US)
    S1 = _geom(a, b, t0, c)
    ref = 2.0 * (N0 * S0 + N0 * A * (np.exp(1j * math.radians(phi)) * S1).real + Nbkg * (b - a + 1))
    mle, _, _, _ = oracle.cost(p, np.array([N0, Nbkg, A, lam, nu, phi]), MLE, grad=False)
    assert mle == pytest.approx(ref, rel=1e-12)


def test_likelihood_undefined_when_model_not_positive():
    """-2lnL is +inf (status 1) when N <= 0 in a bin with d > 0; d = 0 bins stay finite."""
    p = _problem(np.array([[0.0, 3.0, 0.0]]), [], [[0, 1]], 2, fit=(0.0, 1e9))
    v, g, gs, st = oracle.cost(p, np.array([0.0, -1.0]), MLE)
    assert st == 1 and math.isinf(v) and np.all(g == 0.0)
    p0 = p.with_counts(np.array([[0.0, 0.0, 0.0]]))
    v, _, _, st = oracle.cost(p0, np.array([0.0, -1.0]), MLE)
    assert st == 0 and v == pytest.approx(-6.0)
    v, _, _, st = oracle.cost(p, np.array([0.0, -1.0]), CHI2)
    assert st == 0 and np.isfinite(v)


def test_costs_are_nonnegative_and_chi2_weights_use_data():
    """Both costs are >= 0 on Poisson data; the chi^2 variance is max(d, 1) of the data
    (Neyman), so doubling the model leaves the weights unchanged.  Catches a variance taken
    from the theory."""
    rng = np.random.default_rng(11)
    d = rng.poisson(3.0, size=(2, 300)).astype(float)
    p = _problem(d, [], [[0, 1], [0, 1]], 2, fit=(0.0, 1e9))
    for c in (0.5, 3.0, 9.0):
        for mode in (CHI2, MLE):
            v, _, _, _ = oracle.cost(p, np.array([0.0, c]), mode, grad=False)
            assert v >= 0.0
        chi2, _, _, _ = oracle.cost(p, np.array([0.0, c]), CHI2, grad=False)
        ref = math.fsum(((dd - c) ** 2 / max(dd, 1.0)) for dd in d.ravel())
        assert chi2 == pytest.approx(ref, rel=1e-14)


def test_neumaier_sum_is_exact_on_cancelling_series():
    """The compensated sum matches the exactly rounded sum (math.fsum) where naive
    summation loses every digit."""
    rng = np.random.default_rng(3)
    big = rng.uniform(1e15, 1e16, 5000)
    v = np.concatenate([big, rng.uniform(0, 1, 5000), -big])
    rng.shuffle(v)
    assert oracle.neumaier_sum(v) == pytest.approx(math.fsum(v), abs=1e-9)


# ------------------------------------------------------------------------------------------
# Gradient: analytic vs complex step vs central differences
# ------------------------------------------------------------------------------------------

def _small_problems():
    import musr_inputs as mi
    return [
        mi.cfg1(nbins=700, bin_width_ns=11.0, seed=21, dtype=np.float64),
        mi.cfg2(nhist=3, nbins=400, bin_width_ns=30.0, seed=22),
        mi.cfg3(nhist=2, nbins=500, bin_width_ns=25.0, seed=23),
        mi.cfg5(nhist=2, nbins=600, seed=24, n0=40.0, nbkg=0.5),
        mi.paper_tf16(nhist=3, nbins=300, seed=25, n0=50.0),
    ]


@pytest.mark.parametrize("mode", [CHI2, MLE])
def test_gradient_matches_complex_step(mode):
    """Every component of the analytic gradient equals the complex-step derivative of the
    value (same model, different differentiation).  Catches a wrong primitive derivative,
    a wrong chain factor (2 pi / 360, sigma t^2, ...) and a map scatter to the wrong index."""
    rng = np.random.default_rng(5)
    for p in _small_problems():
        x = p.truth * rng.uniform(0.9, 1.1, p.nparams)
        v, g, gs, st = oracle.cost(p, x, mode)
        assert st == 0
        for i in range(p.nparams):
            e = np.zeros(p.nparams)
            e[i] = 1.0
            cs = oracle.cost_cstep(p, x, e, mode)
            assert abs(cs - g[i]) <= 1e-11 * gs[i] + 1e-300, (p.name, i, cs, g[i], gs[i])


@pytest.mark.parametrize("mode", [CHI2, MLE])
def test_gradient_matches_complex_step_lorentzian(mode):
    """The same check for a theory with the Lorentzian Kubo-Toyabe primitive (alone and
    multiplied by other relaxations)."""
    import musr_inputs as mi
    p = mi.lkt_zf(nhist=2, nbins=500, bin_width_ns=25.0, seed=26, n0=200.0)
    terms = [[("AMP", (2,)), ("LKT", (3,))], [("AMP", (4,)), ("LKT", (5,)), ("EXP", (6,))]]
    rows = [[0, 1, 2, 3, 4, 5, 6], [7, 8, 2, 3, 4, 5, 6]]
    q = Problem(p.counts, p.t0, p.bin_width_ns, p.fit_range_us, terms, np.array(rows, np.int32), np.zeros(0), 9,
                np.zeros(9), [f"p{i}" for i in range(9)])
    x = np.array([200.0, 2.0, 0.15, 0.6, 0.08, 1.1, 0.3, 190.0, 2.5])
    v, g, gs, st = oracle.cost(q, x, mode)
    assert st == 0
    for i in range(q.nparams):
        e = np.zeros(q.nparams)
        e[i] = 1.0
        cs = oracle.cost_cstep(q, x, e, mode)
        assert abs(cs - g[i]) <= 1e-11 * gs[i] + 1e-300, (i, cs, g[i], gs[i])


def test_gradient_matches_central_differences():
    """Central differences of the value agree with the analytic gradient to FD accuracy."""
    import musr_inputs as mi
    p = mi.cfg3(nhist=2, nbins=300, bin_width_ns=40.0, seed=31)
    x = p.truth * 1.05
    for mode in (CHI2, MLE):
        _, g, gs, _ = oracle.cost(p, x, mode)
        for i in range(p.nparams):
            h = 1e-6 * max(abs(x[i]), 1e-3)
            xp, xm = x.copy(), x.copy()
            xp[i] += h
            xm[i] -= h
            fd = (oracle.cost(p, xp, mode, grad=False)[0] - oracle.cost(p, xm, mode, grad=False)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * gs[i], (i, fd, g[i])


# ------------------------------------------------------------------------------------------
# The minimiser: optima known in closed form
# ------------------------------------------------------------------------------------------

def test_fit_constant_model_optima():
    """The -2lnL optimum of a constant model is c = mean(d); the chi^2 optimum is the
    weighted mean c = sum(d / w) / sum(1 / w), w = max(d, 1) (= n / sum(1 / w) when every
    d >= 1).  Pins the minimiser and both gradients at the optimum."""
    rng = np.random.default_rng(7)
    d = rng.poisson(4.2, size=(2, 900)).astype(float)
    p = _problem(d, [], [[0, 1], [0, 1]], 2, fit=(0.0, 1e9))
    # parameter 0 (N0) is held at 0 through a constant in the map: map slot 0 -> const 0
    p = Problem(p.counts, p.t0, p.bin_width_ns, p.fit_range_us, [], np.array([[-1, 0], [-1, 0]], np.int32),
                np.array([0.0]), 1, np.zeros(1), ["c"])
    r = oracle.fit(p, np.array([1.0]), MLE)
    assert r["status"] == 0
    assert r["x"][0] == pytest.approx(d.mean(), rel=1e-9)
    r = oracle.fit(p, np.array([1.0]), CHI2)
    assert r["status"] == 0
    w = np.maximum(d, 1.0)
    assert r["x"][0] == pytest.approx(np.sum(d / w) / np.sum(1.0 / w), rel=1e-9)


def test_sigma_of_constant_model_is_poisson():
    """At the -2lnL optimum of a constant model, sigma(c) = sqrt(c / n) (Poisson error of a mean)."""
    rng = np.random.default_rng(8)
    d = rng.poisson(6.0, size=(1, 2000)).astype(float)
    p = Problem(d, np.zeros(1), 0.5, (0.0, 1e9), [], np.array([[-1, 0]], np.int32), np.array([0.0]), 1,
                np.zeros(1), ["c"])
    c = d.mean()
    s = oracle.sigmas(p, np.array([c]), MLE)
    assert s[0] == pytest.approx(math.sqrt(c / d.size), rel=1e-6)


# ------------------------------------------------------------------------------------------
# Parameter layout of the paper's benchmark
# ------------------------------------------------------------------------------------------

def test_paper_parameter_count_and_map_layout():
    """Section 4: 16 positron detectors with Eq. asymmetry need 66 fit parameters
    (tests/golden/paper_parameter_count.txt).  The configs' maps reference every
    parameter exactly as laid out."""
    import musr_inputs as mi
    golden = {}
    with open(__import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                         "paper_parameter_count.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                golden[k.strip()] = int(v)
    p = mi.paper_tf16(nbins=64)
    assert p.H == golden["detectors"]
    assert p.nparams == golden["parameters"] == 4 * p.H + 2
    for cfg, H, P in ((mi.cfg1, 1, 6), (mi.cfg2, 8, 28), (mi.cfg3, 4, 11)):
        q = cfg(nbins=64) if cfg is mi.cfg1 else cfg(nbins=64, nhist=H)
        assert q.nparams == P
        used = set(int(v) for v in q.map.ravel() if v >= 0)
        assert used == set(range(P))
    q = mi.cfg5(nhist=64, nbins=64)
    assert q.nparams == 197
    assert set(int(v) for v in q.map.ravel() if v >= 0) == set(range(197))


# ------------------------------------------------------------------------------------------
# Gauss-Newton matrix (error estimates)
# ------------------------------------------------------------------------------------------

def test_gauss_newton_equals_hessian_when_data_equal_model():
    """Where the data equal the model, d cost/dN = 0 in every bin, so the Gauss-Newton matrix
    is the exact Hessian: it matches central differences of the analytic gradient.  Catches a
    wrong weight (d^2 cost/dN^2) or a wrong Jacobian."""
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))], [("AMP", (6,)), ("KT", (7,))],
             [("AMP", (8,)), ("GAUSS", (9,))]]
    x10 = np.array([250.0, 3.0, 0.2, 0.4, 3.0, 20.0, 0.1, 0.5, 0.08, 0.7])
    # second map: one parameter in two slots of the row (the first and third amplitudes, the
    # exponential rate and the Gaussian width), whose Jacobian entries must add
    for mp, x in (([[0, 1, 2, 3, 4, 5, 6, 7, 8, 9]], x10), ([[0, 1, 2, 3, 4, 5, 6, 7, 2, 3]], x10[:8])):
        p = _problem(np.zeros((1, 700)), terms, mp, len(x), bin_width_ns=10.0, fit=(0.0, 6.0))
        dt = p.bin_width_ns / 1000.0
        p = p.with_counts(np.array([[oracle.model(p, x, 0, n * dt) for n in range(700)]]))
        for mode in (CHI2, MLE):
            gn = oracle.gauss_newton(p, x, mode)
            h = oracle.hessian(p, x, mode, steps=1e-6 * np.maximum(np.abs(x), 1e-2))
            scale = np.sqrt(np.outer(np.diag(gn), np.diag(gn)))
            assert np.all(np.abs(gn - h) <= 1e-6 * scale + 1e-9), np.max(np.abs(gn - h) / scale)
            assert np.allclose(gn, gn.T, rtol=1e-14, atol=0)
            assert np.linalg.eigvalsh(gn).min() > -1e-9 * np.abs(gn).max()


def test_gauss_newton_of_constant_model_closed_form():
    """N = c on any data: sum 2/max(d,1) for chi^2 and sum 2d/c^2 for -2lnL (the model is
    linear in c, so this is also the exact second derivative)."""
    rng = np.random.default_rng(11)
    d = rng.poisson(3.0, size=(2, 500)).astype(float)
    p = Problem(d, np.zeros(2), 0.5, (0.0, 1e9), [], np.array([[-1, 0], [-1, 0]], np.int32), np.array([0.0]), 1,
                np.zeros(1), ["c"])
    c = 2.75
    assert oracle.gauss_newton(p, np.array([c]), CHI2)[0, 0] == pytest.approx(
        np.sum(2.0 / np.maximum(d, 1.0)), rel=1e-14)
    assert oracle.gauss_newton(p, np.array([c]), MLE)[0, 0] == pytest.approx(np.sum(2.0 * d / c**2), rel=1e-14)


# ------------------------------------------------------------------------------------------
# Asymmetry data: forward / backward pairs, a = (f - alpha b) / (f + alpha b)
# ------------------------------------------------------------------------------------------

def _asym(F, Bk, alpha, bkg_f, bkg_b, terms, mp, nparams, consts=(), bin_width_ns=1.0, fit=(0.0, 1e9)):
    from musr_inputs import AsymmetryProblem
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    Bk = np.atleast_2d(np.asarray(Bk, dtype=np.float64))
    H = F.shape[0]
    return AsymmetryProblem(F, Bk, np.asarray(alpha, float).reshape(H), np.asarray(bkg_f, float).reshape(H),
                            np.asarray(bkg_b, float).reshape(H), np.zeros(H), bin_width_ns, fit, terms,
                            np.atleast_2d(np.asarray(mp, np.int32)), np.asarray(consts, dtype=np.float64), nparams,
                            np.zeros(nparams), [f"p{i}" for i in range(nparams)])


def test_asymmetry_of_an_exact_pair():
    """A pair built from an asymmetry T (F = K (1 + T) + bkg_F, B = K (1 - T) / alpha + bkg_B)
    gives a = T to rounding: the backgrounds are subtracted and alpha scales the backward
    count.  A bin without signal (f + alpha b <= 0) gets weight 0.  Catches alpha on the
    wrong count, a sign flip and a background not subtracted."""
    rng = np.random.default_rng(3)
    T = rng.uniform(-0.6, 0.6, size=(2, 500))
    K = rng.uniform(50.0, 5000.0, size=(2, 500))
    alpha, bf, bb = np.array([1.3, 0.8]), np.array([4.0, 0.5]), np.array([2.5, 7.0])
    F = K * (1.0 + T) + bf[:, None]
    Bk = K * (1.0 - T) / alpha[:, None] + bb[:, None]
    a, w = oracle.asymmetry(F, Bk, alpha, bf, bb)
    assert np.max(np.abs(a - T)) < 1e-13
    assert np.all(w > 0.0)
    a0, w0 = oracle.asymmetry(np.array([[4.0, 3.0]]), np.array([[2.5, 1.0]]), [1.3], [4.0], [2.5])
    assert w0[0, 0] == 0.0 and w0[0, 1] == 0.0


def test_asymmetry_weight_is_the_inverse_poisson_variance():
    """1/w at the expected counts equals the variance of the asymmetry over Poisson draws of
    the pair (first-order error propagation; at these counts the higher orders are below
    0.1 %).  Catches a dropped factor 4 or alpha^2, the forward and backward variances
    exchanged, and background-subtracted counts used as the variances."""
    rng = np.random.default_rng(11)
    for lf, lb, al, bf, bb in ((9000.0, 4000.0, 1.3, 300.0, 150.0), (2500.0, 6000.0, 0.7, 0.0, 900.0)):
        n = 400000
        Fs = rng.poisson(lf, n).astype(np.float64)[None, :]
        Bs = rng.poisson(lb, n).astype(np.float64)[None, :]
        a, _ = oracle.asymmetry(Fs, Bs, [al], [bf], [bb])
        _, w = oracle.asymmetry(np.array([[lf]]), np.array([[lb]]), [al], [bf], [bb])
        assert np.var(a) * w[0, 0] == pytest.approx(1.0, abs=0.015), (lf, lb, np.var(a) * w[0, 0])


def test_asymmetry_constant_data_and_baseline_optimum():
    """Constant asymmetry data are fitted exactly by a constant amplitude with scale 1 and
    baseline 0 (chi^2 = 0 at amplitude = the data value), which only holds when the model of
    asymmetry data carries no decay envelope; with a baseline alone the optimum is the
    weighted mean sum(w a) / sum(w).  -2lnL is refused for asymmetry data (status 2)."""
    rng = np.random.default_rng(13)
    K = rng.uniform(200.0, 900.0, size=(2, 600))
    al = np.array([1.1, 0.9])
    F = K * 1.3
    Bk = K * 0.7 / al[:, None]
    p = _asym(F, Bk, al, [0.0, 0.0], [0.0, 0.0], [[("AMP", (2,))]], [[-1, -2, 0], [-1, -2, 0]], 1,
              consts=(1.0, 0.0), bin_width_ns=20.0)
    r = oracle.fit(p, np.array([0.1]), CHI2)
    assert r["status"] == 0 and r["x"][0] == pytest.approx(0.3, abs=1e-10) and r["f"] < 1e-18
    assert oracle.cost(p, np.array([0.3]), MLE)[3] == 2
    Fn = rng.poisson(500.0, size=(2, 800)).astype(float)
    Bn = rng.poisson(450.0, size=(2, 800)).astype(float)
    q = _asym(Fn, Bn, al, [3.0, 1.0], [2.0, 4.0], [], [[-1, 0], [-1, 0]], 1, consts=(1.0,), bin_width_ns=20.0)
    a, w = oracle.asymmetry(Fn, Bn, al, [3.0, 1.0], [2.0, 4.0])
    r = oracle.fit(q, np.array([0.0]), CHI2)
    assert r["status"] == 0 and r["x"][0] == pytest.approx(np.sum(w * a) / np.sum(w), rel=1e-9)


def test_asymmetry_gradient_matches_complex_step():
    """The analytic gradient of the asymmetry chi^2 equals the complex-step derivative, with
    the scale and the baseline fitted too.  Catches the envelope left in the slot
    derivatives and a weight missing from the gradient."""
    import musr_inputs as mi
    p = mi.asym_tf(npairs=2, nbins=500, bin_width_ns=16.0, seed=27, n0=300.0)
    terms = [[("AMP", (2,)), ("GAUSS", (3,)), ("TFCOS", (4, 5))], [("AMP", (6,)), ("EXP", (7,))]]
    rows = [[0, 1, 2, 3, 4, 5, 6, 7], [0, 1, 2, 3, 4, 8, 6, 7]]
    import dataclasses
    q = dataclasses.replace(p, terms=terms, map=np.array(rows, np.int32), consts=np.zeros(0), nparams=9,
                            truth=np.zeros(9), names=[f"p{i}" for i in range(9)])
    x = np.array([0.95, 0.01, 0.2, 0.45, 3.05, 21.0, 0.04, 0.3, 108.0])
    v, g, gs, st = oracle.cost(q, x, CHI2)
    assert st == 0 and v > 0
    for i in range(q.nparams):
        e = np.zeros(q.nparams)
        e[i] = 1.0
        cs = oracle.cost_cstep(q, x, e, CHI2)
        assert abs(cs - g[i]) <= 1e-11 * gs[i] + 1e-300, (i, cs, g[i], gs[i])


def test_asymmetry_gauss_newton_equals_hessian_when_data_equal_model():
    """Pairs built from the asymmetry model itself: there the Gauss-Newton matrix (weight 2 w)
    is the exact Hessian of the chi^2, which central differences of the gradient measure."""
    import dataclasses
    import musr_inputs as mi
    p = mi.asym_tf(npairs=2, nbins=300, bin_width_ns=25.0, seed=28, n0=300.0)
    t = (np.arange(p.B) - p.t0[0]) * p.bin_width_ns / 1000.0
    T = np.array([[oracle.model(p, p.truth, h, tt) for tt in t] for h in range(p.H)])
    K = 800.0
    F = K * (1.0 + T) + p.bkg_f[:, None]
    Bk = K * (1.0 - T) / p.alpha[:, None] + p.bkg_b[:, None]
    q = dataclasses.replace(p, forward=F, backward=Bk)
    assert oracle.cost(q, p.truth, CHI2)[0] < 1e-20
    Hg = oracle.gauss_newton(q, p.truth, CHI2)
    Hc = oracle.hessian(q, p.truth, CHI2)
    scale = np.sqrt(np.outer(np.diag(Hg), np.diag(Hg)))
    assert np.max(np.abs(Hg - Hc) / scale) < 1e-6


# ------------------------------------------------------------------------------------------
# Stretched exponential and Bessel precession
# ------------------------------------------------------------------------------------------

def test_stretched_exponential_special_cases():
    """exp(-(lambda t)^beta) is EXP at beta = 1 and GAUSS with sigma = sqrt(2) lambda at
    beta = 2; 1 at and before time zero; even in lambda.  Catches a missing exponent, a
    rate inside the power taken as lambda^beta t, and a wrong branch at t <= 0."""
    for lam in (0.2, 0.9, 3.0):
        for t in (0.05, 0.7, 4.0):
            assert oracle.primitive("STREXP", lam, 1.0, t) == pytest.approx(oracle.primitive("EXP", lam, 0.0, t),
                                                                            rel=1e-14)
            assert oracle.primitive("STREXP", lam, 2.0, t) == pytest.approx(
                oracle.primitive("GAUSS", math.sqrt(2.0) * lam, 0.0, t), rel=1e-13)
            assert oracle.primitive("STREXP", -lam, 0.6, t) == oracle.primitive("STREXP", lam, 0.6, t)
        assert oracle.primitive("STREXP", lam, 0.5, 0.0) == 1.0
        assert oracle.primitive("STREXP", lam, 0.5, -1.0) == 1.0
    # exp(-(lambda t)^beta) = 1/e at t = 1/lambda for every beta
    for beta in (0.3, 0.5, 1.7):
        assert oracle.primitive("STREXP", 0.4, beta, 2.5) == pytest.approx(math.exp(-1.0), rel=1e-14)


def test_bessel_precession_against_a_library_j0():
    """BESSEL(nu, phi) = J0(2 pi (nu t + phi / 360)) against scipy's J0, including the first zero
    2.404825557695773 and large arguments.  Catches a missing 2 pi, a phase in radians and
    a J1 in place of J0."""
    from scipy.special import j0
    rng = np.random.default_rng(17)
    for _ in range(400):
        nu, phi, t = rng.uniform(0.0, 30.0), rng.uniform(-360.0, 360.0), rng.uniform(-2.0, 12.0)
        x = 2.0 * math.pi * (nu * t + phi / 360.0)
        assert abs(oracle.primitive("BESSEL", nu, phi, t) - j0(x)) < 1e-12  # two libraries, arguments to ~2000
    assert oracle.primitive("BESSEL", 3.0, 0.0, 0.0) == 1.0
    assert abs(oracle.primitive("BESSEL", 2.404825557695773 / (2.0 * math.pi), 0.0, 1.0)) < 1e-15


def _new_primitive_problem(mode_seed=0):
    import musr_inputs as mi
    p = mi.cfg3(nhist=2, nbins=400, bin_width_ns=25.0, seed=29)
    terms = [[("AMP", (2,)), ("STREXP", (3, 4))], [("AMP", (5,)), ("BESSEL", (6, 7)), ("EXP", (8,))]]
    rows = [[0, 1, 2, 3, 4, 5, 6, 7, 8], [9, 10, 2, 3, 4, 5, 6, 11, 8]]
    x = np.array([300.0, 2.0, 0.12, 0.7, 0.55, 0.1, 1.3, 25.0, 0.2, 310.0, 2.5, -40.0])
    q = Problem(p.counts, p.t0, p.bin_width_ns, p.fit_range_us, terms, np.array(rows, np.int32), np.zeros(0), 12,
                np.zeros(12), [f"p{i}" for i in range(12)])
    return q, x


@pytest.mark.parametrize("mode", [CHI2, MLE])
def test_gradient_matches_complex_step_new_primitives(mode):
    """Complex-step derivative of a theory with a stretched exponential and a Bessel term
    (the chain factors 2 pi t, 2 pi / 360, beta (lambda t)^beta / lambda, ln(lambda t))."""
    q, x = _new_primitive_problem()
    v, g, gs, st = oracle.cost(q, x, mode)
    assert st == 0
    for i in range(q.nparams):
        e = np.zeros(q.nparams)
        e[i] = 1.0
        cs = oracle.cost_cstep(q, x, e, mode)
        assert abs(cs - g[i]) <= 1e-11 * gs[i] + 1e-300, (i, cs, g[i], gs[i])


def test_gradient_of_new_primitives_matches_central_differences():
    """Central differences of the value (no derivative formula involved): pins J0' = -J1 and
    the exponent derivative of the stretched exponential."""
    q, x = _new_primitive_problem()
    for mode in (CHI2, MLE):
        _, g, gs, _ = oracle.cost(q, x, mode)
        for i in range(q.nparams):
            h = 1e-6 * max(abs(x[i]), 1e-3)
            xp, xm = x.copy(), x.copy()
            xp[i] += h
            xm[i] -= h
            fd = (oracle.cost(q, xp, mode, grad=False)[0] - oracle.cost(q, xm, mode, grad=False)[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * gs[i], (i, fd, g[i])


# ------------------------------------------------------------------------------------------
# Dynamic Gaussian Kubo-Toyabe relaxation (strong collisions): the renewal equation
# G = f + nu f * G, f = g exp(-nu t), g the static function, solved on a grid by the oracle
# ------------------------------------------------------------------------------------------

def _static_kt(D, t):
    """The textbook static Gaussian Kubo-Toyabe function (the test's own statement of g)."""
    u = (D * t) ** 2
    return 1.0 / 3.0 + 2.0 / 3.0 * (1.0 - u) * math.exp(-0.5 * u)


def test_dkt_without_fluctuations_is_the_static_function():
    """nu = 0: no renewals, so G is the static function: G(0) = 1 and the minimum
    1/3 - (4/3) e^{-3/2} at t = sqrt(3) / Delta (catches a solver that drops f's first
    term or misplaces the grid)."""
    D = 0.7
    tmin = math.sqrt(3.0) / D
    G = oracle.dkt(D, 0.0, 6.0, [0.0, tmin, 1.0, 5.9])
    assert G[0] == 1.0
    assert abs(G[1] - (1.0 / 3.0 - 4.0 / 3.0 * math.exp(-1.5))) < 1e-11
    assert abs(G[2] - _static_kt(D, 1.0)) < 1e-11 and abs(G[3] - _static_kt(D, 5.9)) < 1e-11
    assert oracle.dkt(D, 0.9, 6.0, [0.0])[0] == 1.0
    assert oracle.primitive("DKT", D, 0.9, -1.0) == 1.0  # the relaxation starts at time zero


def test_dkt_laplace_transform_of_the_renewal_equation():
    """The Laplace transform of G = f + nu f * G is L[G](s) = F(s) / (1 - nu F(s)) with
    F(s) = L[g](s + nu): F by adaptive quadrature of the static function, L[G] by Simpson's
    rule on the oracle's G.  Catches a wrong trapezoidal weight, sign, rate or Richardson
    step in the solver (each moves L[G] by far more than 1e-10)."""
    from scipy.integrate import quad
    D, nu, span = 0.6, 0.9, 16.0
    ts = np.linspace(0.0, span, 16001)
    G = oracle.dkt(D, nu, span, ts)
    hs = ts[1] - ts[0]
    for s in (2.0, 3.5):
        y = G * np.exp(-s * ts)
        lhs = hs / 3.0 * (y[0] + y[-1] + 4.0 * y[1:-1:2].sum() + 2.0 * y[2:-1:2].sum())
        F = quad(lambda t: _static_kt(D, t) * math.exp(-(s + nu) * t), 0.0, 60.0, limit=400, epsabs=1e-15,
                 epsrel=1e-13)[0]
        rhs = F / (1.0 - nu * F)
        assert abs(lhs / rhs - 1.0) < 1e-10, (s, lhs, rhs)


def test_dkt_motional_narrowing():
    """Fast fluctuations (nu >> Delta) narrow the relaxation to exp(-2 Delta^2 t / nu): the
    log-slope of G at late times is 2 Delta^2 / nu to second order in Delta / nu."""
    for D, nu in ((0.1, 5.0), (0.2, 5.0)):
        G = oracle.dkt(D, nu, 8.0, [4.0, 8.0])
        lam = -math.log(G[1] / G[0]) / 4.0
        assert abs(lam / (2.0 * D * D / nu) - 1.0) <= 2.0 * (D / nu) ** 2, (D, nu, lam)


def test_dkt_grid_refinement():
    """Grids over different spans (other spacings and nodes) give the same relaxation."""
    ts = np.linspace(0.3, 7.9, 50)
    a = oracle.dkt(0.6, 0.9, 8.0, ts)
    b = oracle.dkt(0.6, 0.9, 9.3, ts)
    assert np.max(np.abs(a - b)) < 1e-10


def test_dkt_derivatives_central_differences():
    """The derivative recursions against central differences of the value (no derivative
    formula involved); parameters away from a change of the grid's size."""
    D, nu, span = 0.4137, 0.8123, 8.0
    ts = np.linspace(0.2, 7.8, 30)
    G, dD, dn = oracle.dkt(D, nu, span, ts, derivs=True)
    e = 1e-6
    fdD = (oracle.dkt(D + e, nu, span, ts) - oracle.dkt(D - e, nu, span, ts)) / (2 * e)
    fdn = (oracle.dkt(D, nu + e, span, ts) - oracle.dkt(D, nu - e, span, ts)) / (2 * e)
    assert np.max(np.abs(fdD - dD)) < 1e-8 and np.max(np.abs(fdn - dn)) < 1e-8


def _dkt_problem():
    import musr_inputs as mi
    p = mi.cfg3(nhist=2, nbins=300, bin_width_ns=25.0, seed=31)
    terms = [[("AMP", (2,)), ("DKT", (3, 4))], [("AMP", (5,)), ("EXP", (6,))]]
    rows = [[0, 1, 2, 3, 4, 5, 6], [7, 8, 2, 3, 4, 5, 6]]
    x = np.array([300.0, 2.0, 0.2, 0.45, 0.7, 0.05, 0.3, 310.0, 2.5])
    q = Problem(p.counts, p.t0, p.bin_width_ns, p.fit_range_us, terms, np.array(rows, np.int32), np.zeros(0), 9,
                np.zeros(9), [f"p{i}" for i in range(9)])
    return q, x


@pytest.mark.parametrize("mode", [CHI2, MLE])
def test_gradient_matches_complex_step_dynamic_kt(mode):
    """Complex step through the whole cost, the renewal equation solved in complex
    arithmetic: pins the derivative recursions and their scatter to Delta and nu."""
    q, x = _dkt_problem()
    v, g, gs, st = oracle.cost(q, x, mode)
    assert st == 0
    for i in range(q.nparams):
        e = np.zeros(q.nparams)
        e[i] = 1.0
        cs = oracle.cost_cstep(q, x, e, mode)
        assert abs(cs - g[i]) <= 1e-10 * gs[i] + 1e-300, (i, cs, g[i], gs[i])


# ------------------------------------------------------------------------------------------
# The particle-mesh Poisson solve (Section 3, Eq. openbruteforceconv), the second workload
# ------------------------------------------------------------------------------------------

def test_poisson_point_charge():
    """One charge q at a mesh point: phi = hx hy hz q / r at every other point (anisotropic
    spacing) and hx hy hz q / min(h) at the charge (the reading of the singular self term).
    Catches transposed spacings, a missing volume factor and an offset of the source."""
    h = (0.5, 0.7, 1.1)
    rho = np.zeros((7, 6, 5))
    rho[2, 4, 1] = 3.0
    phi = oracle.poisson_direct(rho, h)
    V = h[0] * h[1] * h[2]
    i, j, k = np.meshgrid(np.arange(7), np.arange(6), np.arange(5), indexing="ij")
    r = np.sqrt(((i - 2) * h[0]) ** 2 + ((j - 4) * h[1]) ** 2 + ((k - 1) * h[2]) ** 2)
    far = r > 0
    assert np.max(np.abs(phi[far] * r[far] / (V * 3.0) - 1.0)) < 1e-14
    assert phi[2, 4, 1] == pytest.approx(V * 3.0 / 0.5, rel=1e-15)


def test_poisson_direct_sum_equals_fft_convolution():
    """The direct sum equals the linear convolution computed by numpy's FFT on the doubled,
    zero-padded mesh (an independent algorithm for the same sum)."""
    rng = np.random.default_rng(19)
    h = (0.3, 0.45, 0.2)
    rho = rng.normal(size=(9, 7, 6))
    phi = oracle.poisson_direct(rho, h)
    M = rho.shape
    N = tuple(2 * m for m in M)
    a, b, c = np.meshgrid(*[np.minimum(np.arange(n), n - np.arange(n)) for n in N], indexing="ij")
    G = 1.0 / np.sqrt((a * h[0]) ** 2 + (b * h[1]) ** 2 + (c * h[2]) ** 2 + (a + b + c == 0))
    G[0, 0, 0] = 1.0 / min(h)
    ax = (0, 1, 2)
    conv = np.fft.irfftn(np.fft.rfftn(rho, N, axes=ax) * np.fft.rfftn(G, axes=ax), N, axes=ax)[: M[0], : M[1], : M[2]]
    ref = h[0] * h[1] * h[2] * conv
    assert np.max(np.abs(phi - ref)) < 1e-12 * np.max(np.abs(ref))


def test_poisson_far_field_is_the_monopole():
    """Far from a compact, symmetric charge the potential is that of its total charge,
    hx hy hz Q / r, to the order (size / r)^4 (the dipole and quadrupole vanish)."""
    h = (1.0, 1.0, 1.0)
    rho = np.zeros((26, 26, 26))
    rho[11:14, 11:14, 11:14] = 1.0
    rho[12, 12, 12] = 5.0
    Q = rho.sum()
    ijk = np.array([[0, 0, 0], [25, 12, 12], [12, 0, 25], [25, 25, 0]])
    phi = oracle.poisson_points(rho, h, ijk)
    r = np.sqrt(((ijk - 12) ** 2).sum(axis=1))
    assert np.max(np.abs(phi * r / Q - 1.0)) < 2e-3
