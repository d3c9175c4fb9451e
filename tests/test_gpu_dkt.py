"""Dynamic Gaussian Kubo-Toyabe relaxation (strong collisions) on the GPU against the oracle.

The device solves the renewal equation G = f + nu f * G once per evaluation and (Delta, nu)
pair on its own grid (trapezoidal rule with Richardson extrapolation, spacing times the faster
of Delta and nu at most 0.02 for FP64 tables and 0.03 for the FP32 tables of the SPLIT path) and interpolates it per bin with the cubic through the four
nearest grid points (at SPLIT precision as a basis function of its term where the term allows
one, else within the per-bin term list); the oracle solves it on a five times finer grid.  Tolerance: the
table's error eps_T -- discretisation O((h rate)^4), interpolation 0.023 h^4 |G''''|, and
for the FP32 tables of the SPLIT path the rounding of sums of up to 2K terms -- stays below
3e-6 of G's range (1) for these parameters (a model of the device's scheme run in numpy
against the oracle: 1e-8 .. 3e-7 for FP64 tables, 2e-7 .. 3e-6 for FP32 ones).  It enters
every bin's model and derivatives at most at that level relative to their scale, so:

  * value:    |dv| <= tol_path |v| + 1e-5 * sum_h gscale[Nbkg_h] * N0_h |A|max
              (sum |dcost/dN| over a histogram is the gradient scale of its background);
  * gradient: |dg_i| <= (tol_path + 1e-5) * gscale_i,

with tol_path = 1e-12 (FP64 path) or 2^-16 (SPLIT path, FP32 arithmetic).
"""
import dataclasses

import numpy as np
import pytest

import musr_inputs as mi
import oracle
from musr_inputs import Problem

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SPLIT_EPS = 2.0 ** -16
EPS_T = 1e-5


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _mixed_problem(seed=41):
    """3 detectors with fractional time zeros; A = A0 DKT(Delta, nu) exp(-lambda t) + A1 cos(...)."""
    p = mi.cfg3(nhist=3, nbins=1200, bin_width_ns=10.0, seed=seed)
    terms = [[("AMP", (2,)), ("DKT", (3, 4)), ("EXP", (5,))], [("AMP", (6,)), ("TFCOS", (7, 8))]]
    rows = [[9 + 2 * j, 10 + 2 * j, 0, 1, 2, 3, 4, 5, 6 + j] for j in range(3)]
    names = ["A0", "Delta", "nu", "lambda", "A1", "nu_tf", "phi_0", "phi_1", "phi_2"]
    truth = [0.2, 0.45, 0.7, 0.05, 0.08, 1.3, 10.0, 50.0, 90.0]
    for j in range(3):
        names += [f"N0_{j}", f"Nbkg_{j}"]
        truth += [300.0 + 10 * j, 2.0]
    q = Problem(p.counts, np.array([0.3, 1.7, 2.25]), p.bin_width_ns, (0.05, 11.9), terms,
                np.array(rows, np.int32), np.zeros(0), len(truth), np.array(truth), names, "dkt_mixed")
    return q


def _list_problem(seed=45):
    """The dynamic KT factor beside a cosine in one term (no basis form: the SPLIT path
    evaluates the term list per bin)."""
    p = mi.cfg3(nhist=2, nbins=1200, bin_width_ns=10.0, seed=seed)
    terms = [[("AMP", (2,)), ("DKT", (3, 4)), ("TFCOS", (5, 6))]]
    rows = [[5 + 2 * j, 6 + 2 * j, 0, 1, 2, 3, 4] for j in range(2)]
    truth = [0.2, 0.4, 0.9, 2.0, 30.0]
    names = ["A0", "Delta", "nu", "nu_tf", "phi"]
    for j in range(2):
        names += [f"N0_{j}", f"Nbkg_{j}"]
        truth += [300.0, 2.0]
    return Problem(p.counts, np.array([0.0, 0.0]), p.bin_width_ns, (0.05, 11.9), terms, np.array(rows, np.int32),
                   np.zeros(0), len(truth), np.array(truth), names, "dkt_list")


def _problems():
    return {"dkt_zf": mi.dkt_zf(nhist=2, nbins=1600, bin_width_ns=8.0, seed=20),
            "mixed": _mixed_problem(),
            "fast": mi.dkt_zf(nhist=2, nbins=1600, bin_width_ns=8.0, seed=21, delta=0.15, nu_c=4.0),
            "list": _list_problem()}


PROBLEMS = None


def problems():
    global PROBLEMS
    if PROBLEMS is None:
        PROBLEMS = _problems()
    return PROBLEMS


def _value_slack(p, x, gs):
    """1e-5 x sum over histograms of gscale[Nbkg_h] N0_h |A|max (|A| <= sum of the amplitudes)."""
    amp = sum(abs(x[i]) for i, n in enumerate(p.names) if n.startswith("A"))
    s = 0.0
    for h in range(p.H):
        s += gs[p.map[h][1]] * abs(x[p.map[h][0]]) * amp
    return EPS_T * s


def _check(p, x, v, g, ref, tol):
    rv, rg, rgs, _ = ref
    assert abs(v - rv) <= tol * abs(rv) + _value_slack(p, x, rgs), (v, rv, (v - rv) / rv)
    bad = np.abs(g - rg) > (tol + EPS_T) * rgs + 1e-300
    assert not bad.any(), (np.nonzero(bad), g[bad], rg[bad], rgs[bad])


@pytest.mark.parametrize("name", ["dkt_zf", "mixed", "fast", "list"])
def test_dynamic_kt_matches_oracle(B, name):
    p = problems()[name]
    X = mi.jitter(p.truth, 3, seed=5, lo=0.95, hi=1.05)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            refs = [oracle.cost(p, x, mode) for x in X]
            for prec, tol in ((B.MUSR_FP64, FP64_TOL), (B.MUSR_SPLIT, SPLIT_EPS)):
                v, g, st = ctx.eval(X[0], mode, prec)
                assert st == 0
                _check(p, X[0], v, g, refs[0], tol)
                vals, grads, st = ctx.eval_batch(X, mode, prec)  # one table per vector
                assert st == 0
                for k in range(len(X)):
                    _check(p, X[k], vals[k], grads[k], refs[k], tol)
                vals2, grads2, _ = ctx.eval_batch(X, mode, prec)
                assert np.array_equal(vals, vals2) and np.array_equal(grads, grads2)


def test_dynamic_kt_without_fluctuations_is_the_static_kt(B):
    """nu = 0: no renewals, the relaxation is the static Kubo-Toyabe function, a closed form
    the kernels evaluate directly: the two theories' costs and gradients agree (FP64) to the
    table's interpolation error (cubic on a grid of spacing 0.02 / Delta: 0.023 h^4 times the
    fourth derivative, a few 1e-9 of the cost here)."""
    p = mi.cfg3(nhist=2, nbins=1500, bin_width_ns=8.0, seed=42)
    dkt = dataclasses.replace(p, terms=[[("AMP", (2,)), ("DKT", (3, 5)), ("EXP", (4,))]],
                              map=np.hstack([p.map, np.full((p.H, 1), -1, np.int32)]), consts=np.array([0.0]))
    x = p.truth * 1.02
    with B.Context(p) as c1, B.Context(dkt) as c2:
        for mode in (0, 1):
            v1, g1, _ = c1.eval(x, mode, B.MUSR_FP64)
            v2, g2, _ = c2.eval(x, mode, B.MUSR_FP64)
            gs = oracle.cost(p, x, mode)[2]
            assert abs(v1 - v2) <= 1e-7 * abs(v1), (v1, v2)
            assert np.all(np.abs(g1 - g2) <= 1e-5 * gs)


def test_dynamic_kt_fits(B):
    """Fits of the Monte Carlo of fluctuating fields: the SPLIT fit within 0.01 sigma of the
    FP64 fit, the FP64 fit within 0.01 sigma of the oracle's."""
    from paper_1509_07685_gb300 import fit as F
    p = mi.dkt_zf(nhist=2, nbins=1600, bin_width_ns=8.0, seed=43)
    x0 = mi.start_point(p, 3)
    ro = oracle.fit(p, x0, 1)
    assert ro["status"] == 0
    sig = oracle.sigmas(p, ro["x"], 1)
    with B.Context(p) as ctx:
        r64 = F.fit_context(ctx, x0, 1, B.MUSR_FP64)
        r32 = F.fit_context(ctx, x0, 1, B.MUSR_SPLIT)
    assert np.max(np.abs(r64["x"] - ro["x"]) / sig) < 0.01, np.abs(r64["x"] - ro["x"]) / sig
    assert np.max(np.abs(r32["x"] - r64["x"]) / sig) < 0.01, np.abs(r32["x"] - r64["x"]) / sig


@pytest.mark.parametrize("name", ["mixed", "dkt_zf"])
def test_dynamic_kt_gauss_newton(B, name):
    """Gauss-Newton matrices of theories with the dynamic KT factor in their basis form: FP64
    and SPLIT against the oracle, within the tables' accuracy (and 2^-16 for SPLIT)."""
    p = problems()[name]
    x = p.truth * 1.01
    with B.Context(p) as ctx:
        for mode in (0, 1):
            R = oracle.gauss_newton(p, x, mode)
            scale = np.sqrt(np.outer(np.diag(R), np.diag(R)))
            for prec, tol in ((B.MUSR_FP64, EPS_T), (B.MUSR_SPLIT, EPS_T + SPLIT_EPS)):
                H = ctx.gauss_newton(x, mode, prec)
                assert np.all(np.abs(H - R) <= tol * scale + 1e-300), (prec, np.max(np.abs(H - R) / scale))


def test_dynamic_kt_refused_where_no_tables_are_solved(B):
    """Served fits and the allocation-free entry point have no room for per-evaluation
    tables: both refuse the primitive with a reason."""
    import torch
    p = mi.dkt_zf(nhist=1, nbins=400, bin_width_ns=20.0, seed=44)
    with B.Server(hbm_budget_bytes=1 << 28, max_active=4) as srv:
        with pytest.raises(B.MusrError):
            srv.submit(p, p.truth, 1, B.MUSR_FP64)
    d_counts = torch.zeros((p.H, 400), dtype=torch.float32, device="cuda")
    d_x = torch.tensor(p.truth, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(1 + p.nparams, dtype=torch.float64, device="cuda")
    st = B.musr_eval_noalloc(d_counts.data_ptr(), B.MUSR_DTYPE_FP32, p.H, p.B, 400, p.t0, p.bin_width_ns,
                             p.fit_range_us, p.terms, p.map, p.nparams, p.consts, d_x.data_ptr(), 0,
                             B.MUSR_FP64, True, d_out.data_ptr(), None)
    assert st == B.MUSR_EINVAL and "Kubo-Toyabe" in B.musr_last_error(None)


def test_context_releases_its_evaluation_buffers(B):
    """A context gives back every device buffer it allocated, the per-evaluation tables of the
    dynamic KT factor, their solve's scratch and counters and the Gauss-Newton directions
    included: contexts made, used and destroyed in turn leave the device's free memory where
    it was."""
    import torch
    p = problems()["mixed"]
    X = mi.jitter(p.truth, 32, seed=7, lo=0.98, hi=1.02)

    def cycle():
        with B.Context(p) as ctx:
            for prec in (B.MUSR_FP64, B.MUSR_SPLIT):
                ctx.eval_batch(X, 1, prec)
                ctx.gauss_newton(X[0], 1, prec)
        torch.cuda.synchronize()

    cycle()  # first use: the library's own one-time allocations
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    # 32 vectors of FP64 table scratch alone are ~17 MB per cycle: nothing of that may stay
    assert free0 - free1 < 4 << 20, (free0, free1)
