"""GPU parity: libmusr (through its C ABI) against the FP64 CPU oracle.

Tolerances:
  * FP64 path: |dvalue| <= 1e-12 |value|; |dg_i| <= 1e-12 * sum_n |dterm_n/dtheta_i|
    (the gradient scale returned by the oracle; g_i -> 0 at the optimum makes a
    plain relative error ill-posed).
  * SPLIT path: per-bin FP32 evaluation with hardware ex2/lg2/rcp/sin/cos whose
    relative error is below 2^-20 (about 1e-6) per factor; a bin's model combines a
    handful of such factors, so every per-bin term and gradient term carries a
    relative error below SPLIT_EPS = 2^-16 (1.5e-5, a margin of ~16 over the factor
    error).  Summed terms are bounded by SPLIT_EPS times the sum of their absolute
    values: the value (all terms >= 0) to SPLIT_EPS relative, the gradient to
    SPLIT_EPS * gscale.  FP32 accumulation below the warp adds far less.
"""
import dataclasses

import numpy as np
import pytest

import musr_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SPLIT_EPS = 2.0 ** -16


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _problems():
    # Sizes the oracle finishes in seconds, spanning several tiles with ragged tails.
    return {
        "cfg1": mi.cfg1(nbins=16384 + 37, seed=10, dtype=np.int32),
        "cfg2": mi.cfg2(nhist=8, nbins=20000 + 13, bin_width_ns=0.64, seed=11),
        "cfg3": mi.cfg3(nhist=4, nbins=9000 + 3, bin_width_ns=1.4, seed=12),
        "cfg5": mi.cfg5(nhist=10, nbins=6000 + 5, seed=13, n0=20.0, nbkg=0.1),
        "paper_tf16": mi.paper_tf16(nhist=16, nbins=3000 + 1, seed=14, n0=100.0),
    }


PROBLEMS = None


def problems():
    global PROBLEMS
    if PROBLEMS is None:
        PROBLEMS = _problems()
    return PROBLEMS


def _check_fp64(v, g, ref):
    rv, rg, rgs, _ = ref
    assert abs(v - rv) <= FP64_TOL * abs(rv), (v, rv, (v - rv) / rv)
    bad = np.abs(g - rg) > FP64_TOL * rgs + 1e-300
    assert not bad.any(), (np.nonzero(bad), g[bad], rg[bad], rgs[bad])


def _check_split(v, g, ref):
    rv, rg, rgs, _ = ref
    assert abs(v - rv) <= SPLIT_EPS * abs(rv), (v, rv, (v - rv) / rv)
    bad = np.abs(g - rg) > SPLIT_EPS * rgs + 1e-300
    assert not bad.any(), (np.nonzero(bad), g[bad], rg[bad], rgs[bad])


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg3", "cfg5", "paper_tf16"])
@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_and_split_match_oracle(B, name, mode):
    p = problems()[name]
    rng = np.random.default_rng(100 + mode)
    with B.Context(p) as ctx:
        for trial in range(2):
            x = p.truth * rng.uniform(0.9, 1.1, p.nparams) if trial else mi.start_point(p, 3)
            ref = oracle.cost(p, x, mode)
            assert ref[3] == 0
            v, g, st = ctx.eval(x, mode, B.MUSR_FP64)
            assert st == 0
            _check_fp64(v, g, ref)
            v1, _, _ = ctx.eval(x, mode, B.MUSR_FP64, grad=False)
            assert v1 == v  # the value-only kernel sums in the same order
            v, g, st = ctx.eval(x, mode, B.MUSR_SPLIT)
            assert st == 0
            _check_split(v, g, ref)
            v2, _, _ = ctx.eval(x, mode, B.MUSR_SPLIT, grad=False)
            assert abs(v2 - v) <= 1e-12 * abs(v)


def test_batch_equals_single_and_is_deterministic(B):
    """A batch may use larger tiles than a single evaluation (so its sums run in another
    order): equal within the path's tolerance.  The same launch repeated is bit-identical."""
    p = problems()["cfg2"]
    X = mi.jitter(p.truth, 40, seed=3, lo=0.95, hi=1.05)
    with B.Context(p) as ctx:
        for prec, tol in ((B.MUSR_FP64, FP64_TOL), (B.MUSR_SPLIT, SPLIT_EPS)):
            vals, grads, st = ctx.eval_batch(X, 1, prec)
            assert st == 0
            for i in range(0, len(X), 7):
                v, g, _ = ctx.eval(X[i], 1, prec)
                gs = oracle.cost(p, X[i], 1)[2]
                assert abs(v - vals[i]) <= tol * abs(v)
                assert np.all(np.abs(g - grads[i]) <= tol * gs + 1e-300)
            vals2, grads2, _ = ctx.eval_batch(X, 1, prec)
            assert np.array_equal(vals, vals2) and np.array_equal(grads, grads2)


def test_repeated_evaluations_follow_every_change(B):
    """musr_eval_batch replays a recorded launch while nothing it refers to changes: new
    parameter values, another batch size, new histograms and a new map must each reach the
    kernels (every result against the oracle)."""
    p = mi.cfg3(nhist=3, nbins=3001, bin_width_ns=4.0, seed=91)
    q = mi.cfg3(nhist=3, nbins=3001, bin_width_ns=4.0, seed=92)
    X = mi.jitter(p.truth, 3, seed=9, lo=0.95, hi=1.05)
    with B.Context(p) as ctx:
        for prec, check in ((B.MUSR_SPLIT, _check_split), (B.MUSR_FP64, _check_fp64)):
            for k in range(3):  # the same launch with new parameter values
                v, g, _ = ctx.eval(X[k], 1, prec)
                check(v, g, oracle.cost(p, X[k], 1))
            for n in (2, 1, 3):  # other batch sizes, then back
                vals, grads, _ = ctx.eval_batch(X[:n], 1, prec)
                for k in range(n):
                    check(vals[k], grads[k], oracle.cost(p, X[k], 1))
        ctx.configure(q)  # new histograms (same theory and map)
        for prec, check in ((B.MUSR_SPLIT, _check_split), (B.MUSR_FP64, _check_fp64)):
            v, g, _ = ctx.eval(X[0], 1, prec)
            check(v, g, oracle.cost(q, X[0], 1))
        r = np.array(q.map)
        r[:, 1] = r[0, 1]  # one shared background: a new map
        q2 = dataclasses.replace(q, map=r)
        B.musr_set_map(ctx.ctx, q2.map, q2.nparams, q2.consts)
        for prec, check in ((B.MUSR_SPLIT, _check_split), (B.MUSR_FP64, _check_fp64)):
            v, g, _ = ctx.eval(X[0], 1, prec)
            check(v, g, oracle.cost(q2, X[0], 1))


def test_device_resident_eval(B):
    import torch
    p = problems()["cfg3"]
    X = mi.jitter(p.truth, 3, seed=5, lo=0.95, hi=1.05)
    stream = torch.cuda.current_stream().cuda_stream
    with B.Context(p, cuda_stream=stream) as ctx:
        d_x = torch.tensor(X, dtype=torch.float64, device="cuda")
        d_out = torch.empty((3, 1 + p.nparams), dtype=torch.float64, device="cuda")
        for prec in (B.MUSR_FP64, B.MUSR_SPLIT):
            B.musr_eval_device(ctx.ctx, d_x.data_ptr(), 3, 0, prec, True, d_out.data_ptr())
            torch.cuda.synchronize()
            out = d_out.cpu().numpy()
            vals, grads, _ = ctx.eval_batch(X, 0, prec)
            assert np.array_equal(out[:, 0], vals) and np.array_equal(out[:, 1:], grads)


def test_borrowed_device_histograms(B):
    import torch
    p = problems()["cfg2"]
    x = mi.start_point(p, 4)
    stride = (p.B + 3) // 4 * 4
    d = torch.zeros((p.H, stride), dtype=torch.float32, device="cuda")
    d[:, :p.B] = torch.from_numpy(np.ascontiguousarray(p.counts, dtype=np.float32)).cuda()
    ref = oracle.cost(p, x, 1)
    ctx = B.musr_ctx_create(0)
    try:
        B.musr_upload_histograms_device(ctx, d.data_ptr(), B.MUSR_DTYPE_FP32, p.H, p.B, stride, p.t0,
                                        p.bin_width_ns, p.fit_range_us)
        B.musr_set_theory(ctx, p.terms)
        B.musr_set_map(ctx, p.map, p.nparams, p.consts)
        v, g, st = B.musr_eval(ctx, x, 1, B.MUSR_FP64)
        _check_fp64(v, g, ref)
        v, g, st = B.musr_eval(ctx, x, 1, B.MUSR_SPLIT)
        _check_split(v, g, ref)
    finally:
        B.musr_ctx_destroy(ctx)


# ------------------------------------------------------------------------------------------
# Edge cases
# ------------------------------------------------------------------------------------------

def test_data_equal_model_fp64_counts_give_zero(B):
    """FP64 counts equal to the model (computed by the oracle) give chi^2 = -2lnL = 0."""
    base = mi.cfg3(nhist=2, nbins=1500, bin_width_ns=8.0, seed=1)
    x = base.truth.copy()
    dt = base.bin_width_ns / 1000.0
    d = np.array([[oracle.model(base, x, h, n * dt) for n in range(base.B)] for h in range(base.H)])
    p = base.with_counts(d)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            v, g, st = ctx.eval(x, mode, B.MUSR_FP64)
            assert st == 0 and abs(v) < 1e-9
            v, g, st = ctx.eval(x, mode, B.MUSR_SPLIT)
            ref_scale = oracle.cost(p, x * 1.01, mode)[0]
            assert st == 0 and abs(v) <= SPLIT_EPS * ref_scale


def test_empty_fit_range_and_single_bin(B):
    p = mi.cfg1(nbins=4096, seed=2, dtype=np.float32)
    x = p.truth
    q = mi.Problem(p.counts, p.t0, p.bin_width_ns, (100.0, 200.0), p.terms, p.map, p.consts, p.nparams,
                   p.truth, p.names)
    with B.Context(q) as ctx:
        assert ctx.bins_in_fit() == 0
        for prec in (0, 1):
            v, g, st = ctx.eval(x, 0, prec)
            assert st == 0 and v == 0.0 and not g.any()
    dt = p.bin_width_ns / 1000.0
    q = mi.Problem(p.counts, p.t0, p.bin_width_ns, (1001 * dt, 1001 * dt), p.terms, p.map, p.consts,
                   p.nparams, p.truth, p.names)
    ref = oracle.cost(q, x, 1)
    with B.Context(q) as ctx:
        assert ctx.bins_in_fit() == 1
        v, g, st = ctx.eval(x, 1, B.MUSR_FP64)
        _check_fp64(v, g, ref)
        v, g, st = ctx.eval(x, 1, B.MUSR_SPLIT)
        _check_split(v, g, ref)


def test_per_histogram_t0_and_fit_range_edges(B):
    """Fractional, different t0 per histogram: SPLIT groups split by t0; a fit range that
    starts and ends inside tiles."""
    p = mi.cfg2(nhist=6, nbins=7001, bin_width_ns=1.6, seed=21)
    t0 = np.array([0.0, 0.0, 3.25, 3.25, 17.5, 0.0])
    q = mi.Problem(p.counts, t0, p.bin_width_ns, (0.37, 9.9), p.terms, p.map, p.consts, p.nparams,
                   p.truth, p.names)
    x = mi.start_point(q, 9)
    with B.Context(q) as ctx:
        for mode in (0, 1):
            ref = oracle.cost(q, x, mode)
            v, g, _ = ctx.eval(x, mode, B.MUSR_FP64)
            _check_fp64(v, g, ref)
            v, g, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
            _check_split(v, g, ref)


def test_mle_undefined_is_nonfinite(B):
    p = mi.cfg1(nbins=2048, seed=3, dtype=np.float32)
    x = p.truth.copy()
    x[0] = -50.0  # N0 < 0 with Nbkg small: N <= 0 where d > 0
    x[1] = 0.0
    with B.Context(p) as ctx:
        for prec in (0, 1):
            v, g, st = ctx.eval(x, 1, prec)
            assert st == B.MUSR_ENONFINITE and np.isinf(v) and not g.any()
            v, g, st = ctx.eval(x, 0, prec)  # chi^2 stays finite
            assert st == 0 and np.isfinite(v)


def test_generic_and_noncanonical_theories(B):
    """A term list outside the compiled SPLIT shapes runs the generic SPLIT kernel; a term
    with two cosines has no basis form: SPLIT evaluates its term list per bin."""
    base = mi.cfg1(nbins=3000, bin_width_ns=3.0, seed=5, dtype=np.float32)
    terms = [[("AMP", (2,)), ("EXP", (3,))], [("AMP", (4,)), ("GAUSS", (5,)), ("EXP", (3,))],
             [("AMP", (6,)), ("KT", (7,))], [("AMP", (8,)), ("TFCOS", (9, 10))]]
    mp = np.array([[0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10]], np.int32)
    x = np.array([300.0, 2.0, 0.05, 0.3, 0.05, 0.4, 0.05, 0.5, 0.1, 5.0, 20.0])
    p = mi.Problem(base.counts, base.t0, base.bin_width_ns, base.fit_range_us, terms, mp, np.zeros(0), 11,
                   x, [f"p{i}" for i in range(11)])
    with B.Context(p) as ctx:
        for mode in (0, 1):
            ref = oracle.cost(p, x, mode)
            v, g, _ = ctx.eval(x, mode, B.MUSR_FP64)
            _check_fp64(v, g, ref)
            v, g, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
            _check_split(v, g, ref)
    terms2 = [[("AMP", (2,)), ("TFCOS", (3, 4)), ("TFCOS", (5, 4))]]
    mp2 = np.array([[0, 1, 2, 3, 4, 5]], np.int32)
    x2 = np.array([300.0, 2.0, 0.2, 5.0, 10.0, 0.3])
    p2 = mi.Problem(base.counts, base.t0, base.bin_width_ns, base.fit_range_us, terms2, mp2, np.zeros(0), 6,
                    x2, [f"p{i}" for i in range(6)])
    with B.Context(p2) as ctx:
        for mode in (0, 1):
            ref = oracle.cost(p2, x2, mode)
            v, g, _ = ctx.eval(x2, mode, B.MUSR_FP64)
            _check_fp64(v, g, ref)
            v, g, _ = ctx.eval(x2, mode, B.MUSR_SPLIT)  # no basis form: the term list per bin
            _check_split(v, g, ref)


def test_invalid_arguments(B):
    p = mi.cfg1(nbins=512, seed=4, dtype=np.float32)
    ctx = B.musr_ctx_create(0)
    try:
        with pytest.raises(B.MusrError) as e:
            B.musr_eval(ctx, p.truth, 0, 0)
        assert e.value.status == B.MUSR_ESTATE
        B.musr_upload_histograms(ctx, p.counts, p.t0, p.bin_width_ns, p.fit_range_us)
        B.musr_set_theory(ctx, p.terms)
        bad = p.map.copy()
        bad[0, 3] = 99
        with pytest.raises(B.MusrError) as e:
            B.musr_set_map(ctx, bad, p.nparams, p.consts)
        assert e.value.status == B.MUSR_EINVAL
        B.musr_set_map(ctx, p.map, p.nparams, p.consts)
        x = p.truth.copy()
        x[2] = np.nan
        with pytest.raises(B.MusrError) as e:
            B.musr_eval(ctx, x, 0, 0)
        assert e.value.status == B.MUSR_EINVAL
        with pytest.raises(B.MusrError):
            B.musr_eval(ctx, p.truth[:3], 0, 0)
        with pytest.raises(B.MusrError):
            B.musr_eval(ctx, p.truth, 2, 0)
    finally:
        B.musr_ctx_destroy(ctx)


def test_upload_checks_counts_on_device(B):
    """Counts are copied as they are and checked on the device: a non-finite float or an
    INT32 count beyond 2^24 anywhere (here the last bin of the last row, in a row length
    that is not a multiple of the device row stride) fails with MUSR_EINVAL and leaves no
    histograms; the limits themselves pass, and a valid upload afterwards evaluates as
    the oracle does."""
    p = mi.cfg1(nbins=1000, seed=6, dtype=np.float32)
    ctx = B.musr_ctx_create(0)
    try:
        for dtype, bad in ((np.float32, np.nan), (np.float32, np.inf), (np.float32, -np.inf),
                           (np.float64, np.nan), (np.float64, np.inf),
                           (np.int32, 1 << 24), (np.int32, -(1 << 24)), (np.int32, np.iinfo(np.int32).max)):
            c = np.ascontiguousarray(np.tile(p.counts[0].astype(dtype), (3, 1)))
            c[-1, -1] = bad
            with pytest.raises(B.MusrError) as e:
                B.musr_upload_histograms(ctx, c, np.zeros(3), p.bin_width_ns, p.fit_range_us)
            assert e.value.status == B.MUSR_EINVAL, (dtype, bad)
            B.musr_set_theory(ctx, p.terms)
            with pytest.raises(B.MusrError) as e:  # no histograms
                B.musr_set_map(ctx, np.tile(p.map, (3, 1)), p.nparams, p.consts)
            assert e.value.status == B.MUSR_ESTATE
        for dtype, edge in ((np.int32, (1 << 24) - 1), (np.int32, -(1 << 24) + 1),
                            (np.float32, np.finfo(np.float32).max), (np.float64, np.finfo(np.float64).max)):
            c = np.ascontiguousarray(p.counts[0].astype(dtype)[None, :])
            c[0, -1] = edge
            B.musr_upload_histograms(ctx, c, p.t0, p.bin_width_ns, p.fit_range_us)
        c = np.ascontiguousarray(p.counts[0].astype(np.int32)[None, :])
        B.musr_upload_histograms(ctx, c, p.t0, p.bin_width_ns, p.fit_range_us)
        B.musr_set_theory(ctx, p.terms)
        B.musr_set_map(ctx, p.map, p.nparams, p.consts)
        q = mi.Problem(c, p.t0, p.bin_width_ns, p.fit_range_us, p.terms, p.map, p.consts, p.nparams, p.truth,
                       p.names)
        for mode in (0, 1):
            v, g, _ = B.musr_eval(ctx, p.truth, mode, B.MUSR_FP64)
            _check_fp64(v, g, oracle.cost(q, p.truth, mode))
    finally:
        B.musr_ctx_destroy(ctx)


# Per-detector time-zero bins.  Histograms whose t0 differ by whole bins are moved onto one
# time grid on the device (and share the time factors there); the cost is the same sum.
T0_CASES = {
    "integer": lambda H: np.arange(H, dtype=float),
    "multiple_of_4": lambda H: 4.0 * np.arange(H),
    "equal_fractions": lambda H: np.arange(H) + 0.5,
    "equal_fractions_inexact": lambda H: np.arange(H) + 0.37,  # (h + 0.37) - h is not exactly 0.37
    "mixed_fractions": lambda H: 3.0 + 0.25 * np.arange(H),
    "negative": lambda H: np.arange(H) - 3.0,
    "one_beyond_the_data": lambda H: np.where(np.arange(H) == H - 1, 5100.0, np.arange(H, dtype=float)),
    "large_offsets": lambda H: 997.0 * np.arange(H),
}


@pytest.mark.parametrize("case", sorted(T0_CASES))
@pytest.mark.parametrize("window", [(0.05, 9.0), (-0.02, 9.9)])
def test_per_detector_t0_offsets(B, case, window):
    base = mi.paper_tf16(nhist=6, nbins=5000, bin_width_ns=2.0, seed=77)
    p = dataclasses.replace(base, t0=T0_CASES[case](6), fit_range_us=window)
    x = mi.start_point(p, 3)
    X = mi.jitter(x, 5, seed=4, lo=0.97, hi=1.03)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            ref = oracle.cost(p, x, mode)
            v, g, _ = ctx.eval(x, mode, B.MUSR_FP64)
            _check_fp64(v, g, ref)
            v, g, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
            _check_split(v, g, ref)
            vals, grads, st = ctx.eval_batch(X, mode, B.MUSR_SPLIT)
            assert st == 0
            for i in (0, 4):
                _check_split(vals[i], grads[i], oracle.cost(p, X[i], mode))


def test_shifted_upload_every_dtype_and_check(B):
    """The shifted upload path in each dtype, and its check of every value: a NaN in bins
    the shift leaves out of the device image (before a histogram's fit window) still fails."""
    base = mi.paper_tf16(nhist=4, nbins=3001, bin_width_ns=3.0, seed=78)
    t0 = np.array([0.0, 2.0, 5.0, 9.0])
    x = mi.start_point(base, 1)
    for dtype in (np.int32, np.float32, np.float64):
        p = dataclasses.replace(base, counts=np.ascontiguousarray(base.counts.astype(dtype)), t0=t0,
                                fit_range_us=(0.01, 8.5))
        with B.Context(p) as ctx:
            for mode in (0, 1):
                ref = oracle.cost(p, x, mode)
                v, g, _ = ctx.eval(x, mode, B.MUSR_FP64)
                _check_fp64(v, g, ref)
    bad = np.ascontiguousarray(base.counts.astype(np.float32))
    bad[3, 2] = np.nan  # bin 2 of the histogram with t0 = 9 bins: moved out of the image
    ctx = B.musr_ctx_create(0)
    try:
        with pytest.raises(B.MusrError) as e:
            B.musr_upload_histograms(ctx, bad, t0, base.bin_width_ns, (0.01, 8.5))
        assert e.value.status == B.MUSR_EINVAL
    finally:
        B.musr_ctx_destroy(ctx)


def test_term_lists_without_basis_form(B):
    """The stretched exponential and the Bessel precession (no basis form): both paths against
    the oracle (single and batched, both costs) for Monte Carlo configurations and a theory
    mixing them with the other primitives; SPLIT evaluates the term list per bin in FP32, and
    its Gauss-Newton products are refused (FP64 only)."""
    import test_oracle_pins as pins
    q, xq = pins._new_primitive_problem()
    # three terms, one of four primitives: the general term-list kernel (the others fit the
    # kernel for at most two terms of at most three primitives)
    big_terms = q.terms + [[("AMP", (9,)), ("STREXP", (10, 4)), ("GAUSS", (6,)), ("TFCOS", (6, 7))]]
    big_map = np.hstack([q.map, np.array([[12, 13], [12, 14]], np.int32)])
    qb = mi.Problem(q.counts, q.t0, q.bin_width_ns, q.fit_range_us, big_terms, big_map, q.consts, 15, np.zeros(15),
                    [f"p{i}" for i in range(15)])
    xb = np.concatenate([xq, [0.05, 0.9, 1.2]])
    cases = [(mi.inc_bessel(nhist=2, nbins=3000, bin_width_ns=4.0, seed=71), None),
             (mi.levy_lf(nhist=3, nbins=2500, bin_width_ns=5.0, seed=72), None), (q, xq), (qb, xb)]
    for p, x in cases:
        x = mi.start_point(p, 2) if x is None else x
        X = mi.jitter(x, 4, seed=3, lo=0.98, hi=1.02)
        with B.Context(p) as ctx:
            for mode in (0, 1):
                ref = oracle.cost(p, x, mode)
                v, g, _ = ctx.eval(x, mode, B.MUSR_FP64)
                _check_fp64(v, g, ref)
                v, g, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
                _check_split(v, g, ref)
                for prec, check in ((B.MUSR_FP64, _check_fp64), (B.MUSR_SPLIT, _check_split)):
                    vals, grads, st = ctx.eval_batch(X, mode, prec)
                    assert st == 0
                    for i in (0, 3):
                        check(vals[i], grads[i], oracle.cost(p, X[i], mode))
            with pytest.raises(B.MusrError) as e:
                ctx.gauss_newton(x, 1, B.MUSR_SPLIT)
            assert e.value.status == B.MUSR_EINVAL and "basis form" in str(e.value)


def test_full_size_in_the_benchmark_launch_configuration(B):
    """cfg2 at its full size (8 x 65536 bins) with 64 parameter vectors per launch of -2lnL
    value+gradient, the launch the benchmark times (its decomposition: tiles of 16384 bins):
    sampled vectors of the batch against the oracle, SPLIT and FP64."""
    p = mi.cfg2()
    X = mi.jitter(p.truth, 64, seed=1, lo=0.95, hi=1.05)
    with B.Context(p) as ctx:
        vs, gs, st = ctx.eval_batch(X, 1, B.MUSR_SPLIT)
        assert st == 0
        v64, g64, st = ctx.eval_batch(X, 1, B.MUSR_FP64)
        assert st == 0
    for i in (0, 31, 63):
        ref = oracle.cost(p, X[i], 1)
        _check_split(vs[i], gs[i], ref)
        _check_fp64(v64[i], g64[i], ref)


@pytest.mark.slow
def test_large_fit_in_the_benchmark_launch_configuration(B):
    """64 x 2^20 bins with 64 parameter vectors per launch of -2lnL value+gradient, the launch
    the benchmark's contract line times (tiles of 32768 bins, the longest FP32 runs per
    thread): the first and the last vector of the batch against the oracle's full sums."""
    p = mi.cfg5()
    X = mi.jitter(p.truth, 64, seed=1, lo=0.98, hi=1.02)
    with B.Context(p) as ctx:
        vs, gs, st = ctx.eval_batch(X, 1, B.MUSR_SPLIT)
        assert st == 0
    for i in (0, 63):
        _check_split(vs[i], gs[i], oracle.cost(p, X[i], 1))


@pytest.mark.parametrize("mode", [0, 1])
def test_launch_level_partition_matches_oracle(B, mode):
    """Batches whose work items do not divide evenly over the grid take the launch-level
    partition (pieces of CTA ranges crossing vectors and chunks): the paper benchmark's
    16 x 81920 bins at 64 and 8 parameter vectors, sampled vectors against the oracle, every
    vector against the plain FP64 path, and bit-identical on repetition."""
    p = mi.paper_tf16()
    X = mi.jitter(p.truth, 64, seed=12, lo=0.97, hi=1.03)
    with B.Context(p) as ctx:
        for n in (64, 8):
            vals, grads, st = ctx.eval_batch(X[:n], mode, B.MUSR_SPLIT)
            assert st == 0
            v64, g64, _ = ctx.eval_batch(X[:n], mode, B.MUSR_FP64)
            for i in (0, n // 2, n - 1):
                _check_split(vals[i], grads[i], oracle.cost(p, X[i], mode))
            assert np.all(np.abs(vals - v64) <= SPLIT_EPS * np.abs(v64))
            vals2, grads2, _ = ctx.eval_batch(X[:n], mode, B.MUSR_SPLIT)
            assert np.array_equal(vals, vals2) and np.array_equal(grads, grads2)


def test_hbm_budget_is_enforced(B):
    p = mi.cfg2(nhist=8, nbins=65536, seed=2)
    ctx = B.musr_ctx_create(0, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(B.MusrError) as e:
            B.musr_upload_histograms(ctx, p.counts, p.t0, p.bin_width_ns, p.fit_range_us)
        assert e.value.status == B.MUSR_ENOMEM
    finally:
        B.musr_ctx_destroy(ctx)


@pytest.mark.slow
def test_full_size_large_fit_fp64_matches_oracle(B):
    """64 x 2^20 bins (FP32 counts, 256 MiB), the launch configuration of the large-fit
    workload: the FP64 path against the oracle's full sum, and SPLIT within its bound."""
    p = mi.cfg5()
    x = p.truth * np.random.default_rng(55).uniform(0.98, 1.02, p.nparams)
    ref = oracle.cost(p, x, 1)
    with B.Context(p) as ctx:
        v, g, st = ctx.eval(x, 1, B.MUSR_FP64)
        _check_fp64(v, g, ref)
        v, g, st = ctx.eval(x, 1, B.MUSR_SPLIT)
        _check_split(v, g, ref)


# ------------------------------------------------------------------------------------------
# Every SPLIT shape (musr_plan.h): term lists chosen so that each compiled shape runs, on
# several histograms (a chunk that is not full) with a ragged bin count.
# ------------------------------------------------------------------------------------------

def _build(terms, slots, H, nbins=2500 + 7, bw=2.0, seed=0):
    """A problem from slot descriptors: ("hist", v) a parameter per histogram, ("shared", v)
    one parameter, ("const", v) one constant, ("const_h", [v_j]) a constant per histogram.
    Counts are Poisson draws of the oracle's model at the truth."""
    params, consts, rows = [], [], [[0] * len(slots) for _ in range(H)]
    for s, (kind, v) in enumerate(slots):
        if kind == "shared":
            params.append(v)
            for j in range(H):
                rows[j][s] = len(params) - 1
        elif kind == "hist":
            for j in range(H):
                params.append(v * (1.0 + 0.05 * j) if s != 1 else v)
                rows[j][s] = len(params) - 1
        elif kind == "const":
            consts.append(v)
            for j in range(H):
                rows[j][s] = -len(consts)
        else:  # const_h
            for j in range(H):
                consts.append(v[j])
                rows[j][s] = -len(consts)
    truth = np.array(params)
    mp = np.array(rows, np.int32)
    dummy = np.zeros((H, nbins), np.float32)
    p0 = mi.Problem(dummy, np.zeros(H), bw, (bw / 2000.0, nbins * bw / 1000.0), terms, mp, np.array(consts),
                    len(params), truth, [f"p{i}" for i in range(len(params))])
    dt = bw / 1000.0
    lam = np.array([[oracle.model(p0, truth, h, n * dt) for n in range(nbins)] for h in range(H)])
    counts = np.random.default_rng(seed).poisson(np.maximum(lam, 0.0)).astype(np.float32)
    return p0.with_counts(counts)


def _shape_cases():
    N0, BKG = ("hist", 120.0), ("hist", 1.5)
    cases = {}
    # one cosine term and one other term, amplitudes per histogram (T1N1)
    cases["T1N1"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))], [("AMP", (6,)), ("KT", (7,))]],
                     [N0, BKG, ("hist", 0.2), ("shared", 0.4), ("shared", 1.5), ("hist", 30.0),
                      ("shared", 0.05), ("shared", 0.35)])
    # two cosine terms with their own phases (T2, unmerged)
    cases["T2"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
                    [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 9))]],
                   [N0, BKG, ("const", 0.12), ("shared", 0.5), ("shared", 1.2), ("hist", 20.0),
                    ("const", 0.1), ("shared", 0.3), ("shared", 1.7), ("hist", 75.0)])
    # T2 plus an exponential with a fitted amplitude (T2N1, unmerged)
    cases["T2N1"] = (cases["T2"][0] + [[("AMP", (10,)), ("EXP", (11,))]],
                     cases["T2"][1] + [("shared", 0.06), ("shared", 0.8)])
    # shared phase, constant shared amplitudes, plus a plain exponential: merged with a plain term
    cases["T2N1m"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
                       [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 5))],
                       [("AMP", (9,)), ("EXP", (10,))]],
                      [N0, BKG, ("const", 0.12), ("shared", 0.5), ("shared", 1.2), ("hist", 20.0),
                       ("const", 0.1), ("shared", 0.3), ("shared", 1.7), ("const", 0.05), ("shared", 0.9)])
    # shared phase but amplitudes that differ between histograms: not merged (T2)
    cases["T2_const_h"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
                            [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 5))]],
                           [N0, BKG, ("const_h", [0.10, 0.12, 0.14, 0.16, 0.18]), ("shared", 0.5),
                            ("shared", 1.2), ("hist", 20.0), ("const", 0.1), ("shared", 0.3),
                            ("shared", 1.7)])
    # two terms without cosine (generic)
    cases["generic_N2"] = ([[("AMP", (2,)), ("EXP", (3,))], [("AMP", (4,)), ("GAUSS", (5,)), ("KT", (6,))]],
                           [N0, BKG, ("hist", 0.15), ("shared", 0.4), ("shared", 0.1), ("shared", 0.6),
                            ("shared", 0.3)])
    # static Lorentzian Kubo-Toyabe terms: alone with an exponential (N1), beside a cosine term
    # (T1N1), as the third term of a merged list (T2N1m), and beside two other terms (generic)
    cases["N1_lkt"] = ([[("AMP", (2,)), ("LKT", (3,)), ("EXP", (4,))]],
                       [N0, BKG, ("shared", 0.2), ("shared", 0.7), ("shared", 0.1)])
    cases["T1N1_lkt"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))], [("AMP", (6,)), ("LKT", (7,))]],
                         [N0, BKG, ("hist", 0.2), ("shared", 0.4), ("shared", 1.5), ("hist", 30.0),
                          ("shared", 0.05), ("shared", 0.9)])
    cases["T2N1m_lkt"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
                           [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 5))],
                           [("AMP", (9,)), ("LKT", (10,))]],
                          [N0, BKG, ("const", 0.12), ("shared", 0.5), ("shared", 1.2), ("hist", 20.0),
                           ("const", 0.1), ("shared", 0.3), ("shared", 1.7), ("const", 0.05), ("shared", 0.6)])
    cases["generic_lkt"] = ([[("AMP", (2,)), ("LKT", (3,))], [("AMP", (4,)), ("KT", (5,))],
                             [("AMP", (6,)), ("EXP", (7,))]],
                            [N0, BKG, ("shared", 0.1), ("shared", 0.8), ("shared", 0.08), ("shared", 0.4),
                             ("hist", 0.05), ("shared", 0.3)])
    # three cosine terms (generic)
    cases["generic_T3"] = ([[("AMP", (2,)), ("EXP", (3,)), ("TFCOS", (4, 5))],
                            [("AMP", (6,)), ("GAUSS", (7,)), ("TFCOS", (8, 5))],
                            [("AMP", (9,)), ("TFCOS", (10, 11))]],
                           [N0, BKG, ("shared", 0.1), ("shared", 0.5), ("shared", 1.2), ("hist", 20.0),
                            ("shared", 0.08), ("shared", 0.3), ("shared", 1.7), ("shared", 0.05),
                            ("shared", 0.45), ("hist", 60.0)])
    return cases


@pytest.mark.parametrize("name", sorted(_shape_cases()))
def test_every_split_shape_matches_oracle(B, name):
    terms, slots = _shape_cases()[name]
    p = _build(terms, slots, H=5, seed=sum(map(ord, name)))
    x = p.truth * np.random.default_rng(7).uniform(0.97, 1.03, p.nparams)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            ref = oracle.cost(p, x, mode)
            assert ref[3] == 0
            v, g, _ = ctx.eval(x, mode, B.MUSR_FP64)
            _check_fp64(v, g, ref)
            v, g, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
            _check_split(v, g, ref)
            v2, _, _ = ctx.eval(x, mode, B.MUSR_SPLIT, grad=False)
            assert v2 == v


def _limits_problem(nhist=1360, nbins=48, seed=71):
    """A problem at the ABI's limits: MUSR_MAX_PARAMS (4096) parameters, MUSR_MAX_SLOTS (32)
    slots with the phase in the last one, MUSR_MAX_TERMS (4) terms of MUSR_MAX_PRIMS (4)
    primitives each; 1360 short histograms with N0, Nbkg and the phase per histogram, 16
    shared parameters, slots 18 ... 30 mapped to a constant."""
    terms = [[("AMP", (2,)), ("EXP", (3,)), ("GAUSS", (4,)), ("TFCOS", (5, 31))],
             [("AMP", (6,)), ("EXP", (7,)), ("GAUSS", (8,)), ("TFCOS", (9, 31))],
             [("AMP", (10,)), ("EXP", (11,)), ("KT", (12,)), ("EXP", (13,))],
             [("AMP", (14,)), ("GAUSS", (15,)), ("LKT", (16,)), ("EXP", (17,))]]
    shared = [0.10, 0.3, 0.2, 1.5, 0.08, 0.2, 0.1, 2.2, 0.05, 0.1, 0.4, 0.05, 0.04, 0.1, 0.3, 0.1]
    rng = np.random.default_rng(seed)
    mp = np.full((nhist, 32), -1, np.int32)
    mp[:, 2:18] = np.arange(16)
    h = np.arange(nhist)
    mp[:, 0] = 16 + 3 * h
    mp[:, 1] = 16 + 3 * h + 1
    mp[:, 31] = 16 + 3 * h + 2
    P = 16 + 3 * nhist
    truth = np.empty(P)
    truth[:16] = shared
    truth[16::3] = 400.0 * (1.0 + 0.2 * h / nhist)
    truth[17::3] = 3.0
    truth[18::3] = 360.0 * h / nhist
    dt_ns = 250.0
    t = (np.arange(nbins) * dt_ns * 1e-3)[None, :]
    shape = np.exp(-t / 2.197019) * (1.0 + 0.1 * np.exp(-0.3 * t) * np.cos(2 * np.pi * (1.5 * t + h[:, None] / nhist)))
    counts = rng.poisson(truth[16::3, None] * shape + 3.0).astype(np.float32)
    return mi.Problem(counts, np.zeros(nhist), dt_ns, (0.2, 11.8), terms, mp, np.zeros(1), P, truth,
                      [f"p{i}" for i in range(P)])


@pytest.mark.parametrize("mode", [0, 1])
def test_abi_limits_match_oracle(B, mode):
    """Every size limit of the ABI at once (4096 parameters, 32 slots, 4 terms of 4
    primitives, 1360 histograms): both paths against the oracle, single and batched."""
    p = _limits_problem()
    assert p.nparams == 4096 and p.nslots == 32
    X = mi.jitter(p.truth, 3, seed=72 + mode, lo=0.97, hi=1.03)
    with B.Context(p) as ctx:
        for prec, check in ((B.MUSR_FP64, _check_fp64), (B.MUSR_SPLIT, _check_split)):
            ref = oracle.cost(p, X[0], mode)
            assert ref[3] == 0
            v, g, st = ctx.eval(X[0], mode, prec)
            assert st == 0
            check(v, g, ref)
            vals, grads, st = ctx.eval_batch(X, mode, prec)
            assert st == 0
            for i in (1, 2):
                check(vals[i], grads[i], oracle.cost(p, X[i], mode))
