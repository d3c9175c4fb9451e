"""musr_eval_noalloc, the entry point that allocates nothing, against musr_eval.

Callers that cannot allocate device memory -- a framework whose pool owns the GPU,
a host that reserves all HBM up front, a loop that cannot afford an allocation's
synchronisation -- cannot create a context either, so musr_eval_noalloc keeps its
scratch in a fixed device array inside the library.  This test allocates the
inputs and outputs with torch (a test may); the entry point itself allocates
nothing.  Two calls in a row, with different parameters, must each match the
context path within the parity tolerances: the second call also checks that what
the first one left in the shared scratch does not leak into its result.
"""
import numpy as np
import pytest

import musr_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SPLIT_EPS = 2.0 ** -16


def test_noalloc_matches_context_on_two_calls_in_a_row(musr_lib):
    import torch

    from paper_1509_07685_gb300 import binding as B
    p = mi.cfg2(nhist=6, nbins=12001, bin_width_ns=1.0, seed=61)
    stride = (p.B + 3) // 4 * 4
    d_counts = torch.zeros((p.H, stride), dtype=torch.float32, device="cuda")
    d_counts[:, :p.B] = torch.from_numpy(np.ascontiguousarray(p.counts, dtype=np.float32)).cuda()
    xs = [mi.start_point(p, 1), mi.start_point(p, 2)]
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    with B.Context(p) as ctx:
        for prec, tol in ((B.MUSR_FP64, FP64_TOL), (B.MUSR_SPLIT, SPLIT_EPS)):
            for mode in (B.MUSR_CHI2, B.MUSR_MLE):
                for x in xs:  # two calls in a row on the same scratch
                    d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
                    d_out = torch.full((1 + p.nparams,), float("nan"), dtype=torch.float64, device="cuda")
                    st = B.musr_eval_noalloc(d_counts.data_ptr(), B.MUSR_DTYPE_FP32, p.H, p.B, stride, p.t0,
                                             p.bin_width_ns, p.fit_range_us, p.terms, p.map, p.nparams,
                                             p.consts, d_x.data_ptr(), mode, prec, True, d_out.data_ptr(),
                                             stream)
                    assert st == B.MUSR_OK
                    torch.cuda.synchronize()
                    out = d_out.cpu().numpy()
                    v, g, _ = ctx.eval(x, mode, prec)
                    gs = oracle.cost(p, x, mode)[2]
                    assert abs(out[0] - v) <= tol * abs(v), (prec, mode, out[0], v)
                    assert np.all(np.abs(out[1:] - g) <= tol * gs + 1e-300), (prec, mode)


def test_noalloc_rejects_sizes_beyond_its_scratch(musr_lib):
    import torch

    from paper_1509_07685_gb300 import binding as B
    p = mi.cfg3(nhist=65, nbins=64, bin_width_ns=200.0, seed=62)  # 65 histograms: above the limit of 64
    d_counts = torch.zeros((p.H, 64), dtype=torch.float32, device="cuda")
    d_x = torch.tensor(p.truth, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(1 + p.nparams, dtype=torch.float64, device="cuda")
    st = B.musr_eval_noalloc(d_counts.data_ptr(), B.MUSR_DTYPE_FP32, p.H, p.B, 64, p.t0, p.bin_width_ns,
                             p.fit_range_us, p.terms, p.map, p.nparams, p.consts, d_x.data_ptr(), 0,
                             B.MUSR_FP64, True, d_out.data_ptr(), None)
    assert st == B.MUSR_EINVAL


def test_noalloc_at_its_limits_matches_oracle(musr_lib):
    """64 histograms, 1024 parameters and 256 constants (the scratch's limits), 32 slots and
    4 terms of 4 primitives: both precisions against the oracle.  Slots the theory does not
    read carry parameters of their own, whose derivatives must come out as zero."""
    import dataclasses

    import torch

    from paper_1509_07685_gb300 import binding as B
    from test_gpu_parity import _check_fp64, _check_split, _limits_problem
    p = _limits_problem(nhist=64, nbins=700, seed=63)
    mp = p.map.copy()
    H, P0 = p.H, p.nparams  # 16 shared + 3 per histogram
    extra = np.arange(12 * H, dtype=np.int32).reshape(H, 12) + P0
    mp[:, 18:30] = extra  # unread slots
    P = P0 + 12 * H
    mp[:48, 30] = P + np.arange(48)
    P += 48
    mp[48:, 30] = -256  # consts[255]
    consts = np.linspace(0.0, 1.0, 256)
    rng = np.random.default_rng(64)
    truth = np.concatenate([p.truth, rng.uniform(-1.0, 1.0, P - P0)])
    q = dataclasses.replace(p, map=mp, consts=consts, nparams=P, truth=truth)
    assert q.H == 64 and q.nparams == 1024 and len(q.consts) == 256 and q.nslots == 32
    stride = (q.B + 3) // 4 * 4
    d_counts = torch.zeros((q.H, stride), dtype=torch.float32, device="cuda")
    d_counts[:, :q.B] = torch.from_numpy(np.ascontiguousarray(q.counts, dtype=np.float32)).cuda()
    x = q.truth * np.random.default_rng(65).uniform(0.98, 1.02, q.nparams)
    d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for prec, check in ((B.MUSR_FP64, _check_fp64), (B.MUSR_SPLIT, _check_split)):
        for mode in (B.MUSR_CHI2, B.MUSR_MLE):
            d_out = torch.full((1 + q.nparams,), float("nan"), dtype=torch.float64, device="cuda")
            st = B.musr_eval_noalloc(d_counts.data_ptr(), B.MUSR_DTYPE_FP32, q.H, q.B, stride, q.t0,
                                     q.bin_width_ns, q.fit_range_us, q.terms, q.map, q.nparams, q.consts,
                                     d_x.data_ptr(), mode, prec, True, d_out.data_ptr(), stream)
            assert st == B.MUSR_OK
            torch.cuda.synchronize()
            out = d_out.cpu().numpy()
            ref = oracle.cost(q, x, mode)
            assert ref[3] == 0
            check(out[0], out[1:], ref)
            assert np.all(out[1 + P0:1 + P0 + 12 * H] == 0.0) and np.all(out[1 + P0 + 12 * H:] == 0.0)


def test_noalloc_term_list_without_basis_form_matches_context(musr_lib):
    """A theory without a basis form (a stretched exponential) at SPLIT precision: the entry
    point evaluates the term list per bin, as a context does, and matches it."""
    import torch

    from paper_1509_07685_gb300 import binding as B
    p = mi.levy_lf(nhist=2, nbins=1600, bin_width_ns=8.0, seed=66)
    stride = (p.B + 3) // 4 * 4
    d_counts = torch.zeros((p.H, stride), dtype=torch.float32, device="cuda")
    d_counts[:, :p.B] = torch.from_numpy(np.ascontiguousarray(p.counts, dtype=np.float32)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    with B.Context(p) as ctx:
        for mode in (B.MUSR_CHI2, B.MUSR_MLE):
            for seed in (1, 2):  # two calls in a row
                x = mi.start_point(p, seed)
                d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
                d_out = torch.full((1 + p.nparams,), float("nan"), dtype=torch.float64, device="cuda")
                st = B.musr_eval_noalloc(d_counts.data_ptr(), B.MUSR_DTYPE_FP32, p.H, p.B, stride, p.t0,
                                         p.bin_width_ns, p.fit_range_us, p.terms, p.map, p.nparams, p.consts,
                                         d_x.data_ptr(), mode, B.MUSR_SPLIT, True, d_out.data_ptr(), stream)
                assert st == B.MUSR_OK, B.musr_last_error(None)
                torch.cuda.synchronize()
                out = d_out.cpu().numpy()
                v, g, _ = ctx.eval(x, mode, B.MUSR_SPLIT)
                gs = oracle.cost(p, x, mode)[2]
                assert abs(out[0] - v) <= SPLIT_EPS * abs(v)
                assert np.all(np.abs(out[1:] - g) <= SPLIT_EPS * gs + 1e-300)


def test_noalloc_refuses_a_capturing_stream_and_names_its_reasons(musr_lib):
    """The tables are staged from a host buffer that later calls overwrite, so a call on a
    stream that is capturing returns MUSR_EINVAL and enqueues nothing; every refusal leaves
    its reason for musr_last_error(NULL).  The scratch still works afterwards."""
    import torch

    from paper_1509_07685_gb300 import binding as B
    p = mi.cfg3(nhist=2, nbins=2048, bin_width_ns=6.0, seed=67)
    stride = (p.B + 3) // 4 * 4
    d_counts = torch.zeros((p.H, stride), dtype=torch.float32, device="cuda")
    d_counts[:, :p.B] = torch.from_numpy(np.ascontiguousarray(p.counts, dtype=np.float32)).cuda()
    x = mi.start_point(p, 3)
    d_x = torch.tensor(x, dtype=torch.float64, device="cuda")
    d_out = torch.full((1 + p.nparams,), float("nan"), dtype=torch.float64, device="cuda")
    args = lambda stream: (d_counts.data_ptr(), B.MUSR_DTYPE_FP32, p.H, p.B, stride, p.t0, p.bin_width_ns,
                           p.fit_range_us, p.terms, p.map, p.nparams, p.consts, d_x.data_ptr(), 0,
                           B.MUSR_FP64, True, d_out.data_ptr(), stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = B.musr_eval_noalloc(*args(torch.cuda.current_stream().cuda_stream))
        msg = B.musr_last_error(None)
    assert st == B.MUSR_EINVAL and "capturing" in msg
    bad = list(args(None))
    bad[4] = stride + 2  # row stride not a multiple of 4
    assert B.musr_eval_noalloc(*bad) == B.MUSR_EINVAL
    assert "row_stride" in B.musr_last_error(None)
    st = B.musr_eval_noalloc(*args(torch.cuda.current_stream().cuda_stream))
    assert st == B.MUSR_OK and B.musr_last_error(None) == ""
    torch.cuda.synchronize()
    ref = oracle.cost(p, x, 0)
    out = d_out.cpu().numpy()
    assert abs(out[0] - ref[0]) <= FP64_TOL * abs(ref[0])
