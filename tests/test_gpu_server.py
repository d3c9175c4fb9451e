"""Serving (continuous batching) and the native fit.

* Each fit's result is the same alone and in a mix: a fit served by itself and the
  same fit served among others (different theories, sizes, costs and arrival times)
  give bit-identical parameters, because a fit's launches use its own decomposition
  and fixed-order reductions.
* Admission by budget: with room for only a few fits, all fits still complete, the
  arena never exceeds its size, and a fit larger than the whole budget is rejected.
* The native fit (musr_fit) and the Python BFGS reach the same optimum (0.01 sigma).
"""
import time

import numpy as np
import pytest

import musr_inputs as mi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _small_pool():
    return [
        (mi.cfg1(nbins=4096, bin_width_ns=2.0, seed=301, dtype=np.float32), 1, 1),
        (mi.cfg2(nhist=3, nbins=8192, bin_width_ns=1.5625, seed=302), 1, 1),
        (mi.cfg3(nhist=2, nbins=6000, bin_width_ns=2.0, seed=303), 0, 1),
        (mi.cfg2(nhist=5, nbins=5000, bin_width_ns=2.56, seed=304), 0, 0),
        (mi.cfg3(nhist=6, nbins=3000, bin_width_ns=4.0, seed=305), 1, 0),
        (mi.cfg1(nbins=9000, bin_width_ns=1.0, seed=306, dtype=np.float32), 0, 1),
    ]


def test_results_identical_alone_and_in_mix(B):
    pool = _small_pool()
    starts = [mi.start_point(p, 10 + i) for i, (p, _, _) in enumerate(pool)]
    alone = []
    with B.Server(hbm_budget_bytes=1 << 30, max_active=64) as srv:
        for (p, mode, prec), x0 in zip(pool, starts):
            fid = srv.submit(p, x0, mode, prec)
            r = srv.wait(fid, timeout_ms=120000)
            assert r is not None and r["status"] == 0, r
            alone.append(r)
    with B.Server(hbm_budget_bytes=1 << 30, max_active=64) as srv:
        ids = []
        for i, ((p, mode, prec), x0) in enumerate(zip(pool, starts)):
            ids.append(srv.submit(p, x0, mode, prec))
            if i == 2:
                time.sleep(0.002)  # later arrivals join while the first fits run
        mix = [srv.wait(fid, timeout_ms=120000) for fid in ids]
        st = srv.stats()
    for a, m in zip(alone, mix):
        assert m["status"] == 0
        assert np.array_equal(a["x"], m["x"]), np.max(np.abs(a["x"] - m["x"]))
        assert a["iters"] == m["iters"] and a["nfev"] == m["nfev"]
    assert st["completed"] == len(pool) and st["steps"] > 0 and st["launches"] >= st["steps"]


def test_borrowed_and_copied_counts_give_the_same_fits(B):
    """A request that lends its counts (read at admission) and one whose counts are copied
    at submission give bit-identical fits; unknown request flags are refused."""
    pool = _small_pool()
    starts = [mi.start_point(p, 40 + i) for i, (p, _, _) in enumerate(pool)]
    res = {}
    for borrow in (False, True):
        with B.Server(hbm_budget_bytes=1 << 30, max_active=64) as srv:
            ids = [srv.submit(p, x0, mode, prec, borrow=borrow) for (p, mode, prec), x0 in zip(pool, starts)]
            res[borrow] = [srv.wait(fid, timeout_ms=120000) for fid in ids]
            assert not srv.lent
    for a, b in zip(res[False], res[True]):
        assert a["status"] == 0 and b["status"] == 0
        assert np.array_equal(a["x"], b["x"]) and a["nfev"] == b["nfev"]
    p, mode, prec = pool[0]
    with B.Server(hbm_budget_bytes=1 << 28) as srv:
        q, keep = B.make_request(p, starts[0], mode, prec)
        q.flags = 2
        fid = B.ctypes.c_int64()
        assert B.load().musr_server_submit(srv.srv, B.ctypes.byref(q), B.ctypes.byref(fid)) == B.MUSR_EINVAL


def test_admission_by_budget_and_rejection(B):
    # ~0.7 MB per fit: a 2 MiB budget holds about two of them at a time
    p = mi.cfg2(nhist=8, nbins=20000, bin_width_ns=0.64, seed=311)
    with B.Server(hbm_budget_bytes=2 << 20, max_active=64) as srv:
        ids = [srv.submit(p, mi.start_point(p, 20 + i), 1, 1) for i in range(6)]
        big = mi.cfg5(nhist=64, nbins=1 << 17, seed=312)  # 32 MiB of counts alone
        big_id = srv.submit(big, big.truth, 1, 1)
        res = [srv.wait(fid, timeout_ms=120000) for fid in ids]
        rbig = srv.wait(big_id, timeout_ms=120000)
        st = srv.stats()
    assert all(r is not None and r["status"] == 0 for r in res)
    assert rbig["status"] == B.MUSR_ENOMEM
    assert st["completed"] == 6 and st["rejected"] == 1
    assert st["arena_used"] <= st["arena_bytes"]


def test_poll_before_completion_and_unknown_ids(B):
    p = mi.cfg2(seed=2)
    with B.Server(hbm_budget_bytes=1 << 30) as srv:
        fid = srv.submit(p, mi.start_point(p, 1), 1, 1)
        assert srv.poll(fid) is None  # a full cfg2 fit cannot be done within microseconds
        r = srv.wait(fid, timeout_ms=120000)
        assert r["status"] == 0
        with pytest.raises(B.MusrError):
            B.musr_server_poll(srv.srv, 999, 1)


def test_split_request_for_theory_without_basis_form(B):
    """A theory without a basis form (a stretched exponential of simulated Levy-rate
    depolarisation): a SPLIT request is served through the term list kernel and lands within
    0.01 sigma of the FP64 fit of the same request."""
    p = mi.levy_lf(seed=109)
    x0 = mi.start_point(p, 1)
    with B.Server(hbm_budget_bytes=1 << 28) as srv:
        r = {prec: srv.wait(srv.submit(p, x0, 1, prec), timeout_ms=60000) for prec in (0, 1)}
    assert r[0]["status"] == 0 and r[1]["status"] == 0, r
    sig = oracle.sigmas(p, r[0]["x"], 1)
    dev = np.abs(r[1]["x"] - r[0]["x"]) / sig
    assert np.all(dev < 0.01), (dev, r[0], r[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_native_fit_matches_python_fit(B, prec):
    from paper_1509_07685_gb300 import fit as F
    p = mi.cfg2(nhist=4, nbins=16384, bin_width_ns=0.78125, seed=331)
    x0 = mi.start_point(p, 3)
    with B.Context(p) as ctx:
        rn = B.musr_fit(ctx.ctx, x0, 1, prec)
        rp = F.fit_context(ctx, x0, 1, prec)
        sig = F.sigmas_context(ctx, rp["x"], 1)
    assert rn["status"] == 0 and rp["status"] == 0
    assert np.all(np.abs(rn["x"] - rp["x"]) / sig < 0.01)
