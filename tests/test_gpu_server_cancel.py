"""Serving loop: bounded waits and cancellation (host logic, no GPU fault).

* musr_server_wait with a short timeout returns MUSR_ETIMEOUT while the fit runs; the fit
  still completes, and a later wait takes its result.
* A queued fit that is canceled ends at once without running: status MUSR_ECANCELED, its
  start point as the result.
* A running fit that is canceled ends at its next step boundary with MUSR_ECANCELED, its
  memory goes back to the budget, and the server keeps serving other fits.
* Canceling a finished fit leaves its result (MUSR_ESTATE); unknown ids are refused.
"""
import time

import numpy as np
import pytest

import musr_inputs as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _long_fit_problem():
    # FP64 path, 8 x 65536 bins: each evaluation takes a fraction of a millisecond
    return mi.cfg2(nhist=8, nbins=65536, seed=401)


def test_wait_times_out_then_the_fit_completes(B):
    p = _long_fit_problem()
    with B.Server(hbm_budget_bytes=1 << 30, max_active=4) as srv:
        fid = srv.submit(p, mi.start_point(p, 1), B.MUSR_MLE, B.MUSR_FP64)
        st = B.load().musr_server_wait(srv.srv, fid, 1, None, None)
        assert st == B.MUSR_ETIMEOUT
        r = srv.wait(fid, timeout_ms=120000)
        assert r is not None and r["status"] == 0, r


def test_cancel_a_queued_fit(B):
    p = _long_fit_problem()
    x0 = mi.start_point(p, 2)
    with B.Server(hbm_budget_bytes=1 << 30, max_active=1) as srv:
        first = srv.submit(p, mi.start_point(p, 3), B.MUSR_MLE, B.MUSR_FP64)
        second = srv.submit(p, x0, B.MUSR_MLE, B.MUSR_FP64)  # waits for the only slot
        assert srv.cancel(second) == B.MUSR_OK
        r = srv.wait(second, timeout_ms=60000)
        assert r is not None and r["status"] == B.MUSR_ECANCELED
        assert r["iters"] == 0 and np.array_equal(r["x"], x0)
        r1 = srv.wait(first, timeout_ms=120000)
        assert r1["status"] == 0
        st = srv.stats()
        assert st["canceled"] == 1 and st["completed"] == 1 and st["rejected"] == 0
        assert srv.cancel(first) == B.MUSR_EINVAL  # result already taken
        assert srv.cancel(10 ** 9) == B.MUSR_EINVAL


def test_cancel_a_running_fit_and_keep_serving(B):
    # 64 histograms, 196 parameters on the FP64 path: the minimiser's first step alone (the
    # curvature estimate, one point per parameter) keeps the device busy for a good part of
    # a second, so the cancel below reaches a fit that has launched
    p = mi.cfg2(nhist=64, nbins=65536, seed=403, n0=20.0)
    with B.Server(hbm_budget_bytes=2 << 30, max_active=4) as srv:
        fid = srv.submit(p, mi.start_point(p, 4), B.MUSR_MLE, B.MUSR_FP64)
        t = time.perf_counter()
        while srv.stats()["active"] < 1 and time.perf_counter() - t < 30.0:
            time.sleep(0.001)
        time.sleep(0.05)
        assert srv.cancel(fid) == B.MUSR_OK
        r = srv.wait(fid, timeout_ms=60000)
        assert r is not None and r["status"] == B.MUSR_ECANCELED, r
        assert r["nfev"] > 0 and np.all(np.isfinite(r["x"]))
        st = srv.stats()
        assert st["active"] == 0 and st["canceled"] == 1
        t = time.perf_counter()
        while srv.stats()["arena_used"] != 0 and time.perf_counter() - t < 5.0:
            time.sleep(0.001)
        assert srv.stats()["arena_used"] == 0  # its memory went back to the budget
        q = mi.cfg3(nhist=2, nbins=4000, bin_width_ns=3.0, seed=402)
        fid2 = srv.submit(q, mi.start_point(q, 5), B.MUSR_CHI2, B.MUSR_SPLIT)
        r2 = srv.wait(fid2, timeout_ms=60000)
        assert r2["status"] == 0
        # a finished fit whose result has not been taken: canceling it changes nothing
        done = srv.stats()["completed"]
        fid3 = srv.submit(q, mi.start_point(q, 6), B.MUSR_CHI2, B.MUSR_SPLIT)
        t = time.perf_counter()
        while srv.stats()["completed"] == done and time.perf_counter() - t < 60.0:
            time.sleep(0.001)
        assert srv.cancel(fid3) == B.MUSR_ESTATE
        r3 = srv.wait(fid3, timeout_ms=60000)
        assert r3["status"] == 0
