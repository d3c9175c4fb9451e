"""Thin ctypes binding of libmusr (``include/musr.h``): argument marshalling only.

Every function named ``musr_*`` here calls the C entry point of the same name;
all arithmetic of the cost runs in the library's CUDA kernels.  The library is
built in-tree (``paper_1509_07685_gb300/libmusr.so``) by ``build.py``; if it
is missing, :func:`load` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmusr.so")

MUSR_OK, MUSR_EINVAL, MUSR_ENOMEM, MUSR_ECUDA = 0, -1, -2, -3
MUSR_ENONFINITE, MUSR_ETIMEOUT, MUSR_ESTATE, MUSR_EAGAIN, MUSR_ECANCELED = -4, -5, -6, -7, -8
MUSR_DTYPE_INT32, MUSR_DTYPE_FP32, MUSR_DTYPE_FP64 = 0, 1, 2
MUSR_REQ_BORROW_COUNTS = 1  # musr_fit_request.flags: the server reads the caller's counts at admission
MUSR_CHI2, MUSR_MLE = 0, 1
MUSR_FP64, MUSR_SPLIT = 0, 1
PRIM = {"AMP": 1, "EXP": 2, "GAUSS": 3, "KT": 4, "TFCOS": 5, "LKT": 6, "STREXP": 7, "BESSEL": 8, "DKT": 9}
MAX_PRIMS = 4

# Every symbol include/musr.h declares (checked by the ABI test).
EXPORTS = (
    "musr_ctx_create", "musr_ctx_destroy", "musr_last_error", "musr_upload_histograms",
    "musr_upload_asymmetry", "musr_upload_histograms_device", "musr_set_theory", "musr_set_map", "musr_eval",
    "musr_eval_batch", "musr_eval_device", "musr_sync", "musr_bins_in_fit", "musr_gn_product",
    "musr_gauss_newton",
    "musr_launches_per_eval", "musr_debug_word", "musr_eval_noalloc", "musr_binary_version", "musr_fit", "musr_server_create",
    "musr_server_destroy", "musr_server_submit", "musr_server_poll", "musr_server_wait",
    "musr_server_cancel", "musr_server_stats_get", "musr_poisson_create", "musr_poisson_destroy", "musr_poisson_last_error",
    "musr_poisson_solve", "musr_poisson_solve_device",
)


class MusrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmusr status {status}: {msg}")
        self.status = status


class musr_term(ctypes.Structure):
    _fields_ = [("nprim", ctypes.c_int32), ("kind", ctypes.c_int32 * MAX_PRIMS),
                ("slot", (ctypes.c_int32 * 2) * MAX_PRIMS)]


class musr_fit_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("nfev", ctypes.c_int32),
                ("nparams", ctypes.c_int32), ("f", ctypes.c_double), ("edm", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class musr_fit_request(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("nhist", ctypes.c_int32),
                ("nbins", ctypes.c_int64), ("t0", ctypes.POINTER(ctypes.c_double)),
                ("bin_width_ns", ctypes.c_double), ("fit_range_us", ctypes.c_double * 2),
                ("terms", ctypes.POINTER(musr_term)), ("nterms", ctypes.c_int32), ("nslots", ctypes.c_int32),
                ("map", ctypes.POINTER(ctypes.c_int32)), ("nparams", ctypes.c_int32),
                ("nconsts", ctypes.c_int32), ("consts", ctypes.POINTER(ctypes.c_double)),
                ("x0", ctypes.POINTER(ctypes.c_double)), ("mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("maxit", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("gtol", ctypes.c_double)]


class musr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("canceled", ctypes.c_int64), ("steps", ctypes.c_int64), ("launches", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("active", ctypes.c_int64), ("queued", ctypes.c_int64), ("bin_evals", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("clock_s", ctypes.c_double), ("arena_bytes", ctypes.c_uint64),
                ("arena_used", ctypes.c_uint64), ("minimizer_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("wait_s", ctypes.c_double), ("cfg_create_s", ctypes.c_double),
                ("cfg_upload_s", ctypes.c_double), ("cfg_plan_s", ctypes.c_double),
                ("cfg_buffers_s", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def _declare(lib):
    P = ctypes.POINTER
    vp, d, i32, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64
    sig = {
        "musr_ctx_create": ([P(vp), ctypes.c_int, ctypes.c_size_t, vp], ctypes.c_int),
        "musr_ctx_destroy": ([vp], None),
        "musr_last_error": ([vp], ctypes.c_char_p),
        "musr_upload_histograms": ([vp, vp, ctypes.c_int, ctypes.c_int, i64, P(d), d, P(d)], ctypes.c_int),
        "musr_poisson_create": ([P(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d, d,
                                 ctypes.c_int, vp], ctypes.c_int),
        "musr_poisson_destroy": ([vp], None),
        "musr_poisson_last_error": ([vp], ctypes.c_char_p),
        "musr_poisson_solve": ([vp, P(d), P(d)], ctypes.c_int),
        "musr_poisson_solve_device": ([vp, vp, vp], ctypes.c_int),
        "musr_upload_asymmetry": ([vp, vp, vp, ctypes.c_int, ctypes.c_int, i64, P(d), d, P(d), P(d), P(d), P(d)],
                                  ctypes.c_int),
        "musr_upload_histograms_device": ([vp, vp, ctypes.c_int, ctypes.c_int, i64, i64, P(d), d, P(d)],
                                          ctypes.c_int),
        "musr_set_theory": ([vp, P(musr_term), ctypes.c_int], ctypes.c_int),
        "musr_set_map": ([vp, P(i32), ctypes.c_int, ctypes.c_int, P(d), ctypes.c_int], ctypes.c_int),
        "musr_eval": ([vp, P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d), P(d)], ctypes.c_int),
        "musr_eval_batch": ([vp, P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d), P(d)],
                            ctypes.c_int),
        "musr_eval_device": ([vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp], ctypes.c_int),
        "musr_sync": ([vp, ctypes.c_int], ctypes.c_int),
        "musr_gn_product": ([vp, P(d), ctypes.c_int, P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d)],
                            ctypes.c_int),
        "musr_gauss_newton": ([vp, P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(d)], ctypes.c_int),
        "musr_bins_in_fit": ([vp, P(i64)], ctypes.c_int),
        "musr_launches_per_eval": ([vp, P(ctypes.c_int)], ctypes.c_int),
        "musr_debug_word": ([vp, P(ctypes.c_uint32)], ctypes.c_int),
        "musr_eval_noalloc": ([vp, ctypes.c_int, ctypes.c_int, i64, i64, P(d), d, P(d), P(musr_term),
                               ctypes.c_int, P(i32), ctypes.c_int, ctypes.c_int, P(d), ctypes.c_int, vp,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
        "musr_binary_version": ([ctypes.c_int, P(ctypes.c_int)], ctypes.c_int),
        "musr_fit": ([vp, P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, d, P(d), P(musr_fit_result)],
                     ctypes.c_int),
        "musr_server_create": ([P(vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_int], ctypes.c_int),
        "musr_server_destroy": ([vp], None),
        "musr_server_submit": ([vp, P(musr_fit_request), P(i64)], ctypes.c_int),
        "musr_server_poll": ([vp, i64, P(musr_fit_result), P(d)], ctypes.c_int),
        "musr_server_wait": ([vp, i64, ctypes.c_int, P(musr_fit_result), P(d)], ctypes.c_int),
        "musr_server_cancel": ([vp, i64], ctypes.c_int),
        "musr_server_stats_get": ([vp, P(musr_server_stats)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


def load():
    """The loaded libmusr; raises if the library has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                                   "(there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            _declare(lib)
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _err(ctx, status: int):
    msg = load().musr_last_error(ctx)
    raise MusrError(status, msg.decode() if msg else "")


def _check(ctx, status: int):
    if status != MUSR_OK:
        _err(ctx, status)


def terms_to_c(terms) -> Tuple[ctypes.Array, int]:
    """Term list [[(kind, slots), ...], ...] -> musr_term array."""
    n = len(terms)
    arr = (musr_term * max(n, 1))()
    for k, term in enumerate(terms):
        if len(term) > MAX_PRIMS:
            raise ValueError("a term holds at most 4 primitives")
        arr[k].nprim = len(term)
        for m, (kind, slots) in enumerate(term):
            arr[k].kind[m] = PRIM[kind]
            for q, s in enumerate(slots):
                arr[k].slot[m][q] = int(s)
    return arr, n


# --------------------------------------------------------------------------------------------
# Functions with the C names
# --------------------------------------------------------------------------------------------

CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the handle of the legacy default stream


def musr_ctx_create(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: Optional[int] = None):
    """cuda_stream: None -> the context creates its own stream; an int handle (e.g.
    torch.cuda.current_stream().cuda_stream) -> run on that stream, where torch's
    handle 0 (the legacy default stream) is passed on as cudaStreamLegacy."""
    lib = load()
    out = ctypes.c_void_p()
    if cuda_stream is None:
        handle = None
    else:
        handle = ctypes.c_void_p(cuda_stream if cuda_stream != 0 else CUDA_STREAM_LEGACY)
    st = lib.musr_ctx_create(ctypes.byref(out), device, hbm_budget_bytes, handle)
    if st != MUSR_OK:
        raise MusrError(st, (lib.musr_last_error(None) or b"").decode())
    return out


def musr_ctx_destroy(ctx) -> None:
    load().musr_ctx_destroy(ctx)


def musr_last_error(ctx) -> str:
    msg = load().musr_last_error(ctx)
    return msg.decode() if msg else ""


def musr_upload_histograms(ctx, counts: np.ndarray, t0: Sequence[float], bin_width_ns: float,
                           fit_range_us: Sequence[float]) -> None:
    counts = np.ascontiguousarray(counts)
    if counts.ndim != 2:
        raise ValueError("counts must be [nhist][nbins]")
    dtype = {np.dtype(np.int32): MUSR_DTYPE_INT32, np.dtype(np.float32): MUSR_DTYPE_FP32,
             np.dtype(np.float64): MUSR_DTYPE_FP64}.get(counts.dtype)
    if dtype is None:
        raise TypeError("counts must be int32, float32 or float64")
    t0 = np.ascontiguousarray(t0, dtype=np.float64)
    fr = np.ascontiguousarray(fit_range_us, dtype=np.float64)
    _check(ctx, load().musr_upload_histograms(ctx, counts.ctypes.data_as(ctypes.c_void_p), dtype,
                                              counts.shape[0], counts.shape[1], _dptr(t0),
                                              float(bin_width_ns), _dptr(fr)))


def musr_upload_asymmetry(ctx, forward: np.ndarray, backward: np.ndarray, t0: Sequence[float], bin_width_ns: float,
                          fit_range_us: Sequence[float], alpha: Sequence[float], bkg_forward: Sequence[float],
                          bkg_backward: Sequence[float]) -> None:
    F = np.ascontiguousarray(forward)
    Bk = np.ascontiguousarray(backward, dtype=F.dtype)
    if F.ndim != 2 or Bk.shape != F.shape:
        raise ValueError("forward and backward must both be [npairs][nbins]")
    dtype = {np.dtype(np.int32): MUSR_DTYPE_INT32, np.dtype(np.float32): MUSR_DTYPE_FP32,
             np.dtype(np.float64): MUSR_DTYPE_FP64}.get(F.dtype)
    if dtype is None:
        raise TypeError("counts must be int32, float32 or float64")
    H = F.shape[0]
    t0 = np.ascontiguousarray(t0, dtype=np.float64).reshape(H)
    fr = np.ascontiguousarray(fit_range_us, dtype=np.float64)
    al = np.ascontiguousarray(alpha, dtype=np.float64).reshape(H)
    bf = np.ascontiguousarray(bkg_forward, dtype=np.float64).reshape(H)
    bb = np.ascontiguousarray(bkg_backward, dtype=np.float64).reshape(H)
    _check(ctx, load().musr_upload_asymmetry(ctx, F.ctypes.data_as(ctypes.c_void_p), Bk.ctypes.data_as(ctypes.c_void_p),
                                             dtype, H, F.shape[1], _dptr(t0), float(bin_width_ns), _dptr(fr),
                                             _dptr(al), _dptr(bf), _dptr(bb)))


def musr_upload_histograms_device(ctx, d_counts: int, dtype: int, nhist: int, nbins: int, row_stride: int,
                                  t0: Sequence[float], bin_width_ns: float,
                                  fit_range_us: Sequence[float]) -> None:
    t0 = np.ascontiguousarray(t0, dtype=np.float64)
    fr = np.ascontiguousarray(fit_range_us, dtype=np.float64)
    _check(ctx, load().musr_upload_histograms_device(ctx, ctypes.c_void_p(d_counts), dtype, nhist, nbins,
                                                     row_stride, _dptr(t0), float(bin_width_ns), _dptr(fr)))


def musr_set_theory(ctx, terms) -> None:
    arr, n = terms_to_c(terms)
    _check(ctx, load().musr_set_theory(ctx, arr, n))


def musr_set_map(ctx, mp: np.ndarray, nparams: int, consts: Sequence[float] = ()) -> None:
    mp = np.ascontiguousarray(mp, dtype=np.int32)
    c = np.ascontiguousarray(consts if len(consts) else np.zeros(1), dtype=np.float64)
    _check(ctx, load().musr_set_map(ctx, mp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), mp.shape[1],
                                    int(nparams), _dptr(c), len(consts)))


def musr_eval(ctx, params: np.ndarray, mode: int, precision: int, grad: bool = True):
    """(value, grad or None, status); status is MUSR_OK or MUSR_ENONFINITE (value +inf)."""
    x = np.ascontiguousarray(params, dtype=np.float64)
    v = ctypes.c_double()
    g = np.zeros(x.size) if grad else None
    st = load().musr_eval(ctx, _dptr(x), x.size, mode, precision, ctypes.byref(v),
                          _dptr(g) if grad else None)
    if st not in (MUSR_OK, MUSR_ENONFINITE):
        _err(ctx, st)
    return v.value, g, st


def musr_eval_batch(ctx, params: np.ndarray, mode: int, precision: int, grad: bool = True):
    """(values[nvec], grads[nvec][P] or None, status)."""
    x = np.ascontiguousarray(np.atleast_2d(params), dtype=np.float64)
    nvec, P = x.shape
    vals = np.zeros(nvec)
    g = np.zeros((nvec, P)) if grad else None
    st = load().musr_eval_batch(ctx, _dptr(x), nvec, P, mode, precision, _dptr(vals),
                                _dptr(g) if grad else None)
    if st not in (MUSR_OK, MUSR_ENONFINITE):
        _err(ctx, st)
    return vals, g, st


def musr_gn_product(ctx, params, dirs, mode: int, precision: int):
    """(vHv[ndir], Hv[ndir][P], status): Gauss-Newton products at params along each row of dirs."""
    x = np.ascontiguousarray(params, dtype=np.float64)
    v = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    ndir, P = v.shape
    out = np.zeros((ndir, 1 + P))
    st = load().musr_gn_product(ctx, _dptr(x), P, _dptr(v), ndir, mode, precision, _dptr(out))
    if st not in (MUSR_OK, MUSR_ENONFINITE):
        _err(ctx, st)
    return out[:, 0].copy(), out[:, 1:].copy(), st


def musr_gauss_newton(ctx, params, mode: int, precision: int) -> np.ndarray:
    """The Gauss-Newton matrix [P][P] of the cost at params."""
    x = np.ascontiguousarray(params, dtype=np.float64)
    P = x.size
    out = np.zeros((P, P))
    _check(ctx, load().musr_gauss_newton(ctx, _dptr(x), P, mode, precision, _dptr(out)))
    return out


def musr_eval_device(ctx, d_params: int, nvec: int, mode: int, precision: int, with_grad: bool,
                     d_out: int) -> None:
    _check(ctx, load().musr_eval_device(ctx, ctypes.c_void_p(d_params), nvec, mode, precision,
                                        int(bool(with_grad)), ctypes.c_void_p(d_out)))


def musr_sync(ctx, timeout_ms: int = 0) -> None:
    _check(ctx, load().musr_sync(ctx, timeout_ms))


def musr_bins_in_fit(ctx) -> int:
    out = ctypes.c_int64()
    _check(ctx, load().musr_bins_in_fit(ctx, ctypes.byref(out)))
    return out.value


def musr_debug_word(ctx):
    """(status, the error word of the kernels' index checks); MUSR_ESTATE in a release build."""
    out = ctypes.c_uint32(0)
    st = load().musr_debug_word(ctx, ctypes.byref(out))
    return st, out.value


def musr_launches_per_eval(ctx) -> int:
    out = ctypes.c_int()
    _check(ctx, load().musr_launches_per_eval(ctx, ctypes.byref(out)))
    return out.value


def musr_eval_noalloc(d_counts: int, dtype: int, nhist: int, nbins: int, row_stride: int,
                      t0: Sequence[float], bin_width_ns: float, fit_range_us: Sequence[float], terms,
                      mp: np.ndarray, nparams: int, consts: Sequence[float], d_params: int, mode: int,
                      precision: int, with_grad: bool, d_out: int, cuda_stream: Optional[int] = None) -> int:
    """The allocation-free evaluation (device pointers in and out); returns the status."""
    t0 = np.ascontiguousarray(t0, dtype=np.float64)
    fr = np.ascontiguousarray(fit_range_us, dtype=np.float64)
    arr, n = terms_to_c(terms)
    mp = np.ascontiguousarray(mp, dtype=np.int32)
    # the library reads map[nhist][nslots], t0[nhist] and the fit range's two ends
    if mp.ndim != 2 or mp.shape[0] != nhist or t0.shape != (nhist,) or fr.shape != (2,):
        raise ValueError("musr_eval_noalloc: map must be [nhist][nslots], t0 [nhist], fit_range_us [2]")
    c = np.ascontiguousarray(consts if len(consts) else np.zeros(1), dtype=np.float64)
    stream = None if not cuda_stream else ctypes.c_void_p(cuda_stream)
    return load().musr_eval_noalloc(ctypes.c_void_p(d_counts), dtype, nhist, nbins, row_stride, _dptr(t0),
                                    float(bin_width_ns), _dptr(fr), arr, n,
                                    mp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), mp.shape[1],
                                    int(nparams), _dptr(c), len(consts), ctypes.c_void_p(d_params), mode,
                                    precision, int(bool(with_grad)), ctypes.c_void_p(d_out), stream)


def musr_binary_version(device: int = 0):
    """(status, compute capability the loaded kernels were built for: 103 for sm_103a)."""
    out = ctypes.c_int(-1)
    st = load().musr_binary_version(int(device), ctypes.byref(out))
    return st, out.value


# --------------------------------------------------------------------------------------------
# Convenience owner object
# --------------------------------------------------------------------------------------------

class Context:
    """Owns one musr_ctx configured for one problem (histograms, theory, map).

    ``problem`` needs: counts [H][B], t0 [H], bin_width_ns, fit_range_us, terms,
    map [H][nslots], consts, nparams.
    """

    def __init__(self, problem=None, device: int = 0, hbm_budget_bytes: int = 0,
                 cuda_stream: Optional[int] = None):
        self.ctx = musr_ctx_create(device, hbm_budget_bytes, cuda_stream)
        self.P = None
        if problem is not None:
            self.configure(problem)

    def configure(self, problem) -> None:
        if hasattr(problem, "forward"):  # asymmetry data (forward / backward pairs)
            musr_upload_asymmetry(self.ctx, problem.forward, problem.backward, problem.t0, problem.bin_width_ns,
                                  problem.fit_range_us, problem.alpha, problem.bkg_f, problem.bkg_b)
        else:
            musr_upload_histograms(self.ctx, problem.counts, problem.t0, problem.bin_width_ns,
                                   problem.fit_range_us)
        musr_set_theory(self.ctx, problem.terms)
        musr_set_map(self.ctx, problem.map, problem.nparams, problem.consts)
        self.P = int(problem.nparams)

    def eval(self, x, mode=MUSR_CHI2, precision=MUSR_FP64, grad=True):
        return musr_eval(self.ctx, x, mode, precision, grad)

    def eval_batch(self, X, mode=MUSR_CHI2, precision=MUSR_FP64, grad=True):
        return musr_eval_batch(self.ctx, X, mode, precision, grad)

    def gauss_newton(self, x, mode=MUSR_CHI2, precision=MUSR_FP64) -> np.ndarray:
        return musr_gauss_newton(self.ctx, x, mode, precision)

    def gn_product(self, x, dirs, mode=MUSR_CHI2, precision=MUSR_FP64):
        return musr_gn_product(self.ctx, x, dirs, mode, precision)

    def bins_in_fit(self) -> int:
        return musr_bins_in_fit(self.ctx)

    def close(self) -> None:
        if self.ctx:
            musr_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------------------------------------
# Fitting and serving
# --------------------------------------------------------------------------------------------

def _result_dict(r: "musr_fit_result", x: np.ndarray) -> dict:
    return {"status": r.status, "iters": r.iters, "nfev": r.nfev, "f": r.f, "edm": r.edm, "x": x,
            "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}


def musr_fit(ctx, x0, mode: int, precision: int, maxit: int = 0, gtol: float = 0.0) -> dict:
    """The native BFGS fit on a configured context (synchronous)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    x = np.zeros_like(x0)
    r = musr_fit_result()
    _check(ctx, load().musr_fit(ctx, _dptr(x0), mode, precision, maxit, gtol, _dptr(x), ctypes.byref(r)))
    return _result_dict(r, x)


def musr_server_create(device: int = 0, hbm_budget_bytes: int = 8 << 30, max_active: int = 1024):
    out = ctypes.c_void_p()
    st = load().musr_server_create(ctypes.byref(out), device, hbm_budget_bytes, max_active)
    if st != MUSR_OK:
        raise MusrError(st, "musr_server_create failed")
    return out


def musr_server_destroy(srv) -> None:
    load().musr_server_destroy(srv)


def make_request(problem, x0, mode: int, precision: int, maxit: int = 0, gtol: float = 0.0, borrow: bool = False):
    """A musr_fit_request for a problem; returns (request, keepalive).  The arrays must live
    until musr_server_submit returns (it copies them); with borrow the counts are lent to
    the server (MUSR_REQ_BORROW_COUNTS) and must live, unchanged, until the result is taken."""
    counts = np.ascontiguousarray(problem.counts)
    dtype = {np.dtype(np.int32): MUSR_DTYPE_INT32, np.dtype(np.float32): MUSR_DTYPE_FP32,
             np.dtype(np.float64): MUSR_DTYPE_FP64}[counts.dtype]
    t0 = np.ascontiguousarray(problem.t0, dtype=np.float64)
    terms, nterms = terms_to_c(problem.terms)
    mp = np.ascontiguousarray(problem.map, dtype=np.int32)
    consts = np.ascontiguousarray(problem.consts if len(problem.consts) else np.zeros(1), dtype=np.float64)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    q = musr_fit_request()
    q.counts = counts.ctypes.data_as(ctypes.c_void_p)
    q.dtype = dtype
    q.nhist, q.nbins = counts.shape
    q.t0 = _dptr(t0)
    q.bin_width_ns = float(problem.bin_width_ns)
    q.fit_range_us[0], q.fit_range_us[1] = problem.fit_range_us
    q.terms = ctypes.cast(terms, ctypes.POINTER(musr_term))
    q.nterms = nterms
    q.nslots = mp.shape[1]
    q.map = mp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    q.nparams = int(problem.nparams)
    q.nconsts = len(problem.consts)
    q.consts = _dptr(consts)
    q.x0 = _dptr(x0)
    q.mode, q.precision, q.maxit, q.gtol = mode, precision, maxit, gtol
    q.flags = MUSR_REQ_BORROW_COUNTS if borrow else 0
    return q, (counts, t0, terms, mp, consts, x0)


def musr_server_submit(srv, problem, x0, mode: int, precision: int, maxit: int = 0, gtol: float = 0.0,
                       borrow: bool = False):
    """Submits one fit; returns (id, lent) -- lent is the counts array the server borrowed
    (None without borrow), which the caller keeps until the result is taken."""
    q, keep = make_request(problem, x0, mode, precision, maxit, gtol, borrow)
    fid = ctypes.c_int64()
    st = load().musr_server_submit(srv, ctypes.byref(q), ctypes.byref(fid))
    if st != MUSR_OK:
        raise MusrError(st, "musr_server_submit rejected the request")
    return fid.value, (keep[0] if borrow else None)


def musr_server_poll(srv, fid: int, nparams: int):
    r = musr_fit_result()
    x = np.zeros(nparams)
    st = load().musr_server_poll(srv, fid, ctypes.byref(r), _dptr(x))
    if st == MUSR_EAGAIN:
        return None
    if st != MUSR_OK:
        raise MusrError(st, "musr_server_poll failed")
    return _result_dict(r, x)


def musr_server_wait(srv, fid: int, nparams: int, timeout_ms: int = 0):
    r = musr_fit_result()
    x = np.zeros(nparams)
    st = load().musr_server_wait(srv, fid, timeout_ms, ctypes.byref(r), _dptr(x))
    if st == MUSR_ETIMEOUT:
        return None
    if st != MUSR_OK:
        raise MusrError(st, "musr_server_wait failed")
    return _result_dict(r, x)


def musr_server_cancel(srv, fid: int) -> int:
    """Asks fit `fid` to stop; returns the status (MUSR_OK, MUSR_ESTATE if it had finished)."""
    return load().musr_server_cancel(srv, int(fid))


def musr_server_stats_get(srv) -> dict:
    s = musr_server_stats()
    st = load().musr_server_stats_get(srv, ctypes.byref(s))
    if st != MUSR_OK:
        raise MusrError(st, "musr_server_stats_get failed")
    return {name: getattr(s, name) for name, _ in s._fields_}


class Server:
    """Owns one musr_server (continuous batching of many fits).  submit lends each fit's
    counts to the server (no copy) and keeps the array referenced until the result has been
    taken; the caller must not modify it meanwhile (borrow=False copies instead)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 8 << 30, max_active: int = 1024):
        self.srv = musr_server_create(device, hbm_budget_bytes, max_active)
        self.nparams = {}
        self.lent = {}

    def submit(self, problem, x0, mode=MUSR_MLE, precision=MUSR_SPLIT, maxit=0, gtol=0.0, borrow=True) -> int:
        fid, lent = musr_server_submit(self.srv, problem, x0, mode, precision, maxit, gtol, borrow)
        self.nparams[fid] = int(problem.nparams)
        if lent is not None:
            self.lent[fid] = lent
        return fid

    def poll(self, fid: int):
        r = musr_server_poll(self.srv, fid, self.nparams[fid])
        if r is not None:
            self.nparams.pop(fid, None)
            self.lent.pop(fid, None)
        return r

    def wait(self, fid: int, timeout_ms: int = 0):
        r = musr_server_wait(self.srv, fid, self.nparams[fid], timeout_ms)
        if r is not None:
            self.nparams.pop(fid, None)
            self.lent.pop(fid, None)
        return r

    def cancel(self, fid: int) -> int:
        """Asks fit `fid` to stop (its result, taken with poll / wait, has status
        MUSR_ECANCELED); returns the status of the request."""
        return musr_server_cancel(self.srv, fid)

    def stats(self) -> dict:
        return musr_server_stats_get(self.srv)

    def close(self) -> None:
        if self.srv:
            musr_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Poisson:
    """Owns one musr_poisson: the open-boundary particle-mesh Poisson solve of Section 3 on an
    (mx, my, mz) mesh with spacings h = (hx, hy, hz); precision MUSR_FP64 (FP64 transforms) or
    MUSR_SPLIT (FP32 transforms)."""

    def __init__(self, shape, h, precision: int = MUSR_FP64, device: int = 0, cuda_stream: Optional[int] = None):
        self.shape = tuple(int(v) for v in shape)
        out = ctypes.c_void_p()
        st = load().musr_poisson_create(ctypes.byref(out), device, *self.shape, float(h[0]), float(h[1]),
                                        float(h[2]), int(precision),
                                        ctypes.c_void_p(cuda_stream) if cuda_stream else None)
        if st != MUSR_OK:
            msg = load().musr_poisson_last_error(None)
            raise MusrError(st, msg.decode() if msg else "musr_poisson_create failed")
        self.ps = out

    def _check(self, st):
        if st != MUSR_OK:
            msg = load().musr_poisson_last_error(self.ps)
            raise MusrError(st, msg.decode() if msg else "musr_poisson call failed")

    def solve(self, rho: np.ndarray) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        if rho.shape != self.shape:
            raise ValueError(f"rho must have shape {self.shape}")
        phi = np.empty_like(rho)
        self._check(load().musr_poisson_solve(self.ps, _dptr(rho), _dptr(phi)))
        return phi

    def solve_device(self, d_rho: int, d_phi: int) -> None:
        self._check(load().musr_poisson_solve_device(self.ps, ctypes.c_void_p(d_rho), ctypes.c_void_p(d_phi)))

    def close(self) -> None:
        if self.ps:
            load().musr_poisson_destroy(self.ps)
            self.ps = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
