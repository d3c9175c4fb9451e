"""Plain FP64 CPU oracle for the muSR chi^2 / -2lnL cost (arXiv 1509.07685, Section 4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_1509_07685_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``musr_oracle.cpp`` (single-threaded C++17, FP64,
Neumaier-compensated sums, no -ffast-math).  This module only builds that file
with g++ and marshals numpy arrays into it.

Every function here follows Section 4.1 of the paper:
  * Eq. positron_histo  -- :func:`model`
  * Eq. chisq           -- :func:`cost` with ``mode=0``
  * Eq. log-likelihood  -- :func:`cost` with ``mode=1``
  * Eq. asymmetry       -- :func:`primitive` (the primitive factors of A(t)), and
                           :func:`dkt` (the dynamic Kubo-Toyabe relaxation, a renewal
                           equation solved on a grid; a "user defined function" of 4.1)
  * the host-side minimiser that replaces migrad -- :func:`fit`
  * the Gauss-Newton matrix of the cost (error estimates) -- :func:`gauss_newton`

Pins (see ``tests/test_oracle_*.py``): closed-form sums of exponential and
damped-cosine models, constant models, Kubo-Toyabe special values, the
complex-step derivative, exact summation, and fits of event-level Monte Carlo
data against the truth.  Parity is pinned for every function exported here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "musr_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_musr_oracle.so")
_lock = threading.Lock()
_lib = None

KIND = {"AMP": 1, "EXP": 2, "GAUSS": 3, "KT": 4, "TFCOS": 5, "LKT": 6, "STREXP": 7, "BESSEL": 8, "DKT": 9}
CHI2, MLE = 0, 1


def build(force: bool = False) -> str:
    """Compile musr_oracle.cpp into _musr_oracle.so (g++, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
             "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # MUSR_ORACLE_LIB: another build of this file (the mutation test plants
            # mistakes in a copy of the source to show that the pins catch them).
            path = os.environ.get("MUSR_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            prob = [P(d), ctypes.c_int, i64, P(d), d, d, d, ctypes.c_int, P(i32), P(i32), P(i32),
                    P(i32), ctypes.c_int, P(d), ctypes.c_int, ctypes.c_int, P(d), ctypes.c_int]
            lib.oracle_primitive.argtypes = [ctypes.c_int, d, d, d]
            lib.oracle_primitive.restype = d
            lib.oracle_model.argtypes = prob + [P(d), ctypes.c_int, d]
            lib.oracle_model.restype = d
            lib.oracle_cost.argtypes = prob + [P(d), ctypes.c_int, P(d), P(d), P(d)]
            lib.oracle_cost.restype = ctypes.c_int
            lib.oracle_cost_cstep.argtypes = prob + [P(d), P(d), d, ctypes.c_int, P(d)]
            lib.oracle_cost_cstep.restype = ctypes.c_int
            lib.oracle_hessian.argtypes = prob + [P(d), P(d), ctypes.c_int, P(d)]
            lib.oracle_hessian.restype = ctypes.c_int
            lib.oracle_gauss_newton.argtypes = prob + [P(d), ctypes.c_int, P(d)]
            lib.oracle_gauss_newton.restype = ctypes.c_int
            lib.oracle_fit.argtypes = prob + [ctypes.c_int, P(d), P(d), ctypes.c_int, d, P(d), P(d),
                                              P(d), P(ctypes.c_int)]
            lib.oracle_fit.restype = ctypes.c_int
            lib.oracle_poisson_direct.argtypes = [P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d, d, P(d)]
            lib.oracle_poisson_direct.restype = None
            lib.oracle_poisson_points.argtypes = [P(d), ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d, d, P(i32),
                                                  ctypes.c_int, P(d)]
            lib.oracle_poisson_points.restype = None
            lib.oracle_asymmetry.argtypes = [P(d), P(d), ctypes.c_int, i64, P(d), P(d), P(d), P(d), P(d)]
            lib.oracle_asymmetry.restype = None
            lib.oracle_dkt.argtypes = [d, d, d, P(d), ctypes.c_int, P(d), P(d), P(d)]
            lib.oracle_dkt.restype = ctypes.c_int
            lib.oracle_neumaier_sum.argtypes = [P(d), i64]
            lib.oracle_neumaier_sum.restype = d
            _lib = lib
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def theory_arrays(terms):
    """Term list -> (nprim[T], kind[T,4], slot[T,4,2]) int32 arrays.

    ``terms`` is a sequence of terms; a term is a sequence of (kind, slots)
    with kind in AMP, EXP, GAUSS, KT, TFCOS, LKT, STREXP, BESSEL, DKT and slots a tuple of
    local slot indices (two for TFCOS and BESSEL: frequency, phase; two for STREXP: rate,
    exponent; two for DKT: static width, fluctuation rate; one otherwise).
    """
    T = len(terms)
    nprim = np.zeros(max(T, 1), np.int32)
    kind = np.zeros((max(T, 1), 4), np.int32)
    slot = np.zeros((max(T, 1), 4, 2), np.int32)
    for k, term in enumerate(terms):
        if len(term) > 4:
            raise ValueError("a term has at most 4 primitives")
        nprim[k] = len(term)
        for m, (kname, slots) in enumerate(term):
            kind[k, m] = KIND[kname]
            for q, s in enumerate(slots):
                slot[k, m, q] = s
    return nprim, kind, slot


class _Args:
    """Keeps the marshalled arrays alive for one call.  Asymmetry problems (forward /
    backward pairs) enter as their asymmetry values and weights, computed here by
    oracle_asymmetry, with the decay envelope off."""

    def __init__(self, prob):
        if hasattr(prob, "forward"):
            self.data, self.weight = asymmetry(prob.forward, prob.backward, prob.alpha, prob.bkg_f, prob.bkg_b)
            envelope = 0
        else:
            self.data = np.ascontiguousarray(prob.counts, dtype=np.float64)
            self.weight = None
            envelope = 1
        H, B = self.data.shape
        self.t0 = np.ascontiguousarray(prob.t0, dtype=np.float64).reshape(H)
        self.nprim, self.kind, self.slot = theory_arrays(prob.terms)
        self.map = np.ascontiguousarray(prob.map, dtype=np.int32)
        if self.map.shape[0] != H:
            raise ValueError("map must have one row per histogram")
        self.consts = np.ascontiguousarray(
            prob.consts if len(prob.consts) else np.zeros(1), dtype=np.float64)
        lo, hi = prob.fit_range_us
        self.args = [
            _ptr(self.data, ctypes.c_double), H, B, _ptr(self.t0, ctypes.c_double),
            float(prob.bin_width_ns), float(lo), float(hi), len(prob.terms),
            _ptr(self.nprim, ctypes.c_int32), _ptr(self.kind, ctypes.c_int32),
            _ptr(self.slot, ctypes.c_int32), _ptr(self.map, ctypes.c_int32), self.map.shape[1],
            _ptr(self.consts, ctypes.c_double), len(prob.consts), int(prob.nparams),
            None if self.weight is None else _ptr(self.weight, ctypes.c_double), envelope]


def asymmetry(forward, backward, alpha, bkg_f, bkg_b):
    """(a, w) [H][B]: asymmetry of forward / backward pairs and its chi^2 weight 1/sigma_a^2
    (oracle_asymmetry)."""
    F = np.ascontiguousarray(forward, dtype=np.float64)
    Bk = np.ascontiguousarray(backward, dtype=np.float64)
    H, B = F.shape
    al = np.ascontiguousarray(alpha, dtype=np.float64).reshape(H)
    bf = np.ascontiguousarray(bkg_f, dtype=np.float64).reshape(H)
    bb = np.ascontiguousarray(bkg_b, dtype=np.float64).reshape(H)
    a = np.zeros((H, B))
    w = np.zeros((H, B))
    _load().oracle_asymmetry(_ptr(F, ctypes.c_double), _ptr(Bk, ctypes.c_double), H, B, _ptr(al, ctypes.c_double),
                             _ptr(bf, ctypes.c_double), _ptr(bb, ctypes.c_double), _ptr(a, ctypes.c_double),
                             _ptr(w, ctypes.c_double))
    return a, w


def primitive(kind: str, p0: float, p1: float, t: float) -> float:
    """One primitive factor of A(t) at time t (us)."""
    return _load().oracle_primitive(KIND[kind], p0, p1, t)


def dkt(delta: float, nu: float, span: float, ts, derivs: bool = False):
    """The dynamic Gaussian Kubo-Toyabe relaxation (strong-collision model) of static width
    delta and fluctuation rate nu (both 1/us) at the times ts (us), on the oracle's grid over
    [0, span] (span >= max ts): G, or (G, dG/ddelta, dG/dnu) with derivs."""
    ts = np.ascontiguousarray(np.atleast_1d(ts), dtype=np.float64)
    if ts.size and ts.max() > span:
        raise ValueError("times beyond the grid's span")
    G = np.zeros(ts.size)
    dD = np.zeros(ts.size) if derivs else None
    dn = np.zeros(ts.size) if derivs else None
    _load().oracle_dkt(float(delta), float(nu), float(span), _ptr(ts, ctypes.c_double), ts.size,
                       _ptr(G, ctypes.c_double), None if dD is None else _ptr(dD, ctypes.c_double),
                       None if dn is None else _ptr(dn, ctypes.c_double))
    return (G, dD, dn) if derivs else G


def model(prob, x, h: int, t: float) -> float:
    """Eq. positron_histo for histogram h at time t (us)."""
    a = _Args(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return _load().oracle_model(*a.args, _ptr(x, ctypes.c_double), h, float(t))


def cost(prob, x, mode: int = CHI2, grad: bool = True):
    """(value, grad or None, gscale or None, status) of Eq. chisq / Eq. log-likelihood."""
    a = _Args(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = ctypes.c_double()
    if grad:
        g = np.zeros(prob.nparams)
        gs = np.zeros(prob.nparams)
        st = _load().oracle_cost(*a.args, _ptr(x, ctypes.c_double), mode, ctypes.byref(v),
                                 _ptr(g, ctypes.c_double), _ptr(gs, ctypes.c_double))
        return v.value, g, gs, st
    st = _load().oracle_cost(*a.args, _ptr(x, ctypes.c_double), mode, ctypes.byref(v), None, None)
    return v.value, None, None, st


def cost_cstep(prob, x, v, mode: int = CHI2, h: float = 1e-30) -> float:
    """Complex-step directional derivative Im(cost(x + i h v)) / h."""
    a = _Args(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = ctypes.c_double()
    _load().oracle_cost_cstep(*a.args, _ptr(x, ctypes.c_double), _ptr(v, ctypes.c_double), h, mode,
                              ctypes.byref(out))
    return out.value


def default_steps(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return 1e-5 * np.maximum(np.abs(x), 1e-2)


def hessian(prob, x, mode: int = CHI2, steps=None) -> np.ndarray:
    """Symmetrised central-difference Hessian of the analytic gradient."""
    a = _Args(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    st = np.ascontiguousarray(default_steps(x) if steps is None else steps, dtype=np.float64)
    H = np.zeros((prob.nparams, prob.nparams))
    rc = _load().oracle_hessian(*a.args, _ptr(x, ctypes.c_double), _ptr(st, ctypes.c_double), mode,
                                _ptr(H, ctypes.c_double))
    if rc:
        raise FloatingPointError("cost is +inf near x")
    return H


def gauss_newton(prob, x, mode: int = CHI2) -> np.ndarray:
    """Gauss-Newton matrix sum_bins (d^2 cost/dN^2) J J^T, J the parameter gradient of N
    (Eq. chisq: d^2/dN^2 = 2/max(d,1); Eq. log-likelihood: 2 d / N^2)."""
    a = _Args(prob)
    x = np.ascontiguousarray(x, dtype=np.float64)
    H = np.zeros((prob.nparams, prob.nparams))
    rc = _load().oracle_gauss_newton(*a.args, _ptr(x, ctypes.c_double), mode, _ptr(H, ctypes.c_double))
    if rc:
        raise FloatingPointError("-2lnL undefined at x")
    return H


def sigmas(prob, x, mode: int = CHI2, free=None) -> np.ndarray:
    """sigma_i = sqrt(2 (H^-1)_ii): both costs are -2lnL scaled, so Delta cost = 1 is one sigma.

    ``free`` selects the parameters that are fitted (others are held fixed).
    """
    H = hessian(prob, x, mode)
    P = prob.nparams
    free = np.arange(P) if free is None else np.asarray(free)
    cov = 2.0 * np.linalg.inv(H[np.ix_(free, free)])
    out = np.full(P, np.nan)
    out[free] = np.sqrt(np.diag(cov))
    return out


def fit(prob, x0, mode: int = CHI2, maxit: int = 1000, gtol: float = 1e-8, fd_step=None):
    """BFGS fit (see oracle_fit in musr_oracle.cpp).  Returns dict(x, f, g, iters, status)."""
    a = _Args(prob)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    st = np.ascontiguousarray(default_steps(x0) if fd_step is None else fd_step, dtype=np.float64)
    x = np.zeros(prob.nparams)
    g = np.zeros(prob.nparams)
    f = ctypes.c_double()
    it = ctypes.c_int()
    status = _load().oracle_fit(*a.args, mode, _ptr(x0, ctypes.c_double), _ptr(st, ctypes.c_double),
                                maxit, gtol, _ptr(x, ctypes.c_double), ctypes.byref(f),
                                _ptr(g, ctypes.c_double), ctypes.byref(it))
    return {"x": x, "f": f.value, "g": g, "iters": it.value, "status": status}


def neumaier_sum(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _load().oracle_neumaier_sum(_ptr(v, ctypes.c_double), v.size)


def poisson_direct(rho, h):
    """phi [mx][my][mz] of Eq. openbruteforceconv by direct summation (oracle_poisson_direct);
    h = (hx, hy, hz)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.zeros_like(rho)
    _load().oracle_poisson_direct(_ptr(rho, ctypes.c_double), *rho.shape, float(h[0]), float(h[1]), float(h[2]),
                                  _ptr(phi, ctypes.c_double))
    return phi


def poisson_points(rho, h, ijk):
    """phi at the mesh points ijk [n][3] only (oracle_poisson_points)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(len(ijk))
    _load().oracle_poisson_points(_ptr(rho, ctypes.c_double), *rho.shape, float(h[0]), float(h[1]), float(h[2]),
                                  _ptr(ijk, ctypes.c_int32), len(ijk), _ptr(out, ctypes.c_double))
    return out
