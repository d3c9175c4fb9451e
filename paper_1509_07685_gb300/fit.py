"""Host-side BFGS minimiser driving the GPU cost (the role migrad plays in Section 4).

As in the paper's offload, the minimiser runs on the host and each trial point
costs one evaluation on the device: the parameter vector goes in, the value
and -- from the fused kernel -- the analytic gradient come back.  Where the
algorithm needs several points at once (the diagonal curvature estimate that
scales the first step, the Hessian for the parameter errors), they go to the
device as one batched launch.

Algorithm (quasi-Newton, BFGS inverse update):
  * H0 = diag(1 / |h_ii|), h_ii forward differences of the analytic gradient
    along each axis (one batched evaluation of P shifted points);
  * p = -H g (reset to the diagonal when p is not a descent direction);
  * backtracking from alpha = 1, halving, until
    f_new <= f + 1e-4 alpha g.p (Armijo) with f_new finite, or -- for a cost
    with rounding noise -- f_new within f_noise above that bound and a smaller
    gradient (max|g_new| < max|g|);
  * BFGS update when s.y > 0;
  * stop when max|g| <= gtol * max(1, |f|), when the estimated distance to the
    minimum EDM = g.H.g / 2 falls below edm_tol (both costs are -2lnL scaled,
    so EDM is in units where a change of 1 is one standard deviation), or when
    a step leaves x unchanged.
``f_noise`` absorbs the rounding noise of a reduced-precision cost so that the
line search does not stall on it; convergence is decided on the gradient.
"""
from __future__ import annotations

import time
from typing import Callable, Optional, Tuple

import numpy as np

from . import binding as B


def default_steps(x) -> np.ndarray:
    """Difference steps: 1e-5 relative, at least 1e-4 absolute (parameters near zero,
    such as a phase of 0 degrees, would otherwise get steps at the cost's noise level)."""
    x = np.asarray(x, dtype=np.float64)
    return np.maximum(1e-5 * np.abs(x), 1e-4)


def bfgs(fg: Callable[[np.ndarray], Tuple[float, np.ndarray]], x0, *,
         fg_batch: Optional[Callable[[np.ndarray], Tuple[np.ndarray, np.ndarray]]] = None,
         gtol: float = 1e-8, maxit: int = 1000, fd_step=None, f_noise: float = 0.0,
         edm_tol: float = 1e-7) -> dict:
    t_start = time.perf_counter()
    x = np.array(x0, dtype=np.float64)
    P = x.size
    nfev = 0
    f, g = fg(x)
    nfev += 1
    if not np.isfinite(f):
        return {"x": x, "f": f, "g": g, "iters": 0, "nfev": nfev, "status": 1,
                "time_s": time.perf_counter() - t_start}
    steps = default_steps(x) if fd_step is None else np.asarray(fd_step, dtype=np.float64)

    def diag_hinv(xc, gc):
        shifted = xc[None, :] + np.diag(steps)
        if fg_batch is not None:
            _, G = fg_batch(shifted)
        else:
            G = np.stack([fg(shifted[j])[1] for j in range(P)])
        h = np.abs((np.diag(G) - gc) / steps)
        return np.diag(np.where(h > 0, 1.0 / np.where(h > 0, h, 1.0), 1.0)), P

    Hinv, n = diag_hinv(x, g)
    nfev += n
    updates = 0  # BFGS updates since the last reset of Hinv
    status = 2
    it = 0
    for it in range(maxit):
        if np.max(np.abs(g)) <= gtol * max(1.0, abs(f)):
            status = 0
            break
        p = -Hinv @ g
        gp = float(p @ g)
        if not gp < 0.0:
            Hinv, n = diag_hinv(x, g)
            nfev += n
            updates = 0
            p = -np.diag(Hinv) * g
            gp = float(p @ g)
        edm = -0.5 * gp
        if updates >= 2 and edm < edm_tol:
            status = 0
            break
        alpha = 1.0
        ok = False
        gnorm = float(np.linalg.norm(g))
        for _ in range(60):
            xn = x + alpha * p
            fn, gn = fg(xn)
            nfev += 1
            if np.isfinite(fn):
                armijo = f + 1e-4 * alpha * gp
                # Below the noise of the cost, f cannot rank the points: accept a step the
                # quasi-Newton model predicts to gain less than the noise if |g| shrinks.
                small = -alpha * gp < 10.0 * f_noise
                if fn <= armijo or (small and fn <= armijo + f_noise and np.linalg.norm(gn) < gnorm):
                    ok = True
                    break
            if -alpha * gp < 0.01 * f_noise:
                break
            alpha *= 0.5
        if not ok:
            # No acceptable step: converged to the noise floor if the model says so.
            status = 0 if (f_noise > 0 and edm < 100.0 * edm_tol) else 3
            break
        s = xn - x
        y = gn - g
        moved = bool(np.any(xn != x))
        x, f, g = xn, fn, gn
        if not moved:
            status = 0
            break
        sy = float(s @ y)
        if sy > 0.0:
            updates += 1
            rho = 1.0 / sy
            Hy = Hinv @ y
            Hinv = (Hinv - rho * (np.outer(Hy, s) + np.outer(s, Hy))
                    + (rho * rho * float(y @ Hy) + rho) * np.outer(s, s))
    return {"x": x, "f": f, "g": g, "iters": it, "nfev": nfev, "status": status,
            "time_s": time.perf_counter() - t_start}


# Rounding noise of the SPLIT cost relative to its value (per-bin FP32 with hardware
# transcendentals; the measured deviation from the FP64 cost is 2e-8 to 1.4e-7 relative).
SPLIT_F_NOISE_REL = 2e-8
# EDM target of SPLIT fits: the FP32 gradient's rounding puts a floor of ~1e-6 under
# g.H.g / 2 at the cfg2 sizes; 1e-5 still places the fit within ~0.005 sigma of its optimum.
SPLIT_EDM_TOL = 1e-5


def fit_context(ctx: "B.Context", x0, mode: int, precision: int, **kw) -> dict:
    """BFGS fit of the problem held by ``ctx`` (value+gradient from the fused kernel)."""
    def fg(x):
        v, g, _ = ctx.eval(x, mode, precision)
        return v, g

    def fgb(X):
        v, g, _ = ctx.eval_batch(X, mode, precision)
        return v, g

    if precision == B.MUSR_SPLIT:
        if "f_noise" not in kw:
            f0, _ = fg(np.asarray(x0, dtype=np.float64))
            kw["f_noise"] = SPLIT_F_NOISE_REL * abs(f0)
        kw.setdefault("edm_tol", SPLIT_EDM_TOL)
    return bfgs(fg, x0, fg_batch=fgb, **kw)


def hessian_context(ctx: "B.Context", x, mode: int, precision: int = B.MUSR_FP64, steps=None) -> np.ndarray:
    """Central differences of the analytic gradient, 2P points in one batched launch."""
    x = np.asarray(x, dtype=np.float64)
    P = x.size
    st = default_steps(x) if steps is None else np.asarray(steps)
    X = np.concatenate([x[None, :] + np.diag(st), x[None, :] - np.diag(st)])
    _, G, status = ctx.eval_batch(X, mode, precision)
    if status != B.MUSR_OK:
        raise FloatingPointError("cost is +inf near x")
    H = (G[:P] - G[P:]).T / (2.0 * st[None, :])
    return 0.5 * (H + H.T)


def sigmas_context(ctx: "B.Context", x, mode: int) -> np.ndarray:
    """sigma_i = sqrt(2 (H^-1)_ii): both costs are -2lnL scaled (Delta cost = 1 is one sigma)."""
    H = hessian_context(ctx, x, mode)
    return np.sqrt(np.diag(2.0 * np.linalg.inv(H)))


def sigmas_gauss_newton(ctx: "B.Context", x, mode: int, precision: int = B.MUSR_SPLIT) -> np.ndarray:
    """sigma_i = sqrt(2 (H^-1)_ii) with H the Gauss-Newton matrix from the fused kernel (one launch);
    NaN where H is not positive definite."""
    H = ctx.gauss_newton(x, mode, precision)
    with np.errstate(invalid="ignore"):
        return np.sqrt(np.diag(2.0 * np.linalg.inv(H)))


def fd_gradient_batch(ctx: "B.Context", x, mode: int, precision: int, steps=None):
    """Central finite-difference gradient: 2P + 1 cost evaluations (one batched launch,
    value only) -- the cost of a gradient without the fused analytic kernel."""
    x = np.asarray(x, dtype=np.float64)
    P = x.size
    st = default_steps(x) if steps is None else np.asarray(steps)
    X = np.concatenate([x[None, :], x[None, :] + np.diag(st), x[None, :] - np.diag(st)])
    v, _, _ = ctx.eval_batch(X, mode, precision, grad=False)
    return v[0], (v[1:P + 1] - v[P + 1:]) / (2.0 * st)
