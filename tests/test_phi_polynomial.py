"""The polynomial the SPLIT kernels take for the Poisson deviance of a bin near its optimum.

For |u| < 0.2 (u = (N - d)/N) the kernels evaluate phi(u) = u + (1 - u) ln(1 - u) as
u^2 p(u), p a degree-6 polynomial with FP32 coefficients (`phi_u2` in
csrc/musr_kernels.cuh).  Here its coefficients are read from the source and checked
against the series sum_{k>=2} u^k / (k (k - 1)), summed in FP64 to far below the
tolerance: relative error at most 2e-8 of phi over the interval (FP32's unit roundoff is
6e-8), and the packed two-bin form uses the same coefficients in the same order.
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1509_07685_gb300", "csrc",
                   "musr_kernels.cuh")
FLOAT = r"([0-9.]+e[-+][0-9]+)f"


def _bodies():
    s = open(SRC).read()
    scalar = s[s.index("__device__ __forceinline__ float phi_u2(float u)"):]
    scalar = scalar[:scalar.index("\n}\n")]
    packed = s[s.index("__device__ __forceinline__ float2 phi_u2(float2 u)"):]
    packed = packed[:packed.index("\n}\n")]
    return scalar, packed


def _coefficients_high_first(body):
    vals = [float(v) for v in re.findall(FLOAT, body)]
    # each make_float2(c, c) repeats c: keep one of each pair
    out = []
    for v in vals:
        if not out or out[-1] != v:
            out.append(v)
    return out


def test_polynomial_matches_the_series():
    scalar, _ = _bodies()
    c = _coefficients_high_first(scalar)
    assert len(c) == 7 and c[-1] == 0.5
    c32 = np.array(c, dtype=np.float32).astype(np.float64)  # the literals as the compiler rounds them
    u = np.linspace(-0.2, 0.2, 200001)
    exact = sum(u ** (k - 2) / (k * (k - 1)) for k in range(2, 40))  # phi(u) / u^2
    rel = np.abs(np.polyval(c32, u) - exact) / exact
    assert rel.max() < 2e-8, rel.max()
    # the first terms of the series are close to the exact ones (a sanity check of the fit)
    assert abs(c32[-1] - 0.5) == 0 and abs(c32[-2] - 1.0 / 6.0) < 1e-6 and abs(c32[-3] - 1.0 / 12.0) < 1e-6


def test_packed_form_uses_the_same_coefficients():
    scalar, packed = _bodies()
    assert _coefficients_high_first(packed) == _coefficients_high_first(scalar)
