"""torch.autograd.Function around the fused value+gradient kernel.

forward() enqueues one launch that writes the cost and its analytic gradient
to device memory (no host round trip); backward() scales the stored gradient.
This replaces the 2P + 1 cost calls a finite-difference gradient would need.
The context must run on the current torch stream (create it with
``cuda_stream=torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from .fit import bfgs


class MusrCost(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params: torch.Tensor, context: "B.Context", mode: int, precision: int):
        if not params.is_cuda or params.dtype != torch.float64:
            raise TypeError("params must be a float64 CUDA tensor")
        x = params.detach().contiguous()
        out = torch.empty(1 + x.numel(), dtype=torch.float64, device=x.device)
        B.musr_eval_device(context.ctx, x.data_ptr(), 1, mode, precision, True, out.data_ptr())
        fctx.save_for_backward(out[1:])
        return out[0]

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return grad_out * g, None, None, None


def cost(params: torch.Tensor, context: "B.Context", mode: int = B.MUSR_CHI2,
         precision: int = B.MUSR_SPLIT) -> torch.Tensor:
    return MusrCost.apply(params, context, mode, precision)


def fit_autograd(context: "B.Context", x0, mode: int, precision: int, **kw) -> dict:
    """The host BFGS driven through the autograd Function (value and gradient via backward)."""
    dev = torch.device("cuda", torch.cuda.current_device())

    def fg(x):
        t = torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=True)
        f = cost(t, context, mode, precision)
        f.backward()
        return float(f.item()), t.grad.detach().cpu().numpy()

    if precision == B.MUSR_SPLIT:
        from .fit import SPLIT_EDM_TOL, SPLIT_F_NOISE_REL
        if "f_noise" not in kw:
            kw["f_noise"] = SPLIT_F_NOISE_REL * abs(fg(np.asarray(x0, dtype=np.float64))[0])
        kw.setdefault("edm_tol", SPLIT_EDM_TOL)
    return bfgs(fg, x0, **kw)
