"""GB300-native muSR chi^2 / Poisson -2lnL cost and gradient (arXiv 1509.07685, Section 4).

The hot path lives in libmusr (C ABI, ``include/musr.h``; CUDA kernels for
sm_103a in ``csrc/``).  ``binding`` marshals arguments into it; there is no
CPU fallback: importing works without a GPU, calling needs the built library
and a GPU.
"""
from . import binding  # noqa: F401
from .binding import (MUSR_CHI2, MUSR_FP64, MUSR_MLE, MUSR_SPLIT, Context,  # noqa: F401
                      MusrError)

__all__ = ["binding", "Context", "MusrError", "MUSR_CHI2", "MUSR_MLE", "MUSR_FP64", "MUSR_SPLIT"]
