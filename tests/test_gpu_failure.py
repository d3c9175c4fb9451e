"""Failure detection on the GPU without a fault.

No kernel of the library waits on a flag, a barrier of another CTA or an mbarrier: counts are
staged by per-thread asynchronous copies that each thread waits for itself, and completion
counters are atomics nobody spins on.  Failures are reported as statuses the host reads:

* parameters that are not finite give a non-finite cost and MUSR_ENONFINITE, with zero
  gradients, in both precisions and schedules, and the context stays usable -- the next
  evaluation matches the oracle;
* an -2lnL that is undefined (N <= 0 where d > 0) gives MUSR_ENONFINITE the same way;
* the loaded code is the one built for sm_103a (the runtime's own report).
"""
import numpy as np
import pytest

import musr_inputs as mi
import oracle
from test_gpu_parity import _check_fp64, _check_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def test_nonfinite_parameters_are_reported_and_the_context_stays_usable(B):
    p = mi.cfg2(nhist=8, nbins=4001, bin_width_ns=3.0, seed=81)
    X = mi.jitter(p.truth, 16, seed=2, lo=0.97, hi=1.03)
    bad = X.copy()
    bad[3, 0] = np.nan   # a shared rate
    bad[9, 7] = np.inf   # a phase
    with B.Context(p) as ctx:
        for prec in (B.MUSR_FP64, B.MUSR_SPLIT):
            for mode in (0, 1):
                vals, grads, st = ctx.eval_batch(bad, mode, prec)  # 16 vectors: the vector-group schedule at SPLIT
                assert st == B.MUSR_ENONFINITE
                assert not np.isfinite(vals[3]) and not np.isfinite(vals[9])
                assert np.all(grads[3] == 0.0) and np.all(grads[9] == 0.0)
                good = [k for k in range(16) if k not in (3, 9)]
                assert np.all(np.isfinite(vals[good]))
                v, g, st = ctx.eval(X[0], mode, prec)
                assert st == 0
                ref = oracle.cost(p, X[0], mode)
                (_check_fp64 if prec == B.MUSR_FP64 else _check_split)(v, g, ref)


def test_loaded_code_is_sm103a(B):
    st, ver = B.musr_binary_version(0)
    assert st == B.MUSR_OK and ver == 103, (st, ver)
    st, _ = B.musr_binary_version(4096)
    assert st == B.MUSR_EINVAL
