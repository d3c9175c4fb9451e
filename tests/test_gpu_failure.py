"""Failure detection on the GPU without a fault.

No kernel of the library waits on a flag, a barrier of another CTA or an mbarrier: counts are
staged by per-thread asynchronous copies that each thread waits for itself, and completion
counters are atomics nobody spins on.  Failures are reported as statuses the host reads:

* parameters that are not finite are refused on the host (MUSR_EINVAL); passed as device
  arrays they give that evaluation a value of +inf and zero gradients, the other
  evaluations of the launch are unaffected, and the context stays usable -- the next
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
    """Host arrays: refused before any launch (MUSR_EINVAL).  Device arrays (no host check):
    the kernels give that vector a value of +inf and zero gradients, the other vectors of the
    launch are unaffected, and the context stays usable."""
    import torch
    p = mi.cfg2(nhist=8, nbins=4001, bin_width_ns=3.0, seed=81)
    X = mi.jitter(p.truth, 16, seed=2, lo=0.97, hi=1.03)
    bad = X.copy()
    bad[3, 0] = np.nan   # a shared rate
    bad[9, 7] = np.inf   # a phase
    good = [k for k in range(16) if k not in (3, 9)]
    with B.Context(p) as ctx:
        for prec in (B.MUSR_FP64, B.MUSR_SPLIT):
            for mode in (0, 1):
                with pytest.raises(B.MusrError) as e:
                    ctx.eval_batch(bad, mode, prec)
                assert e.value.status == B.MUSR_EINVAL
                ref_vals, ref_grads, st = ctx.eval_batch(X, mode, prec)
                assert st == 0
                d_x = torch.tensor(bad, dtype=torch.float64, device="cuda")
                d_out = torch.zeros((16, 1 + p.nparams), dtype=torch.float64, device="cuda")
                B.musr_eval_device(ctx.ctx, d_x.data_ptr(), 16, mode, prec, True, d_out.data_ptr())
                torch.cuda.synchronize()
                out = d_out.cpu().numpy()
                assert not np.isfinite(out[3, 0]) and not np.isfinite(out[9, 0])
                assert np.all(out[3, 1:] == 0.0) and np.all(out[9, 1:] == 0.0)
                assert np.array_equal(out[good, 0], ref_vals[good])
                assert np.array_equal(out[good, 1:], ref_grads[good])
                v, g, st = ctx.eval(X[0], mode, prec)
                assert st == 0
                ref = oracle.cost(p, X[0], mode)
                (_check_fp64 if prec == B.MUSR_FP64 else _check_split)(v, g, ref)


def test_loaded_code_is_sm103a(B):
    st, ver = B.musr_binary_version(0)
    assert st == B.MUSR_OK and ver == 103, (st, ver)
    st, _ = B.musr_binary_version(4096)
    assert st == B.MUSR_EINVAL
