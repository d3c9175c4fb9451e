"""Failure detection on the GPU without a fault.

The SPLIT kernels wait for their staged counts on shared-memory mbarriers for at most 100 ms
of the GPU's global timer.  musr_check_bounded_wait runs that wait on a barrier that nothing
arrives on: the wait must give up after its 100 ms (a little more: the timer is read every 64
tries), the completed phase must then be seen, and the process's CUDA context must stay
usable.  An evaluation afterwards matches the oracle.
"""
import numpy as np
import pytest

import musr_inputs as mi
import oracle
from test_gpu_parity import _check_split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def test_bounded_wait_gives_up_and_context_stays_usable(B):
    st, t_try, t_wait = B.musr_check_bounded_wait(0)
    print(f"unsatisfied try: {t_try * 1e9:.1f} ns; wait gave up after {t_wait:.3f} s")
    assert st == B.MUSR_OK, (st, t_try, t_wait)
    assert 0.1 <= t_wait <= 0.1 + 64 * t_try + 0.05
    p = mi.cfg1(nbins=3000, seed=8, dtype=np.float32)
    with B.Context(p) as ctx:
        for mode in (0, 1):
            v, g, st = ctx.eval(p.truth, mode, B.MUSR_SPLIT)
            assert st == 0
            _check_split(v, g, oracle.cost(p, p.truth, mode))


def test_bounded_wait_rejects_a_bad_device(B):
    st, _, _ = B.musr_check_bounded_wait(4096)
    assert st == B.MUSR_EINVAL


def test_loaded_code_is_sm103a(B):
    st, ver = B.musr_binary_version(0)
    assert st == B.MUSR_OK and ver == 103, (st, ver)
