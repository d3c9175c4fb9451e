"""One fit split by histograms (paper_1509_07685_gb300.shard) and evaluated on the GPU as
k sub-contexts on one device, their (1 + P) results summed in rank order: the FP64 sum
equals a single context's result within 1e-13 (value relative; gradient against the
oracle's gradient scale), and the SPLIT sum stays within its 2^-16 bound of the oracle.
This is the arithmetic of the multi-rank path (one sub-context per rank, one exchange of
1 + P doubles per evaluation) with the exchange done in-process."""
import numpy as np
import pytest

import musr_inputs as mi
import oracle
from paper_1509_07685_gb300 import shard
from test_gpu_parity import SPLIT_EPS, problems

pytestmark = pytest.mark.gpu

SHARD_TOL = 1e-13


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


@pytest.mark.parametrize("name", ["cfg2", "cfg3", "paper_tf16"])
@pytest.mark.parametrize("k", [2, 3, 5])
def test_k_subcontexts_sum_to_the_single_context(B, name, k):
    p = problems()[name]
    x = mi.start_point(p, 7)
    parts = [h for h in shard.partition_histograms([p.B] * p.H, k) if h]
    assert sorted(i for h in parts for i in h) == list(range(p.H))
    for mode in (0, 1):
        rv, rg, rgs, _ = oracle.cost(p, x, mode)
        with B.Context(p) as ctx:
            v1, g1, _ = ctx.eval(x, mode, B.MUSR_FP64)
        rows = {B.MUSR_FP64: [], B.MUSR_SPLIT: []}
        for hs in parts:
            with B.Context(shard.sub_problem(p, hs)) as c:
                for prec in rows:
                    v, g, st = c.eval(x, mode, prec)
                    assert st == B.MUSR_OK
                    rows[prec].append(np.concatenate([[v], g]))
        tot = shard.combine(rows[B.MUSR_FP64])
        assert abs(tot[0] - v1) <= SHARD_TOL * abs(v1), (tot[0], v1)
        assert np.all(np.abs(tot[1:] - g1) <= SHARD_TOL * rgs + 1e-300)
        tot = shard.combine(rows[B.MUSR_SPLIT])
        assert abs(tot[0] - rv) <= SPLIT_EPS * abs(rv)
        assert np.all(np.abs(tot[1:] - rg) <= SPLIT_EPS * rgs + 1e-300)
