"""The checking build of the library (compiled with MUSR_DEBUG_CHECKS).

compute-sanitizer is not available to this suite, so the kernels carry their own index
checks in a separate build: every computed index of a count, weight, histogram, chunk, work
item, partial row, map entry, dynamic Kubo-Toyabe table, finalize column, job and partition
piece is tested against its bound on the device, and a failed check ORs its bit into the
context's error word and skips the access (nothing traps).  Here the checking build runs
every kind of launch -- the SPLIT basis kernels of each shape group, the FP64 path, term
lists, dynamic Kubo-Toyabe tables, asymmetry data, Gauss-Newton products, ragged tails, a
batch on the launch-level partition -- in a process of its own, and every launch must leave
the word at 0 and still match the oracle.  The release build reports that it carries no
checks.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import musr_inputs as mi
import oracle
from paper_1509_07685_gb300 import binding as B
B.LIB_PATH = sys.argv[2]
B.load()
SPLIT, FP64 = B.MUSR_SPLIT, B.MUSR_FP64
cases = [
    ("cfg2 single SPLIT", mi.cfg2(nhist=8, nbins=5003, bin_width_ns=2.5, seed=71), SPLIT, 1, 1),
    ("cfg2 batch SPLIT", mi.cfg2(nhist=8, nbins=5003, bin_width_ns=2.5, seed=71), SPLIT, 1, 24),
    ("cfg5 batch SPLIT", mi.cfg5(nhist=10, nbins=6005, seed=72, n0=20.0, nbkg=0.1), SPLIT, 1, 16),
    ("cfg3 chi2 FP64", mi.cfg3(nhist=3, nbins=3001, bin_width_ns=4.0, seed=73), FP64, 0, 3),
    ("term list SPLIT", mi.levy_lf(nhist=2, nbins=1601, bin_width_ns=8.0, seed=74), SPLIT, 1, 4),
    ("dynamic KT FP64", mi.dkt_zf(nhist=2, nbins=1201, bin_width_ns=10.0, seed=75), FP64, 1, 2),
    ("dynamic KT SPLIT", mi.dkt_zf(nhist=2, nbins=1201, bin_width_ns=10.0, seed=75), SPLIT, 1, 9),
    ("asymmetry SPLIT", mi.asym_tf(npairs=2, nbins=4001, bin_width_ns=3.0, seed=76), SPLIT, 0, 9),
    ("launch-level partition SPLIT", mi.paper_tf16(seed=77), SPLIT, 1, 64),
]
out = {}
for name, p, prec, mode, nvec in cases:
    with B.Context(p) as ctx:
        X = mi.jitter(p.truth, nvec, seed=3, lo=0.97, hi=1.03)
        vals, grads, st = ctx.eval_batch(X, mode, prec)
        refs = [oracle.cost(p, X[k], mode) for k in range(nvec)]
        err = max(abs(vals[k] - refs[k][0]) / abs(refs[k][0]) for k in range(nvec))
        gerr = max(float(np.max(np.abs(grads[k] - refs[k][1]) / (refs[k][2] + 1e-300))) for k in range(nvec))
        if name == "cfg3 chi2 FP64":
            H = ctx.gauss_newton(X[0], 0, FP64)
            R = oracle.gauss_newton(p, X[0], 0)
            s = np.sqrt(np.outer(np.diag(R), np.diag(R)))
            gerr = max(gerr, float(np.max(np.abs(H - R) / s)))
        dst, word = B.musr_debug_word(ctx.ctx)
        out[name] = {"status": int(st), "word": int(word), "debug_status": int(dst), "err": float(err),
                     "gerr": float(gerr), "prec": int(prec)}
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def checking_lib():
    from paper_1509_07685_gb300 import build
    return build.build(debug=True)


def test_checking_build_finds_no_out_of_bounds_index(checking_lib):
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, checking_lib], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for name, c in out.items():
        tol = 1e-9 if c["prec"] == 0 else 2.0 ** -16
        if "dynamic KT" in name:
            tol += 1e-5  # the tables' stated accuracy (tests/test_gpu_dkt.py)
        assert c["debug_status"] == 0 and c["word"] == 0, (name, c)
        assert c["status"] == 0, (name, c)
        assert c["err"] <= tol and c["gerr"] <= tol, (name, c)


def test_release_build_has_no_checks(musr_lib):
    from paper_1509_07685_gb300 import binding as B
    import musr_inputs as mi
    p = mi.cfg3(nhist=1, nbins=500, bin_width_ns=20.0, seed=77)
    with B.Context(p) as ctx:
        ctx.eval(p.truth, 0, B.MUSR_SPLIT)
        st, word = B.musr_debug_word(ctx.ctx)
    assert st == B.MUSR_ESTATE and word == 0
