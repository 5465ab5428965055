"""The index-checking debug build (-DDSANLS_BOUNDS, libdsanls_bounds.so).

The checking build validates every index it takes from the data (columns of
a CSR, the row keys and scatter destinations of the sub-CSR build) and skips
and counts an access that would leave its array.  On valid inputs it must
report no failed check and compute exactly what the normal build computes:
the checks add branches, not arithmetic.  The child process loads the
checking build (one process cannot load both), runs half-steps of the sparse
paths (subsampling: sub-CSR gather, radix sort, rows; Gaussian and identity:
the CSR product) and writes the factors; the parent runs the same with the
normal build and compares bit for bit.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
from paper_2009_02845_gb300 import build as B
B.build(bounds=True)
from paper_2009_02845_gb300 import _lib
_lib.use_bounds_build()
import paper_2009_02845_gb300 as pkg
sys.path.insert(0, %(tests)r)
from test_gpu_bounds import run_cases
out = run_cases(pkg)
checking, count, site, index = _lib.debug_bounds_report()
np.savez(%(npz)r, **out)
print(json.dumps({"checking": checking, "count": count, "site": site, "index": index}))
"""


def run_cases(pkg):
    from synthdata import initial_factors, sparse_text
    out = {}
    cases = [("sub_u", 3000, 1200, 48, 300, 400, pkg.SUBSAMPLE, 0), ("sub_v", 3000, 1200, 48, 300, 400, pkg.SUBSAMPLE, 1),
             ("long_v", 2000, 5000, 100, 500, 300, pkg.SUBSAMPLE, 1), ("gauss", 1500, 700, 16, 64, 64, pkg.GAUSSIAN, 0),
             ("ident", 900, 400, 8, 400, 900, pkg.IDENTITY, 1)]
    for name, m, n, k, d, dv, kind, side in cases:
        rp, col, val = sparse_text(m, n, 5, mean_len=30.0)
        U, V = initial_factors(m, n, k, 6)
        h = pkg.DSANLS(m, n, k, d, kind, seed=3, d_v=dv, t=2)
        h.set_csr(rp, col, val)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        out[name] = Ug if side == 0 else Vg
    return out


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def test_bounds_build_reports_nothing_and_matches_the_normal_build(pkg, tmp_path):
    npz = str(tmp_path / "bounds_out.npz")
    code = _CHILD % {"root": ROOT, "tests": os.path.join(ROOT, "tests"), "npz": npz}
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1500, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["checking"] is True
    assert rep["count"] == 0, rep
    got = np.load(npz)
    want = run_cases(pkg)
    for name, w in want.items():
        assert np.array_equal(got[name], w), name


def test_normal_build_reports_no_checks(pkg):
    from paper_2009_02845_gb300 import _lib
    checking, count, _, _ = _lib.debug_bounds_report()
    assert checking is False and count == 0
