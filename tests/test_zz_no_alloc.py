"""The allocation-free Gram entry point (dsanls_gram_noalloc) against the Gram
the existing handle API computes and against the FP64 oracle's.

Some callers cannot let a library allocate device memory (a host framework
that owns all device memory through its own pool, or a latency-critical loop
that cannot absorb cudaFree's device synchronisation); this entry point keeps
its scratch in a fixed array inside the library instead.  With the identity
sketch the handle's U-half Gram is exactly V^T V, so feeding B = V^T to the
allocation-free entry point must reproduce it: FP64 sums of the same exact
products, differing only in summation order (relative difference <= 1e-12).
Called twice in a row to show that the shared scratch left by the first call
does not leak into the second.  This file sorts last so that a run stopping
at the first failure has already run every other test.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import method
from synthdata import initial_factors, planted_dense

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _existing_gram(pkg, M, U, V):
    m, n = M.shape
    k = U.shape[1]
    h = pkg.DSANLS(m, n, k, n, pkg.IDENTITY, seed=0)
    h.set_dense(M)
    h.set_factors(U, V)
    h.half_step(0)
    G, _ = h.gram(0)
    h.close()
    return G


# k = 10 and 33 run the masked staging and output paths of k % 4 != 0
@pytest.mark.parametrize("m,n,k", [(300, 257, 16), (200, 1500, 64), (150, 700, 100), (96, 333, 128),
                                   (300, 257, 10), (120, 901, 33)])
def test_noalloc_gram_matches_handle_gram(pkg, m, n, k):
    import torch
    M, _, _ = planted_dense(m, n, min(k, 16), 4)
    U, V = initial_factors(m, n, k, 5)
    want = _existing_gram(pkg, M, U, V)
    B = torch.from_numpy(np.ascontiguousarray(V.T)).cuda()
    Bother = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    G = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
    for _ in range(2):
        pkg.gram_noalloc(B, G)
        torch.cuda.synchronize()
        got = G.cpu().numpy()
        assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))
        # and directly against the FP64 oracle's Gram of the unsketched subproblem
        # (B = V^T S with S = I; binary32 products are exact in FP64)
        S = method.Sketch(method.IDENTITY, 0, 0, 0, n, n)
        _, _, Go, _ = method.sketched_terms(M.astype(np.float64), V.astype(np.float64), S)
        assert np.max(np.abs(got - Go)) <= TOL * np.max(np.abs(Go))
        # a different problem in between must not leave anything behind
        pkg.gram_noalloc(Bother)
        torch.cuda.synchronize()


def test_noalloc_gram_rejects_sizes_beyond_its_scratch(pkg):
    import torch
    lib = pkg.lib()
    B = torch.zeros((129, 8), dtype=torch.float32, device="cuda")
    G = torch.zeros((129, 129), dtype=torch.float64, device="cuda")
    rc = lib.dsanls_gram_noalloc(ctypes.c_void_p(B.data_ptr()), 129, 8, ctypes.c_void_p(G.data_ptr()), None)
    assert rc == -1
    assert b"k must be in [1, 128]" in lib.dsanls_last_error(None)
    assert lib.dsanls_gram_noalloc(None, 4, 8, ctypes.c_void_p(G.data_ptr()), None) == -1


_CAPTURE_PROBE = r"""
import ctypes, sys, torch
sys.path.insert(0, sys.argv[1])
import paper_2009_02845_gb300 as pkg
lib = pkg.lib()
B = torch.ones((8, 64), dtype=torch.float32, device="cuda")
G = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
s = torch.cuda.Stream()
torch.cuda.synchronize()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    G.mul_(1.0)  # keeps the captured graph non-empty
    rc = lib.dsanls_gram_noalloc(ctypes.c_void_p(B.data_ptr()), 8, 64, ctypes.c_void_p(G.data_ptr()),
                                 ctypes.c_void_p(s.cuda_stream))
msg = lib.dsanls_last_error(None)
# outside capture the same first call sets the device up and computes G
rc2 = lib.dsanls_gram_noalloc(ctypes.c_void_p(B.data_ptr()), 8, 64, ctypes.c_void_p(G.data_ptr()), None)
torch.cuda.synchronize()
print(rc, rc2, float(G[0, 0].item()), msg.decode())
"""


def test_noalloc_first_call_inside_capture_is_refused():
    """A fresh process whose first call on the device comes while its stream
    is being captured gets EINVAL (and nothing is queued, so the capture ends
    normally); the next call outside capture works."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _CAPTURE_PROBE, root], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    rc, rc2, g00, msg = out.stdout.strip().splitlines()[-1].split(" ", 3)
    assert int(rc) == -1 and "before any stream capture" in msg
    assert int(rc2) == 0 and float(g00) == 64.0
