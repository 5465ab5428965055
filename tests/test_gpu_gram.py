"""The FP64 Gram G = B B^T of the sketched subproblem (eq. gradient_descent's
B B^T term) against numpy's FP64 product of the same binary32 entries.

Products of two binary32 numbers are exact in FP64, so the two sides differ
only in the order of the FP64 sums (relative difference <= 1e-12 of the
largest entry).  The shapes cover k not a multiple of the 4 x 4 register
tile, k = 128 (the largest thread count), widths below one chunk, and widths
that make every CTA walk several chunks with a ragged last one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


@pytest.mark.parametrize("k,d", [(1, 1), (3, 3), (5, 7), (16, 2048), (64, 2048), (64, 4093), (99, 500),
                                 (100, 5000), (128, 70001), (64, 65536), (2, 100003)])
def test_gram_matches_fp64_product(pkg, k, d):
    import torch
    g = np.random.default_rng(k * 1000 + d)
    B = g.standard_normal((k, d)).astype(np.float32)
    B[:, ::7] *= 1e3  # a spread of magnitudes
    want = B.astype(np.float64) @ B.astype(np.float64).T
    got = pkg.gram_noalloc(torch.from_numpy(B).cuda()).cpu().numpy()
    assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))
    assert np.array_equal(got, got.T)


def test_gram_is_deterministic(pkg):
    """A fixed summation order: two calls give the same bits."""
    import torch
    B = torch.from_numpy(np.random.default_rng(3).standard_normal((64, 30000)).astype(np.float32)).cuda()
    a = pkg.gram_noalloc(B).cpu().numpy()
    b = pkg.gram_noalloc(B).cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
