"""The three-way bf16 split behind the tensor-core row update (CPU only).

The update takes U G on tensor cores from bf16 parts of both operands:
z = z_h + z_m + z_l with z_h = bf16(z), z_m = bf16(z - z_h), z_l = bf16(z - z_h - z_m),
the same for g, and sums the six products z_i g_j with i + j <= 2.  These
tests pin the two facts that make that a binary32-accurate product: the
remainders are exact in binary32, and the dropped terms (i + j >= 3) are of
order 2^-24 of |z g|, while dropping any kept term of order 2^-16 costs far
more.  bf16 rounding is torch's float32 -> bfloat16 conversion.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _bf16(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _split3(x):
    x = np.asarray(x, np.float32)
    h = _bf16(x)
    r1 = (x - h).astype(np.float32)
    m = _bf16(r1)
    r2 = (r1 - m).astype(np.float32)
    lo = _bf16(r2)
    return h, m, lo, r1, r2


def _samples(n, seed):
    g = np.random.default_rng(seed)
    mag = np.exp2(g.integers(-20, 20, size=n)).astype(np.float32)
    return (g.standard_normal(n).astype(np.float32) * mag).astype(np.float32)


def test_remainders_are_exact_in_binary32():
    z = _samples(100000, 1)
    h, m, _, r1, r2 = _split3(z)
    z64 = z.astype(np.float64)
    assert np.array_equal(r1.astype(np.float64), z64 - h.astype(np.float64))
    assert np.array_equal(r2.astype(np.float64), r1.astype(np.float64) - m.astype(np.float64))


def test_three_parts_carry_binary32_precision():
    z = _samples(100000, 2)
    h, m, lo, _, _ = _split3(z)
    rec = h.astype(np.float64) + m.astype(np.float64) + lo.astype(np.float64)
    rel = np.abs(rec - z.astype(np.float64)) / np.abs(z.astype(np.float64))
    assert rel.max() <= 2.0 ** -24


def _products(z, g, keep):
    zp = [p.astype(np.float64) for p in _split3(z)[:3]]
    gp = [p.astype(np.float64) for p in _split3(g)[:3]]
    return sum(zp[i] * gp[j] for i, j in keep)


SIX = [(i, j) for i in range(3) for j in range(3) if i + j <= 2]


def test_six_products_reach_binary32_level():
    z, g = _samples(100000, 3), _samples(100000, 4)
    exact = z.astype(np.float64) * g.astype(np.float64)
    rel = np.abs(_products(z, g, SIX) - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -21  # a binary32 product rounds at 2^-24 relative


@pytest.mark.parametrize("drop", [(0, 2), (1, 1), (2, 0), (0, 1), (1, 0)])
def test_every_kept_product_is_needed(drop):
    z, g = _samples(100000, 5), _samples(100000, 6)
    exact = z.astype(np.float64) * g.astype(np.float64)
    rel = np.abs(_products(z, g, [p for p in SIX if p != drop]) - exact) / np.abs(exact)
    assert rel.max() >= 2.0 ** -19


def test_row_times_gram_matches_fp64_to_binary32_level():
    """A row of length 100 against a 100 x 100 Gram, as in the update: the
    six-product sum differs from the FP64 product by no more than binary32
    accumulation would (relative to sum |z| |g|)."""
    g = np.random.default_rng(7)
    k = 100
    Z = g.random((64, k)).astype(np.float32)
    B = g.standard_normal((k, 300)).astype(np.float32)
    G = (B.astype(np.float64) @ B.T.astype(np.float64)).astype(np.float32)
    zp = [p.astype(np.float64) for p in _split3(Z)[:3]]
    gp = [p.astype(np.float64) for p in _split3(G)[:3]]
    six = sum(zp[i] @ gp[j] for i, j in SIX)
    exact = Z.astype(np.float64) @ G.astype(np.float64)
    scale = np.abs(Z.astype(np.float64)) @ np.abs(G.astype(np.float64))
    assert np.max(np.abs(six - exact) / scale) <= 2.0 ** -21
