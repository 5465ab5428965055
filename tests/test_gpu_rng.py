"""GPU random streams are bit-exact against the oracle (Section 3.3: every node
regenerates the same S^t from the shared seed).  Compared word for word and
value for value through the C ABI."""
import numpy as np
import pytest

from oracle import rng

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


@pytest.mark.parametrize("seed,stream,t,rows,cols", [
    (0, 0, 0, 8, 4), (0xDEADBEEFCAFEF00D, 1, 7, 13, 5), (1, 3, (1 << 32) + 5, 17, 3), (42, 0x7f, 123456, 1, 1),
    (5, 0, 99, 1001, 37)])
def test_philox_field_words(pkg, seed, stream, t, rows, cols):
    got = pkg.philox_field(seed, stream, t, rows, cols).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, rng.field_words(seed, stream, t, rows, cols))


@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("seed,stream,t,rows,cols", [
    (0, 0, 0, 800, 100), (3, 1, 9, 1001, 33), (7, 0, (1 << 33) + 1, 5, 7), (11, 1, 2, 16384, 64)])
def test_gaussian_field_bits(pkg, transposed, seed, stream, t, rows, cols):
    scale = rng.gaussian_scale(cols)
    got = pkg.gaussian_field(seed, stream, t, rows, cols, scale, transposed=transposed).cpu().numpy()
    if transposed:
        got = got.T
    want = rng.gaussian_field(seed, stream, t, rows, cols, scale)
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("seed,stream,t,rows,cols", [
    (0, 0, 0, 800, 100), (3, 1, 9, 1001, 33), (7, 0, (1 << 33) + 1, 5, 7)])
def test_rademacher_field_bits(pkg, transposed, seed, stream, t, rows, cols):
    scale = rng.gaussian_scale(cols)
    got = pkg.rademacher_field(seed, stream, t, rows, cols, scale, transposed=transposed).cpu().numpy()
    if transposed:
        got = got.T
    want = rng.rademacher_field(seed, stream, t, rows, cols, scale)
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("seed,side,t,rows,cols", [(0, 0, 0, 800, 100), (3, 1, 9, 1001, 33), (7, 0, (1 << 33) + 1, 5, 7)])
def test_count_field_bits(pkg, transposed, seed, side, t, rows, cols):
    got = pkg.count_field(seed, side, t, rows, cols, transposed=transposed).cpu().numpy()
    if transposed:
        got = got.T
    want = rng.count_field(seed, side, t, rows, cols)
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("seed,side,t,rows,cols", [
    (0, 0, 0, 800, 100), (3, 1, 9, 1001, 33), (7, 0, (1 << 33) + 1, 5, 7), (2, 1, 4, 512, 512), (5, 0, 3, 1, 1),
    (11, 1, 6, 16384, 2048), (4, 0, 1, 3000, 4096)])
def test_srht_field_bits(pkg, transposed, seed, side, t, rows, cols):
    """SRHT entries bit-exact with the oracle (signs, sampled Hadamard columns
    over the padded order, Sylvester parity), including d = p (every column)
    and d > rows (allowed up to the padded order)."""
    scale = rng.gaussian_scale(cols)
    got = pkg.srht_field(seed, side, t, rows, cols, scale, transposed=transposed).cpu().numpy()
    if transposed:
        got = got.T
    want = rng.srht_field(seed, side, t, rows, cols, scale)
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint32), want.view(np.uint32))


def test_srht_field_rejects_bad_sizes(pkg):
    with pytest.raises(pkg.DSANLSError):
        pkg.srht_field(0, 0, 0, 1000, 1025, 1.0)  # cols above the padded order 1024
    with pytest.raises(pkg.DSANLSError):
        pkg.srht_field(0, 16, 0, 100, 10, 1.0)  # side out of range


def test_uniform_field_bits(pkg):
    got = pkg.uniform_field(9, 2, 0, 1003, 10).cpu().numpy()
    want = rng.uniform_field(9, 2, 0, 1003, 10)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("n,d", [(1, 1), (2, 1), (2, 2), (17, 17), (800, 100), (1000, 100), (16384, 2048),
                                 (65536, 2048), (500_000, 5000), (2_000_000, 5000), (40_000, 16384),
                                 (100_000, 50_000), (70_001, 70_001)])
@pytest.mark.parametrize("side,t", [(0, 0), (1, 3), (0, (1 << 32) + 11)])
def test_subsample_indices_bits(pkg, n, d, side, t):
    got = pkg.subsample_indices(123, side, t, n, d).cpu().numpy()
    want = rng.subsample_indices(123, side, t, n, d)
    assert np.array_equal(got, want)
    assert np.all(np.diff(got) > 0) and got[0] >= 0 and got[-1] < n
