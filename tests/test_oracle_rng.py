"""Pins of the oracle's random streams (CPU only).

The sketch S^t of Section 3.4 must be regenerated identically from a shared
seed (Section 3.3, Alg. 2).  These tests pin the oracle's Philox field,
uniforms, Gaussian transform and subsampling permutation to facts fixed
outside the oracle: published known-answer vectors, the C library's log/sin/
cos (a special case that reduces to a library routine), distribution laws and
the permutation property.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(rng.philox4x32_10(ctr, key)) == out


def test_uniform_open_range_and_exactness():
    assert rng.uniform_open(0) == np.float32(2.0 ** -24)
    assert rng.uniform_open(0xFFFFFFFF) == np.float32(1.0 - 2.0 ** -24)
    ws = np.random.default_rng(1).integers(0, 2 ** 32, 2000, dtype=np.uint64)
    for w in ws:
        u = float(rng.uniform_open(int(w)))
        assert 0.0 < u < 1.0
        # exact: u * 2^24 is the odd integer 2*(w>>9)+1
        assert u * 2 ** 24 == 2 * (int(w) >> 9) + 1


def test_ln_matches_libm_within_two_ulp():
    words = list(np.random.default_rng(2).integers(0, 2 ** 32, 20000, dtype=np.uint64))
    words += [0, 1, 511, 512, 0xFFFFFFFF, 0xB504F300, 0x80000000, 0x7FFFFFFF]
    worst = 0.0
    for w in words:
        u = rng.uniform_open(int(w))
        ref = math.log(float(u))
        got = float(rng.lnf(u))
        ulp = float(np.spacing(np.float32(abs(ref))))
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 2.0, worst


def test_sincos_turn_matches_libm():
    words = list(np.random.default_rng(3).integers(0, 2 ** 32, 20000, dtype=np.uint64))
    # quadrant edges: 4u close to 0.5, 1.5, 2.5, 3.5 and to the integers
    for k in range(5):
        for off in (-3, -1, 0, 1, 3):
            a = (k * (1 << 22) - 1) // 2 + off
            if 0 <= a < (1 << 23):
                words.append(a << 9)
            b = ((2 * k + 1) * (1 << 21) - 1) // 2 + off
            if 0 <= b < (1 << 23):
                words.append(b << 9)
    for w in words:
        u = float(rng.uniform_open(int(w)))
        s, c = rng.sincos_turn(int(w))
        assert abs(float(s) - math.sin(2 * math.pi * u)) <= 2.5e-7
        assert abs(float(c) - math.cos(2 * math.pi * u)) <= 2.5e-7
        assert abs(float(s) ** 2 + float(c) ** 2 - 1.0) <= 6e-7


def test_field_addressing():
    seed, stream, t = 0x123456789ABCDEF, 1, 7
    W = rng.field_words(seed, stream, t, 10, 3)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(10):
        for j in range(3):
            blk = rng.philox4x32_10([i >> 2, j, t, stream], key)
            assert W[i, j] == blk[i & 3]


def test_gaussian_field_is_box_muller_of_field_words():
    seed, stream, t, rows, cols = 5, 0, 3, 9, 4
    scale = rng.gaussian_scale(cols)
    S = rng.gaussian_field(seed, stream, t, rows, cols, scale)
    W = rng.field_words(seed, stream, t, 12, cols)
    for q in range(3):
        for j in range(cols):
            for pair in range(2):
                wa, wb = W[4 * q + 2 * pair, j], W[4 * q + 2 * pair + 1, j]
                u1 = float(rng.uniform_open(int(wa)))
                u2 = float(rng.uniform_open(int(wb)))
                r = math.sqrt(-2.0 * math.log(u1))
                for off, ref in ((0, r * math.cos(2 * math.pi * u2)), (1, r * math.sin(2 * math.pi * u2))):
                    i = 4 * q + 2 * pair + off
                    if i < rows:
                        assert abs(float(S[i, j]) / float(scale) - ref) <= 4e-6 * max(1.0, abs(ref))


def test_gaussian_moments():
    n = 1 << 20
    z = rng.gaussian_field(11, 0, 0, n // 8, 8, np.float32(1.0)).ravel().astype(np.float64)
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * math.sqrt(24.0) * se
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # different t and different stream give uncorrelated draws
    z2 = rng.gaussian_field(11, 0, 1, n // 8, 8, np.float32(1.0)).ravel()
    z3 = rng.gaussian_field(11, 1, 0, n // 8, 8, np.float32(1.0)).ravel()
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5 * se
    assert abs(np.corrcoef(z, z3)[0, 1]) < 5 * se


def test_uniform_field_range_and_law():
    X = rng.uniform_field(0, rng.STREAM_INIT_U, 0, 4000, 50).ravel().astype(np.float64)
    assert X.min() >= 0.0 and X.max() < 1.0
    assert stats.kstest(X, "uniform").pvalue > 1e-4


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 100, 1000, 4097])
def test_feistel_cycle_walk_is_a_permutation(n):
    idx = rng.subsample_indices(9, 0, 4, n, n)
    assert np.array_equal(idx, np.arange(n))


def test_feistel_round_is_a_bijection_on_the_word_domain():
    h = rng.feistel_half_bits(50)
    assert (1 << (2 * h)) >= 50 and (1 << (2 * (h - 1))) < 50 or h == 1
    img = {rng.feistel_once(1, 1, 2, h, x) for x in range(1 << (2 * h))}
    assert img == set(range(1 << (2 * h)))


def test_subsample_inclusion_is_uniform():
    n, d, trials = 50, 10, 4000
    counts = np.zeros(n)
    pair = 0
    for t in range(trials):
        J = rng.subsample_indices(3, 0, t, n, d)
        assert len(np.unique(J)) == d and J.min() >= 0 and J.max() < n
        assert np.all(np.diff(J) > 0)
        counts[J] += 1
        pair += (0 in J) and (1 in J)
    expected = trials * d / n
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert stats.chi2.sf(chi2, n - 1) > 1e-4
    p_pair = d * (d - 1) / (n * (n - 1))
    assert abs(pair / trials - p_pair) < 5 * math.sqrt(p_pair * (1 - p_pair) / trials)


@pytest.mark.parametrize("kind", ["gaussian", "subsample", "rademacher", "count", "srht"])
def test_sketch_second_moment_is_identity(kind):
    """Assumption 1: E[S S^T] = I (Monte-Carlo over t)."""
    from oracle import method
    n, d, trials = 12, 4, 6000
    acc = np.zeros((n, n))
    kinds = {"gaussian": method.GAUSSIAN, "subsample": method.SUBSAMPLE, "rademacher": method.RADEMACHER,
             "count": method.COUNT, "srht": method.SRHT}
    for t in range(trials):
        S = method.Sketch(kinds[kind], 21, t, 0, n, d).dense()
        acc += S @ S.T
    mean = acc / trials
    # Gaussian: Var[(SS^T)_ii] = 2/d, off-diagonal 1/d; subsampling: diag (n/d)^2 p(1-p)
    tol = 6.0 * math.sqrt(max(2.0 / d, (n / d - 1.0)) / trials)
    assert np.max(np.abs(mean - np.eye(n))) < tol


def test_rademacher_field_values_and_balance():
    """Entries are exactly +-float32(1/sqrt(d)); the signs are balanced
    (binomial bound), uncorrelated between neighbouring entries, and differ
    between iterations and streams."""
    from scipy import stats
    d = 64
    sc = rng.gaussian_scale(d)
    S = rng.rademacher_field(5, 0, 3, 4096, d, sc)
    assert set(np.unique(S).tolist()) == {float(-sc), float(sc)}
    pos = int((S > 0).sum())
    assert stats.binomtest(pos, S.size, 0.5).pvalue > 1e-4
    sgn = np.sign(S).astype(np.float64)
    assert abs(np.mean(sgn[:, :-1] * sgn[:, 1:])) < 5.0 / math.sqrt(sgn[:, 1:].size)
    assert abs(np.mean(sgn[:-1] * sgn[1:])) < 5.0 / math.sqrt(sgn[1:].size)
    other_t = np.sign(rng.rademacher_field(5, 0, 4, 4096, d, sc))
    other_s = np.sign(rng.rademacher_field(5, 1, 3, 4096, d, sc))
    for o in (other_t, other_s):
        assert abs(np.mean(sgn * o)) < 5.0 / math.sqrt(sgn.size)


def test_count_sketch_structure_and_law():
    """One nonzero per row, equal to +-1; buckets uniform on [0, d) (chi-square)
    and signs balanced (binomial); hashes differ between iterations and sides."""
    n, d = 60000, 37
    S = rng.count_field(4, 0, 9, n, d)
    nz = S != 0
    assert np.all(nz.sum(axis=1) == 1) and set(np.unique(S[nz]).tolist()) == {-1.0, 1.0}
    h = np.argmax(nz, axis=1)
    counts = np.bincount(h, minlength=d)
    chi2 = float(np.sum((counts - n / d) ** 2 / (n / d)))
    assert stats.chi2.sf(chi2, d - 1) > 1e-4
    assert stats.binomtest(int((S[nz] > 0).sum()), n, 0.5).pvalue > 1e-4
    h_t, _ = rng.count_buckets(4, 0, 10, n, d)
    h_s, _ = rng.count_buckets(4, 1, 9, n, d)
    for o in (h_t, h_s):
        assert np.mean(o == h) < 1.0 / d + 5.0 * math.sqrt(1.0 / (d * n))


def _fwht(X):
    """Unnormalised fast Walsh-Hadamard transform along the last axis (length a
    power of two): the butterfly (a, b) -> (a + b, a - b) over doubling spans."""
    X = np.array(X, dtype=np.float64)
    p = X.shape[-1]
    h = 1
    while h < p:
        Y = X.reshape(X.shape[:-1] + (p // (2 * h), 2, h))
        a, b = Y[..., 0, :].copy(), Y[..., 1, :].copy()
        Y[..., 0, :], Y[..., 1, :] = a + b, a - b
        X = Y.reshape(X.shape)
        h *= 2
    return X


@pytest.mark.parametrize("n,d", [(16, 4), (13, 5), (100, 37), (128, 128), (70, 100)])
def test_srht_field_is_signs_times_sylvester_hadamard_columns(n, d):
    """S = sqrt(p/d) D H R: built here from scipy's Hadamard matrix (Sylvester's
    construction, a library routine) with the oracle's D and J, it matches the
    oracle's closed-form entries; every entry is +-float32(1/sqrt(d))."""
    from scipy.linalg import hadamard
    p = rng.srht_pad(n)
    assert p >= n and p & (p - 1) == 0 and (p == 1 or p // 2 < n)
    sc = rng.gaussian_scale(d)
    S = rng.srht_field(9, 1, 4, n, d, sc)
    D = rng.srht_signs(9, 1, 4, n)
    J = rng.srht_columns(9, 1, 4, n, d)
    assert len(J) == d and np.all(np.diff(J) > 0) and J[0] >= 0 and J[-1] < p
    want = math.sqrt(p / d) * (D[:, None] * hadamard(p)[:n][:, J] / math.sqrt(p))
    assert np.array_equal(np.sign(S), np.sign(want))
    assert np.all(np.abs(S) == sc)
    np.testing.assert_allclose(S, want, rtol=1e-6, atol=0)


def test_srht_with_every_column_is_orthogonal():
    """With d = p every Hadamard column is kept and S S^T = (p s^2) I exactly
    (H is orthogonal, D^2 = I): the off-diagonal sums cancel to zero."""
    for n in (64, 50):
        p = rng.srht_pad(n)
        sc = rng.gaussian_scale(p)
        S = rng.srht_field(2, 0, 7, n, p, sc).astype(np.float64)
        SS = S @ S.T
        off = SS - np.diag(np.diag(SS))
        assert np.all(off == 0.0)
        assert np.all(np.diag(SS) == p * np.float64(sc) ** 2)


def test_srht_product_equals_fast_transform():
    """X S = (fwht(X D) / sqrt(p))[:, J] sqrt(p/d), the transform form of the
    SRHT (the rows of X padded with zeros to p columns)."""
    g = np.random.default_rng(3)
    n, d = 200, 48
    p = rng.srht_pad(n)
    X = g.standard_normal((7, n))
    S = rng.srht_field(5, 0, 11, n, d, rng.gaussian_scale(d)).astype(np.float64)
    D = rng.srht_signs(5, 0, 11, n)
    J = rng.srht_columns(5, 0, 11, n, d)
    Xp = np.zeros((7, p))
    Xp[:, :n] = X * D[None, :]
    want = _fwht(Xp)[:, J] / math.sqrt(d)
    np.testing.assert_allclose(X @ S, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())


def test_srht_signs_and_columns_law():
    """Row signs balanced (binomial); the column subset is the subsampling draw
    over {0..p-1} (inclusion uniform, chi-square over t); signs and subsets
    differ between iterations and sides."""
    n = 50000
    D = rng.srht_signs(6, 0, 2, n)
    assert set(np.unique(D).tolist()) == {-1.0, 1.0}
    assert stats.binomtest(int((D > 0).sum()), n, 0.5).pvalue > 1e-4
    for o in (rng.srht_signs(6, 0, 3, n), rng.srht_signs(6, 1, 2, n)):
        assert abs(np.mean(D * o)) < 5.0 / math.sqrt(n)
    n, d, trials = 20, 6, 4000
    p = rng.srht_pad(n)
    counts = np.zeros(p)
    for t in range(trials):
        counts[rng.srht_columns(1, 1, t, n, d)] += 1
    expected = trials * d / p
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert stats.chi2.sf(chi2, p - 1) > 1e-4
    # its own stream: not the plain subsampling draw over the same range
    assert not np.array_equal(rng.srht_columns(1, 0, 0, 2000, 100), rng.subsample_indices(1, 0, 0, 2048, 100))


def test_srht_pin_catches_a_wrong_hadamard_index(monkeypatch):
    """A planted mistake in the oracle's entry rule (the parity taken with the
    lowest bit forced on, i.e. a wrong Hadamard index) fails the Sylvester pin."""
    from scipy.linalg import hadamard
    monkeypatch.setattr(rng, "_parity", lambda x, f=rng._parity: f(np.asarray(x) | 1))
    n, d = 16, 8
    S = rng.srht_field(9, 1, 4, n, d, rng.gaussian_scale(d))
    D = rng.srht_signs(9, 1, 4, n)
    J = rng.srht_columns(9, 1, 4, n, d)
    want = D[:, None] * hadamard(n)[:, J]
    assert not np.array_equal(np.sign(S), np.sign(want))
