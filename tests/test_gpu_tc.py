"""Parity of the bf16 and fp8 tensor-core (tcgen05) forms of the sketched products.

Acceptance reference: the exact FP64 oracle.  Each half-step must lie within
the bound of ``oracle/bounds.py``, derived from the unit roundoff of the
formats at the form's fixed rounding points (bf16 2^-8, E4M3 2^-4); a run
with three closing FP32 iterations must end within 2e-3 of the oracle's final
relative error.  Diagnostic: the oracle's deterministic rounding models of
the same points (frozen; they differ from the GPU only in fp32 accumulation
order), <= 2e-4 (bf16) and 3e-4 (fp8) per step.
Shapes span several 128 x 256 tiles with ragged row tails and several d-chunks.
"""
import numpy as np
import pytest

from oracle import bounds, method
from synthdata import initial_factors, planted_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


CASES = [
    # m, n, k, d, d_v
    (256, 128, 16, 256, 256),
    (1000, 808, 10, 104, 96),
    (640, 520, 64, 520, 264),
    (384, 1032, 128, 768, 256),
    (136, 200, 32, 2048, 64),
]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_bf16_half_steps(pkg, case, solver):
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 2)
    U, V = initial_factors(m, n, k, 3)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=21, d_v=d_v, solver=solver, precision=pkg.BF16, t=2)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 21, 2, side, X.shape[1], dd)
        mu = method.mu_t(1.0, 1.0, 2)
        assert got.min() >= 0
        rel, rb = bounds.check(got, X, Y, Z, S, solver, mu, "bf16")
        assert rel <= rb, (side, rel, rb)
        model = method.half_step(X, Y, Z, S, solver, mu, bf16=True)
        assert _rel(got, model) <= 2e-4, (side, _rel(got, model))


def test_bf16_run_final_error(pkg):
    """Reduced precision plus closing fp32 iterations ends within 2e-3 of the
    oracle's final relative error (planted 1000 x 808, k = 10, d = 104)."""
    m, n, k, d, T = 1000, 808, 10, 104, 30
    M, _, _ = planted_dense(m, n, k, 0)
    U0, V0 = method.default_init(0, m, n, k)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=0, precision=pkg.BF16)
    h.set_dense(M)
    h.step(T - 3)
    h.set_options(precision=pkg.FP32)
    h.step(3)
    err = h.rel_error()
    h.close()
    _, _, errs = method.run(M, U0, V0, 0, T, method.Options(sketch=method.GAUSSIAN, d=d))
    assert abs(err - errs[-1]) <= 2e-3, (err, errs[-1])


def test_bf16_rejects_unsupported_shapes(pkg):
    h = pkg.DSANLS(104, 64, 8, 20, pkg.GAUSSIAN, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(precision=pkg.BF16)  # d = 20 is not a multiple of 8
    h.close()
    h = pkg.DSANLS(100, 64, 8, 16, pkg.GAUSSIAN, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(precision=pkg.BF16)  # m = 100 is not a multiple of 8
    h.close()
    h = pkg.DSANLS(100, 64, 8, 16, pkg.SUBSAMPLE, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(precision=pkg.BF16)
    h.close()


FP8_CASES = [
    (256, 128, 16, 256, 256),
    (1024, 816, 10, 104, 96),
    (640, 528, 64, 520, 264),
]


@pytest.mark.parametrize("case", FP8_CASES)
def test_fp8_half_steps(pkg, case):
    """fp8 form against the exact oracle within the derived fp8 bound (E4M3
    keeps 3 fraction bits); diagnostic: the oracle's fp8 model (same E4M3
    codes and scales, fp32 accumulation order differs) <= 3e-4."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 4)
    U, V = initial_factors(m, n, k, 5)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=23, d_v=d_v, precision=pkg.FP8, t=2)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 23, 2, side, X.shape[1], dd)
        mu = method.mu_t(1.0, 1.0, 2)
        assert got.min() >= 0
        rel, rb = bounds.check(got, X, Y, Z, S, method.PGD, mu, "fp8")
        assert rel <= rb, (side, rel, rb)
        model = method.half_step(X, Y, Z, S, method.PGD, mu, fp8=(23, 2, side))
        assert _rel(got, model) <= 3e-4, (side, _rel(got, model))


def test_fp8_run_final_error(pkg):
    """fp8 form plus three closing fp32 iterations ends within 2e-3 of the
    oracle's final relative error."""
    m, n, k, d, T = 1024, 816, 10, 104, 30
    M, _, _ = planted_dense(m, n, k, 0)
    U0, V0 = method.default_init(0, m, n, k)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=0, precision=pkg.FP8)
    h.set_dense(M)
    h.step(T - 3)
    h.set_options(precision=pkg.FP32)
    h.step(3)
    err = h.rel_error()
    h.close()
    _, _, errs = method.run(M, U0, V0, 0, T, method.Options(sketch=method.GAUSSIAN, d=d))
    assert abs(err - errs[-1]) <= 2e-3, (err, errs[-1])


def test_fp8_columns_of_very_different_scale(pkg):
    """Data whose columns differ in scale by a factor 1000 (M = U0 V0^T D with
    D = diag(10^(3 c / n))): the fp8 form keeps one scale per 128-row block of
    the K-major operand (per 128 rows of M for the U-half, per 128 columns of M
    for the V-half), so the small columns of a row block sit up to 1000x
    below its scale, down to E4M3's subnormal range.  The half-steps must stay
    within the derived fp8 bound against the exact oracle (the bound's
    absolute floor 2^-10 scale covers the subnormal rounding)."""
    m, n, k, d = 640, 528, 32, 264
    M, _, _ = planted_dense(m, n, 16, 6)
    M = (M * np.power(10.0, 3.0 * np.arange(n) / n)[None, :]).astype(np.float32)
    U, V = initial_factors(m, n, k, 7)
    M64 = M.astype(np.float64)
    for side in (0, 1):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=29, precision=pkg.FP8, t=2)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 29, 2, side, X.shape[1], d)
        rel, rb = bounds.check(got, X, Y, Z, S, method.PGD, method.mu_t(1.0, 1.0, 2), "fp8")
        assert rel <= rb, (side, rel, rb)


@pytest.mark.parametrize("case", [(1000, 808, 10, 104, 96), (640, 520, 64, 520, 264), (136, 200, 32, 2048, 64)])
def test_sketch_drawn_inside_the_gemm_is_bitwise_the_prepass(pkg, case):
    """regen_sketch = 1 draws the Gaussian S^T tiles inside the tensor-core GEMMs
    (B = Y^T S and the fused R = (X S) B^T) from the Philox field instead of
    reading the sketch pre-pass through TMA: the tiles are the same bf16 values,
    so three outer iterations give bitwise equal factors."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 3)
    out = []
    for regen in (0, 1):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=31, d_v=d_v, precision=pkg.BF16, regen_sketch=regen,
                       use_graph=1)
        h.set_dense(M)
        h.step(3)
        out.append(h.factors())
        h.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["FP32", "BF16", "FP8"])
def test_set_dense_refill_matches_a_fresh_handle(pkg, prec):
    """A second set_dense on a handle refills M, its transpose and the reduced-precision
    copies in place (host data arrives in row chunks, each chunk transposed and cast on
    a second stream while the next is copied; 20,000 x 4,096 floats make two chunks):
    the half-steps that follow are bit for bit those of a fresh handle given the same
    data."""
    m, n, k, d = 20000, 4096, 16, 64
    p = getattr(pkg, prec)
    M1, _, _ = planted_dense(m, n, 8, 31)
    M2, _, _ = planted_dense(m, n, 8, 32)
    U, V = initial_factors(m, n, k, 33)
    out = []
    for refill in (True, False):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=4, precision=p, t=1)
        if refill:
            h.set_dense(M1)
            h.step(1)
            h.set_options(t=1)  # the same sketches as the fresh handle's
        h.set_dense(M2)
        h.set_factors(U, V)
        h.half_step(0)
        h.half_step(1)
        out.append(h.factors())
        h.close()
    (u0, v0), (u1, v1) = out
    assert np.array_equal(u0, u1) and np.array_equal(v0, v1)
