"""Parity of the reassociated order R = X (S B^T) of the Gaussian sketch.

P = S B^T (K x k) is formed first, then R = X P (2 K d k + 2 rows K k flops
instead of 2 rows K d + 2 rows d k).  References:
  * FP32 form (dense SIMT GEMMs, sparse CSR SpMM): the FP64 oracle of the
    same order, 1e-5 norm-wise per half-step (the tolerance of the paper
    order, which equals it in exact arithmetic);
  * BF16 and FP8 forms (tcgen05): the exact FP64 oracle within the bound of
    oracle/bounds.py derived from the unit roundoff at the form's fixed
    rounding points (bf16: X, S, Y, B where it enters P, and P; fp8: X and
    P in E4M3); diagnostic: the oracle's frozen rounding models of the same
    points <= 3e-4;
  * a short bf16 run with closing fp32 iterations ends within 2e-3 of the
    oracle's final relative error.
Shapes span several tiles, ragged row tails, the 64- and 128-wide N tiles of
the streaming product (k <= 64 and 64 < k <= 128) and d of one to eight
256-wide chunks.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import bounds, method
from synthdata import initial_factors, planted_dense, sparse_text

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _run_half(pkg, m, n, k, d, d_v, side, U, V, solver, precision, dense=None, csr=None, t=2, seed=21):
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=seed, d_v=d_v, solver=solver, precision=precision, t=t,
                   order=pkg.ORDER_REASSOCIATED)
    if dense is not None:
        h.set_dense(dense)
    else:
        h.set_csr(*csr)
    h.set_factors(U, V)
    h.half_step(side)
    Ug, Vg = h.factors()
    h.close()
    return Ug if side == 0 else Vg


def _oracle(X64, U, V, side, dd, solver, t=2, seed=21, bf16=False):
    X = X64 if side == 0 else X64.T
    if sp.issparse(X):
        X = X.tocsr()
    Y = (V if side == 0 else U).astype(np.float64)
    Z = (U if side == 0 else V).astype(np.float64)
    S = method.Sketch(method.GAUSSIAN, seed, t, side, X.shape[1], dd)
    return method.half_step(X, Y, Z, S, solver, method.mu_t(1.0, 1.0, t), bf16=bf16, reassociate=True)


FP32_CASES = [
    # m, n, k, d, d_v
    (333, 257, 10, 40, 50),
    (640, 515, 64, 130, 129),
    (300, 260, 100, 96, 96),
    (129, 70, 1, 9, 9),
]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("case", FP32_CASES)
def test_fp32_dense_half_steps(pkg, case, solver):
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 1)
    U, V = initial_factors(m, n, k, 2)
    for side, dd in ((0, d), (1, d_v)):
        got = _run_half(pkg, m, n, k, d, d_v, side, U, V, solver, pkg.FP32, dense=M)
        want = _oracle(M.astype(np.float64), U, V, side, dd, solver)
        assert got.min() >= 0
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


@pytest.mark.parametrize("solver", [0, 1])
def test_fp32_sparse_half_steps(pkg, solver):
    m, n, k = 700, 300, 16
    rp, col, val = sparse_text(m, n, 9, mean_len=12.0)
    Msp = sp.csr_matrix((val.astype(np.float64), col, rp), shape=(m, n))
    U, V = initial_factors(m, n, k, 7)
    for side, dd in ((0, 60), (1, 70)):
        got = _run_half(pkg, m, n, k, 60, 70, side, U, V, solver, pkg.FP32, csr=(rp, col, val))
        want = _oracle(Msp, U, V, side, dd, solver)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


BF16_CASES = [
    (256, 128, 16, 256, 256),
    (1000, 808, 10, 104, 96),
    (640, 520, 64, 520, 264),
    (384, 1032, 128, 768, 256),
    (136, 200, 32, 2048, 64),
    (2056, 4104, 100, 512, 1024),
]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("case", BF16_CASES)
def test_bf16_half_steps(pkg, case, solver):
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 2)
    U, V = initial_factors(m, n, k, 3)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        got = _run_half(pkg, m, n, k, d, d_v, side, U, V, solver, pkg.BF16, dense=M)
        assert got.min() >= 0
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 21, 2, side, X.shape[1], dd)
        rel, rb = bounds.check(got, X, Y, Z, S, solver, method.mu_t(1.0, 1.0, 2), "bf16_reassociated")
        assert rel <= rb, (side, rel, rb)
        model = _oracle(M64, U, V, side, dd, solver, bf16=True)
        assert _rel(got, model) <= 3e-4, (side, _rel(got, model))


def test_bf16_run_final_error(pkg):
    """bf16 reassociated iterations plus 3 closing fp32 iterations (paper
    order) end within 2e-3 of the oracle's final relative error."""
    m, n, k, d, T = 1000, 808, 10, 104, 30
    M, _, _ = planted_dense(m, n, k, 0)
    U0, V0 = method.default_init(0, m, n, k)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=0, precision=pkg.BF16, order=pkg.ORDER_REASSOCIATED,
                   use_graph=1)
    h.set_dense(M)
    h.step(T - 3)
    h.set_options(precision=pkg.FP32, order=pkg.ORDER_PAPER)
    h.step(3)
    err = h.rel_error()
    h.close()
    _, _, errs = method.run(M, U0, V0, 0, T, method.Options(sketch=method.GAUSSIAN, d=d))
    assert abs(err - errs[-1]) <= 2e-3, (err, errs[-1])


def test_graph_replay_equals_eager(pkg):
    """Replaying the captured iteration gives the eager iteration's factors."""
    m, n, k, d = 520, 264, 32, 256
    M, _, _ = planted_dense(m, n, 16, 5)
    out = []
    for g in (0, 1):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=4, precision=pkg.BF16, order=pkg.ORDER_REASSOCIATED,
                       use_graph=g)
        h.set_dense(M)
        h.step(4)
        out.append(h.factors())
        h.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_reassociated_rejects_other_forms(pkg):
    h = pkg.DSANLS(256, 128, 8, 64, pkg.GAUSSIAN, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(order=2)
    h.close()
    h = pkg.DSANLS(256, 128, 8, 64, pkg.SUBSAMPLE, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(order=pkg.ORDER_REASSOCIATED)
    h.close()


IDENT_CASES = [(256, 136, 16), (1000, 808, 10), (520, 264, 100)]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("case", IDENT_CASES)
def test_bf16_identity_half_steps(pkg, case, solver):
    """The unsketched subproblem (S = I) in bf16: R = X Y on the streaming
    tensor-core product, against the exact oracle within the derived bound
    (X and Y rounded, G = Y^T Y from the unrounded Y); diagnostic: the
    oracle's bf16 model <= 3e-4."""
    m, n, k = case
    M, _, _ = planted_dense(m, n, min(k, 16), 6)
    U, V = initial_factors(m, n, k, 8)
    M64 = M.astype(np.float64)
    for side in (0, 1):
        h = pkg.DSANLS(m, n, k, n, pkg.IDENTITY, seed=1, solver=solver, precision=pkg.BF16, t=3)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.IDENTITY, 1, 3, side, X.shape[1], X.shape[1])
        mu = method.mu_t(1.0, 1.0, 3)
        rel, rb = bounds.check(got, X, Y, Z, S, solver, mu, "bf16_identity")
        assert rel <= rb, (side, rel, rb)
        model = method.half_step(X, Y, Z, S, solver, mu, bf16=True)
        assert _rel(got, model) <= 3e-4, (side, _rel(got, model))


@pytest.mark.parametrize("kind", ["rademacher", "count", "srht"])
@pytest.mark.parametrize("precision,order", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_other_dense_sketch_half_steps(pkg, kind, precision, order):
    """The +-1/sqrt(d), count and SRHT sketches run through every dense-sketch
    path: FP32, BF16 and FP8 in both orders.  FP32 against the exact oracle
    (1e-5); BF16 / FP8 against the exact oracle within the derived bound of
    the form, and (diagnostic) the oracle's rounding models (3e-4)."""
    m, n, k, d, d_v = 640, 528, 32, 264, 136
    M, _, _ = planted_dense(m, n, 16, 3)
    U, V = initial_factors(m, n, k, 4)
    M64 = M.astype(np.float64)
    gkind, okind = {"rademacher": (pkg.RADEMACHER, method.RADEMACHER), "count": (pkg.COUNT, method.COUNT),
                    "srht": (pkg.SRHT, method.SRHT)}[kind]
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, gkind, seed=9, d_v=d_v, precision=precision, order=order, t=5)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(okind, 9, 5, side, X.shape[1], dd)
        mu = method.mu_t(1.0, 1.0, 5)
        want = method.half_step(X, Y, Z, S, 0, mu, bf16=precision == 1, fp8=(9, 5, side) if precision == 2 else None,
                                reassociate=order == 1)
        tol = 1e-5 if precision == 0 else 3e-4
        assert _rel(got, want) <= tol, (side, _rel(got, want))
        if precision:
            form = {(1, 0): "bf16", (1, 1): "bf16_reassociated", (2, 0): "fp8", (2, 1): "fp8_reassociated"}[
                (precision, order)]
            rel, rb = bounds.check(got, X, Y, Z, S, 0, mu, form)
            assert rel <= rb, (side, rel, rb)


@pytest.mark.parametrize("case", [(1000, 808, 10, 104, 96), (640, 520, 64, 520, 264), (2056, 4104, 100, 512, 1024)])
def test_bf16_reassociated_inner_steps(pkg, case):
    """bf16 reassociated terms with 8 projected-gradient steps on the proximal
    objective: the exact oracle's 8 steps within the derived bound (per-step
    terms added: each step map is nonexpansive), and (diagnostic) the
    oracle's bf16 model with the same steps (<= 3e-4)."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 7)
    U, V = initial_factors(m, n, k, 9)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=3, d_v=d_v, precision=pkg.BF16,
                       order=pkg.ORDER_REASSOCIATED, t=4, inner_iters=8)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 3, 4, side, X.shape[1], dd)
        want = method.half_step(X, Y, Z, S, 0, method.mu_t(1.0, 1.0, 4), bf16=True, reassociate=True,
                                inner_iters=8)
        assert _rel(got, want) <= 3e-4, (side, _rel(got, want))
        rel, rb = bounds.check(got, X, Y, Z, S, 0, method.mu_t(1.0, 1.0, 4), "bf16_reassociated", inner_iters=8)
        assert rel <= rb, (side, rel, rb)


FP8_CASES = [(256, 128, 16, 256, 256), (1024, 816, 10, 104, 96), (640, 528, 64, 520, 264), (2064, 4112, 100, 512, 1024)]


@pytest.mark.parametrize("case", FP8_CASES)
def test_fp8_reassociated_half_steps(pkg, case):
    """fp8 streaming product (M per block and P^T per row in E4M3) against the
    exact oracle within the derived fp8 bound (E4M3 keeps 3 fraction bits);
    diagnostic: the oracle's fp8 model of this order <= 3e-4 (the same codes
    and scales up to the rare rounding-boundary flip of a code)."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 11)
    U, V = initial_factors(m, n, k, 12)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        got = _run_half(pkg, m, n, k, d, d_v, side, U, V, 0, pkg.FP8, dense=M, t=3, seed=13)
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 13, 3, side, X.shape[1], dd)
        mu = method.mu_t(1.0, 1.0, 3)
        assert got.min() >= 0
        rel, rb = bounds.check(got, X, Y, Z, S, 0, mu, "fp8_reassociated")
        assert rel <= rb, (side, rel, rb)
        model = method.half_step(X, Y, Z, S, 0, mu, fp8=(13, 3, side), reassociate=True)
        assert _rel(got, model) <= 3e-4, (side, _rel(got, model))


def test_fp8_reassociated_run_final_error(pkg):
    """fp8 reassociated iterations plus 3 closing fp32 iterations end within
    2e-3 of the oracle's final relative error."""
    m, n, k, d, T = 1024, 816, 10, 104, 30
    M, _, _ = planted_dense(m, n, k, 0)
    U0, V0 = method.default_init(0, m, n, k)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=0, precision=pkg.FP8, order=pkg.ORDER_REASSOCIATED, use_graph=1)
    h.set_dense(M)
    h.step(T - 3)
    h.set_options(precision=pkg.FP32, order=pkg.ORDER_PAPER)
    h.step(3)
    err = h.rel_error()
    h.close()
    _, _, errs = method.run(M, U0, V0, 0, T, method.Options(sketch=method.GAUSSIAN, d=d))
    assert abs(err - errs[-1]) <= 2e-3, (err, errs[-1])


@pytest.mark.parametrize("precision,order", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1)])
def test_new_dense_data_in_a_captured_handle(pkg, precision, order):
    """set_dense on a handle whose iteration graph was captured on other data
    (the buffers are refilled in place and the graph kept): the factors and
    the relative error equal those of a fresh handle on the new data."""
    m, n, k, d = 1024, 768, 32, 128
    M1, _, _ = planted_dense(m, n, 16, 1)
    M2, _, _ = planted_dense(m, n, 16, 2)
    U0, V0 = initial_factors(m, n, k, 4)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=3, precision=precision, order=order, use_graph=1)
    h.set_dense(M1)
    h.set_factors(U0, V0)
    h.step(2)
    h.rel_error()
    h.set_dense(M2)
    h.set_factors(U0, V0)
    h.set_options(t=0)
    h.step(2)
    got_u, got_v = h.factors()
    got_e = h.rel_error()
    h.close()
    ref = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=3, precision=precision, order=order, use_graph=1)
    ref.set_dense(M2)
    ref.set_factors(U0, V0)
    ref.step(2)
    want_u, want_v = ref.factors()
    want_e = ref.rel_error()
    ref.close()
    assert np.array_equal(got_u, want_u) and np.array_equal(got_v, want_v)
    assert got_e == want_e
