"""Parity of the GPU half-steps and outer iterations with the FP64 oracle.

Tolerance (binary32 path): norm-wise relative difference of the updated
factor <= 1e-5 from an identical input state (U^t, V^t, t) -- the sketch values
are bit-identical on both sides, so the difference is binary32 rounding of
the products A = X S (length-n sums), B = Y^T S, R = A B^T and the update,
i.e. O(sqrt(n) * 2^-24) relative, far below 1e-5 at these sizes.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import method, rng
from synthdata import initial_factors, planted_dense, sparse_text

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_half(M64, U, V, kind, solver, seed, t, side, d, alpha=1.0, beta=1.0, sparse=False):
    X = M64 if side == 0 else M64.T
    if sparse:
        X = X.tocsr()
    Y = V if side == 0 else U
    Z = U if side == 0 else V
    S = method.Sketch(kind, seed, t, side, X.shape[1], d)
    mu = method.mu_t(alpha, beta, t)
    return method.half_step(X, Y.astype(np.float64), Z.astype(np.float64), S, solver, mu)


def _gpu_half(pkg, M, U, V, kind, solver, seed, t, side, d, d_v=None, csr=None):
    m, n = U.shape[0], V.shape[0]
    k = U.shape[1]
    h = pkg.DSANLS(m, n, k, d, kind, seed=seed)
    opts = dict(solver=solver, t=t)
    if d_v is not None:
        opts["d_v"] = d_v
    h.set_options(**opts)
    if csr is None:
        h.set_dense(M)
    else:
        h.set_csr(*csr)
    h.set_factors(U, V)
    h.half_step(side)
    Ug, Vg = h.factors()
    G, eta = h.gram(side)
    h.close()
    return (Ug if side == 0 else Vg), G, eta


CASES = [
    # m, n, k, d, d_v
    (333, 257, 10, 40, 50),
    (1000, 800, 10, 100, 100),
    (640, 515, 64, 130, 129),
    (300, 260, 100, 96, 96),
    (260, 300, 128, 64, 70),
    (129, 70, 1, 9, 9),
]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_dense_gaussian_half_steps(pkg, case, solver):
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 1)
    U, V = initial_factors(m, n, k, 2)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        t = 3
        got, G, eta = _gpu_half(pkg, M, U, V, method.GAUSSIAN, solver, 11, t, side, d, d_v=d_v)
        want = _oracle_half(M64, U, V, method.GAUSSIAN, solver, 11, t, side, dd)
        assert got.min() >= 0
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))
        # the Gram matrix and step size of that half-step
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 11, t, side, X.shape[1], dd)
        _, _, Go, _ = method.sketched_terms(X, Y, S)
        assert _rel(G, Go) <= 1e-5
        if solver == 0:
            eta_o = 1.0 / (method.lambda_max(Go) + method.mu_t(1.0, 1.0, t))
            assert abs(eta - eta_o) <= 1e-5 * eta_o


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("case", CASES[:5])
def test_dense_subsample_half_steps(pkg, case, solver):
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 3)
    U, V = initial_factors(m, n, k, 4)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        got, _, _ = _gpu_half(pkg, M, U, V, method.SUBSAMPLE, solver, 5, 7, side, d, d_v=d_v)
        want = _oracle_half(M64, U, V, method.SUBSAMPLE, solver, 5, 7, side, dd)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


SPLIT_CASES = [
    # m, n (multiples of 8: the FP32 product runs on tensor cores from three-way bf16
    # splits), k, d, d_v: several 128 x 256 tiles, ragged row tails, d not a multiple of 256
    (1032, 520, 64, 264, 136),
    (264, 1040, 128, 520, 72),
    (136, 64, 1, 8, 16),
    (2056, 4104, 100, 512, 1024),
]


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("case", SPLIT_CASES)
def test_dense_fp32_split_tensor_core_half_steps(pkg, case, order):
    """The FP32 form of dense Gaussian products on tcgen05 (A = X S in the paper
    order, R = X P in the reassociated order; six bf16 products of the splits)
    against the exact oracle at the binary32 tolerance (1e-5 per step)."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 8)
    U, V = initial_factors(m, n, k, 9)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=17, d_v=d_v, t=3, order=order)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 17, 3, side, X.shape[1], dd)
        want = method.half_step(X, Y, Z, S, 0, method.mu_t(1.0, 1.0, 3), reassociate=order == 1)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


UPDATE_CASES = [
    # m, n, k, d, d_v for the tensor-core row update (32 < k <= 128): several 128-row
    # tiles per CTA (the double-buffered bulk copies of Z), ragged last tiles whose
    # bytes are not a multiple of 16 (read without the bulk copy), k not a multiple
    # of 4 (scalar row slices), one and two 64-column K atoms
    (70001, 300, 99, 64, 64),
    (40000, 333, 50, 48, 48),
    (20001, 257, 77, 80, 80),
    (300, 261, 112, 64, 64),
    (19457, 130, 128, 40, 40),
    (60001, 90, 36, 30, 30),
]


@pytest.mark.parametrize("case", UPDATE_CASES)
def test_tensor_core_update_tiles(pkg, case):
    """One projected-gradient half-step through the tensor-core row update against
    the exact oracle, norm-wise and on every 128-row tile (a tile computed wrong
    would hide in the norm of tens of thousands of rows)."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, 16, 12)
    U, V = initial_factors(m, n, k, 13)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        got, _, _ = _gpu_half(pkg, M, U, V, method.SUBSAMPLE, 0, 9, 5, side, d, d_v=d_v)
        want = _oracle_half(M64, U, V, method.SUBSAMPLE, 0, 9, 5, side, dd)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))
        rows = got.shape[0]
        worst = max(_rel(got[r:r + 128], want[r:r + 128]) for r in range(0, rows, 128))
        assert worst <= 4 * TOL_STEP, (side, worst)


@pytest.mark.parametrize("solver", [0, 1])
def test_dense_identity_half_steps(pkg, solver):
    m, n, k = 200, 150, 12
    M, _, _ = planted_dense(m, n, k, 5)
    U, V = initial_factors(m, n, k, 6)
    M64 = M.astype(np.float64)
    for side, dd in ((0, n), (1, m)):
        got, _, _ = _gpu_half(pkg, M, U, V, method.IDENTITY, solver, 0, 2, side, n, d_v=m)
        want = _oracle_half(M64, U, V, method.IDENTITY, solver, 0, 2, side, dd)
        assert _rel(got, want) <= TOL_STEP


def _csr(m, n, seed):
    rp, col, val = sparse_text(m, n, seed, mean_len=12.0)
    return rp, col, val, sp.csr_matrix((val.astype(np.float64), col, rp), shape=(m, n))


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("kind", [method.SUBSAMPLE, method.GAUSSIAN, method.IDENTITY])
def test_sparse_half_steps(pkg, kind, solver):
    m, n, k = 700, 300, 16
    rp, col, val, Msp = _csr(m, n, 9)
    U, V = initial_factors(m, n, k, 7)
    d, d_v = (n, m) if kind == method.IDENTITY else (60, 70)
    for side, dd in ((0, d), (1, d_v)):
        got, _, _ = _gpu_half(pkg, None, U, V, kind, solver, 3, 4, side, d, d_v=d_v, csr=(rp, col, val))
        want = _oracle_half(Msp, U, V, kind, solver, 3, 4, side, dd, sparse=True)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


def _csr_with_long_rows(m, n, seed):
    """Short random rows (about 10 entries) plus rows 7 and 123 with 3,000 and
    4,500 entries and a column 0 present in 2,500 rows: rows of M and of M^T
    longer than the 2,048 entries that the sampled product takes in one pass."""
    g = np.random.default_rng(seed)
    rows = []
    for i in range(m):
        length = {7: 3000, 123: 4500}.get(i, int(g.integers(1, 20)))
        cols = set(g.choice(n, size=length, replace=False).tolist())
        if i < 2500:
            cols.add(0)
        rows.append(sorted(cols))
    rp = np.zeros(m + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate([np.asarray(r, np.int32) for r in rows])
    val = np.log1p(g.poisson(1.0, size=len(col)) + 1.0).astype(np.float32)
    return rp, col, val, sp.csr_matrix((val.astype(np.float64), col, rp), shape=(m, n))


@pytest.mark.parametrize("solver", [0, 1])
def test_sparse_long_rows_half_steps(pkg, solver):
    """Subsampled sparse half-steps where rows of M and of M^T hold thousands
    of entries (long sampled columns in the gather, many sampled entries per
    row), with the unfused update kernels (k = 24: CUDA-core PGD and RCD),
    against the oracle."""
    m, n, k = 3000, 5000, 24
    rp, col, val, Msp = _csr_with_long_rows(m, n, 11)
    assert np.diff(rp).max() > 2048 and np.diff(Msp.T.tocsr().indptr).max() > 2048
    U, V = initial_factors(m, n, k, 5)
    for side, dd in ((0, 500), (1, 300)):
        got, _, _ = _gpu_half(pkg, None, U, V, method.SUBSAMPLE, solver, 6, 2, side, 500, d_v=300,
                              csr=(rp, col, val))
        want = _oracle_half(Msp, U, V, method.SUBSAMPLE, solver, 6, 2, side, dd, sparse=True)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


@pytest.mark.parametrize("case", [
    # m, n, k, d, d_v: row counts that take 1, 2 and 3 passes of the 8-bit radix sort
    (200, 150, 48, 40, 30),
    (3000, 5000, 100, 500, 300),
    (70000, 300, 40, 120, 2000),
])
def test_sparse_subsample_tensor_core_update(pkg, case):
    """One projected-gradient step with 32 < k <= 128 (tensor-core update) on
    sparse data with a subsampling sketch, R formed from the gathered sub-CSR
    of X[:, J]; against the oracle (1e-5).  The 3000 x 5000 case has rows of M
    and of M^T of 3,000 to 4,500 entries (rows of the sub-CSR with more than
    64 sampled entries are summed by a whole CTA) and a column present in
    2,500 rows."""
    m, n, k, d, d_v = case
    if m == 3000:
        rp, col, val, Msp = _csr_with_long_rows(m, n, 11)
    else:
        rp, col, val, Msp = _csr(m, n, 13)
    U, V = initial_factors(m, n, k, 5)
    for side, dd in ((0, d), (1, d_v)):
        got, _, _ = _gpu_half(pkg, None, U, V, method.SUBSAMPLE, 0, 6, 2, side, d, d_v=d_v, csr=(rp, col, val))
        want = _oracle_half(Msp, U, V, method.SUBSAMPLE, 0, 6, 2, side, dd, sparse=True)
        assert got.min() >= 0
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


def test_sparse_subsample_is_deterministic(pkg):
    """Two handles, and a captured graph against eager launches, give bitwise
    equal factors: the gathered entries are sorted stably by row, so every
    row's right-hand side is summed in the same (ascending column) order."""
    m, n, k = 3000, 5000, 100
    rp, col, val, _ = _csr_with_long_rows(m, n, 11)
    out = []
    for g in (0, 1, 1):
        h = pkg.DSANLS(m, n, k, 500, pkg.SUBSAMPLE, seed=6, d_v=300, use_graph=g)
        h.set_csr(rp, col, val)
        h.step(3)
        out.append(h.factors())
        h.close()
    for a in out[1:]:
        assert np.array_equal(out[0][0], a[0]) and np.array_equal(out[0][1], a[1])


def test_sparse_given_transpose_equals_built_transpose(pkg):
    m, n, k = 500, 200, 8
    rp, col, val, Msp = _csr(m, n, 4)
    T = Msp.T.tocsr()
    U, V = initial_factors(m, n, k, 1)
    a, _, _ = _gpu_half(pkg, None, U, V, method.SUBSAMPLE, 0, 2, 1, 1, 40, d_v=50, csr=(rp, col, val))
    b, _, _ = _gpu_half(pkg, None, U, V, method.SUBSAMPLE, 0, 2, 1, 1, 40, d_v=50,
                        csr=(rp, col, val, T.indptr.astype(np.int64), T.indices.astype(np.int32),
                             T.data.astype(np.float32)))
    assert np.array_equal(a, b)


def test_sparse_rel_error(pkg):
    m, n, k = 600, 250, 10
    rp, col, val, Msp = _csr(m, n, 2)
    U, V = initial_factors(m, n, k, 3)
    h = pkg.DSANLS(m, n, k, 40, pkg.SUBSAMPLE, seed=1)
    h.set_csr(rp, col, val)
    h.set_factors(U, V)
    e = h.rel_error()
    h.close()
    assert abs(e - method.rel_error(Msp, U.astype(np.float64), V.astype(np.float64))) <= 1e-6


def test_config0_run_tracks_oracle(pkg):
    """50 outer iterations of the planted 1000 x 800, k = 10, Gaussian d = 100 problem:
    relative error after every iteration within 1e-4 of the oracle's."""
    m, n, k, d, T = 1000, 800, 10, 100, 50
    M, _, _ = planted_dense(m, n, k, 0)
    U0, V0 = method.default_init(0, m, n, k)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=0)
    h.set_dense(M)
    Ug0, Vg0 = h.factors()
    assert np.array_equal(Ug0, U0) and np.array_equal(Vg0, V0)  # default init is the Philox uniform field
    errs = []
    for _ in range(T):
        h.step(1)
        errs.append(h.rel_error())
    U, V = h.factors()
    h.close()
    Uo, Vo, errs_o = method.run(M, U0, V0, 0, T, method.Options(sketch=method.GAUSSIAN, d=d))
    diffs = np.abs(np.array(errs) - np.array(errs_o))
    assert diffs.max() <= 1e-4, diffs.max()
    assert _rel(U @ V.T, Uo @ Vo.T) <= 1e-3


@pytest.mark.parametrize("kind,solver", [(0, 0), (0, 1), (1, 1)])
def test_graph_replay_is_bitwise_equal_to_eager(pkg, kind, solver):
    m, n, k, d = 400, 300, 16, 50
    M, _, _ = planted_dense(m, n, k, 8)
    out = []
    for use_graph in (0, 1):
        h = pkg.DSANLS(m, n, k, d, kind, seed=4, solver=solver, use_graph=use_graph)
        h.set_dense(M)
        h.step(5)
        out.append(h.factors())
        h.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_resume_from_checkpoint_is_bitwise(pkg):
    """S^t is a pure function of (seed, t, side): factors + t reproduce the trajectory."""
    m, n, k, d = 300, 200, 8, 30
    M, _, _ = planted_dense(m, n, k, 2)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=7)
    h.set_dense(M)
    h.step(10)
    U10, V10 = h.factors()
    h.close()
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=7)
    h.set_dense(M)
    h.step(5)
    U5, V5 = h.factors()
    h.close()
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=7, t=5)
    h.set_dense(M)
    h.set_factors(U5, V5)
    h.step(5)
    U, V = h.factors()
    h.close()
    assert np.array_equal(U, U10) and np.array_equal(V, V10)


@pytest.mark.parametrize("k", [4, 64, 100])  # the CUDA-core update and the tensor-core one (k > 32)
def test_nan_input_raises_numeric_error(pkg, k):
    m, n = 50, 40
    M, _, _ = planted_dense(m, n, 4, 0)
    h = pkg.DSANLS(m, n, k, 10, pkg.GAUSSIAN, seed=0)
    h.set_dense(M)
    U = np.ones((m, k), np.float32)
    U[3, 1] = np.nan
    h.set_factors(U, None)
    h.half_step(1)
    h.half_step(0)
    with pytest.raises(pkg.DSANLSError) as e:
        h.sync()
    assert e.value.code == -5
    h.sync()  # the flag is cleared once reported
    h.close()


def test_state_and_argument_errors(pkg):
    h = pkg.DSANLS(20, 10, 3, 5, pkg.SUBSAMPLE, seed=0)
    with pytest.raises(pkg.DSANLSError) as e:
        h.step(1)
    assert e.value.code == -4
    with pytest.raises(pkg.DSANLSError) as e:
        h.set_options(d_v=21)
    assert e.value.code == -1
    with pytest.raises(pkg.DSANLSError) as e:
        h.half_step(2)
    assert e.value.code == -1
    bad_rp = np.array([0, 2, 1] + [2] * 18, np.int64)  # decreasing
    with pytest.raises(pkg.DSANLSError):
        h.set_csr(bad_rp, np.array([0, 1], np.int32), np.ones(2, np.float32))
    h.close()


@pytest.mark.parametrize("k", [5, 64, 100])
def test_bound_clamp(pkg, k):
    m, n = 300, 280
    M, _, _ = planted_dense(m, n, 5, 0)
    M *= 1e-4
    U, V = initial_factors(m, n, k, 0)
    U *= 50.0
    h = pkg.DSANLS(m, n, k, 20, pkg.GAUSSIAN, seed=0, bound_clamp=1)
    h.set_dense(M)
    h.set_factors(U, V * 50.0)
    h.step(2)
    Ug, Vg = h.factors()
    h.close()
    bound = np.sqrt(2.0 * np.linalg.norm(M.astype(np.float64)))
    assert Ug.max() <= bound * (1 + 1e-6) and Vg.max() <= bound * (1 + 1e-6)


@pytest.mark.parametrize("k,solver", [(16, 1), (100, 0)])
def test_run_is_deterministic(pkg, k, solver):
    m, n, d = 500, 400, 64
    M, _, _ = planted_dense(m, n, 16, 3)
    outs = []
    for _ in range(2):
        h = pkg.DSANLS(m, n, k, d, pkg.SUBSAMPLE, seed=9, solver=solver)
        h.set_dense(M)
        h.step(4)
        outs.append(h.factors())
        h.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("inner", [2, 16])
@pytest.mark.parametrize("case", [(333, 257, 10, 40, 50), (640, 515, 64, 130, 129), (300, 260, 100, 96, 96)])
def test_pgd_inner_iterations(pkg, case, inner):
    """inner_iters projected-gradient steps on the proximal row objective per
    half-step against the oracle's pgd_inner (FP32 vs FP64, 1e-5)."""
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 3)
    U, V = initial_factors(m, n, k, 4)
    M64 = M.astype(np.float64)
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=5, d_v=d_v, t=3, inner_iters=inner)
        h.set_dense(M)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = Ug if side == 0 else Vg
        X = M64 if side == 0 else M64.T
        Y = (V if side == 0 else U).astype(np.float64)
        Z = (U if side == 0 else V).astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, 5, 3, side, X.shape[1], dd)
        want = method.half_step(X, Y, Z, S, method.PGD, method.mu_t(1.0, 1.0, 3), inner_iters=inner)
        assert _rel(got, want) <= TOL_STEP, (side, _rel(got, want))


def test_inner_iterations_need_pgd(pkg):
    h = pkg.DSANLS(64, 48, 4, 16, pkg.GAUSSIAN, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(solver=pkg.RCD, inner_iters=4)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(inner_iters=0)
    h.close()
