"""Pins of the oracle's method steps (CPU only).

Each test checks the FP64 oracle against a fact fixed outside it: the
unbiasedness of the sketched gradient (Section 3.5.1), the reduction of the
sketched steps to textbook unsketched ones when S = I (HALS for Alg. 3 with
mu = 0; the plain projected-gradient step), the exact identity satisfied by a
projected step (Appendix B, eq. delta), monotone descent, coordinate-wise
optimality of Alg. 3, row independence (eq. u_block), Lemma 1's rescaling
invariance, library eigen-solvers and the dense/sparse error identity.
A final group plants mistakes into a copy of the oracle and checks that the
pins above catch them.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import method, rng
from synthdata import planted_dense


def _problem(m=30, n=24, k=4, seed=0):
    M, U0, V0 = planted_dense(m, n, k, seed)
    g = np.random.default_rng(seed + 100)
    U = g.random((m, k))
    V = g.random((n, k))
    return M.astype(np.float64), U, V


# --------------------------------------------------------------------------
# pin functions (take the oracle module so a mutated copy can be checked)
# --------------------------------------------------------------------------

def pin_unbiased_gradient(mod, kind, trials=3000):
    """E over S of (U G - R) equals U V^T V - M V (Section 3.5.1)."""
    M, U, V = _problem(8, 10, 3, 1)
    acc = np.zeros_like(U)
    for t in range(trials):
        S = mod.Sketch(kind, 5, t, 0, M.shape[1], 4)
        _, _, G, R = mod.sketched_terms(M, V, S)
        acc += U @ G - R
    mean = acc / trials
    exact = U @ (V.T @ V) - M @ V
    return np.max(np.abs(mean - exact)) / np.max(np.abs(exact))


def pin_identity_pgd(mod):
    """S = I: the sketched PGD step is the plain projected-gradient step."""
    M, U, V = _problem()
    S = mod.Sketch(mod.IDENTITY, 0, 0, 0, M.shape[1], M.shape[1])
    _, _, G, R = mod.sketched_terms(M, V, S)
    eta = 1.0 / (mod.lambda_max(G) + 0.5)
    got = mod.pgd_update(U, G, R, eta)
    want = method.project(U - eta * (U @ (V.T @ V) - M @ V))
    return np.max(np.abs(got - want))


def pin_identity_rcd_is_hals(mod):
    """S = I, mu = 0: Alg. 3 is the textbook HALS column sweep."""
    M, U, V = _problem()
    S = mod.Sketch(mod.IDENTITY, 0, 0, 0, M.shape[1], M.shape[1])
    _, _, G, R = mod.sketched_terms(M, V, S)
    got = mod.rcd_update(U, G, R, 0.0)
    Z = U.copy()
    XY, YY = M @ V, V.T @ V
    for j in range(Z.shape[1]):
        Z[:, j] = np.maximum(Z[:, j] + (XY[:, j] - Z @ YY[:, j]) / YY[j, j], 0.0)
    return np.max(np.abs(got - Z))


def pin_pgd_identity(mod):
    """(U^t - U^{t+1}) / eta = min(U^t / eta, U G - R) (Appendix B, eq. delta)."""
    M, U, V = _problem()
    S = mod.Sketch(mod.GAUSSIAN, 3, 2, 0, M.shape[1], 8)
    _, _, G, R = mod.sketched_terms(M, V, S)
    eta = 1.0 / (mod.lambda_max(G) + 1.0)
    Un = mod.pgd_update(U, G, R, eta)
    lhs = (U - Un) / eta
    rhs = np.minimum(U / eta, U @ G - R)
    return np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))


# --------------------------------------------------------------------------
# pins
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [method.GAUSSIAN, method.SUBSAMPLE, method.RADEMACHER, method.COUNT, method.SRHT])
def test_sketched_gradient_is_unbiased(kind):
    assert pin_unbiased_gradient(method, kind) < 0.08


def test_identity_sketch_reduces_to_plain_pg():
    assert pin_identity_pgd(method) < 1e-12


def test_identity_rcd_mu0_is_hals():
    assert pin_identity_rcd_is_hals(method) < 1e-12


def test_projected_step_identity():
    assert pin_pgd_identity(method) < 1e-12


def test_lambda_max_matches_eigvalsh():
    M, U, V = _problem(40, 60, 6, 4)
    for t in range(5):
        S = method.Sketch(method.GAUSSIAN, 1, t, 0, 60, 20)
        _, B, G, _ = method.sketched_terms(M, V, S)
        lam = method.lambda_max(G, 32)
        ref = np.linalg.eigvalsh(G)[-1]
        assert abs(lam - ref) <= 1e-6 * ref


@pytest.mark.parametrize("solver", [method.PGD, method.RCD])
def test_identity_sketch_descends(solver):
    """With S = I every half-step decreases ||M - U V^T||_F (step 1/(L+mu) for
    PGD; exact coordinate minimisation plus a proximal term for RCD)."""
    M, U, V = _problem(40, 30, 5, 2)
    opt = method.Options(sketch=method.IDENTITY, solver=solver, alpha=0.1, beta=0.0)
    f = np.linalg.norm(M - U @ V.T)
    for t in range(15):
        S = method.Sketch(method.IDENTITY, 0, t, 0, 30, 30)
        U = method.half_step(M, V, U, S, solver, 0.1)
        f1 = np.linalg.norm(M - U @ V.T)
        assert f1 <= f * (1 + 1e-12)
        S = method.Sketch(method.IDENTITY, 0, t, 1, 40, 40)
        V = method.half_step(M.T, U, V, S, solver, 0.1)
        f2 = np.linalg.norm(M - U @ V.T)
        assert f2 <= f1 * (1 + 1e-12)
        f = f2


def test_rcd_columns_are_coordinate_minimisers():
    """Each column from Alg. 3 minimises the 1-D proximal objective of eq. entry_sol:
    derivative zero where positive, nonnegative where clamped at 0."""
    M, U, V = _problem(25, 20, 4, 7)
    S = method.Sketch(method.GAUSSIAN, 2, 1, 0, 20, 12)
    A, B, G, R = method.sketched_terms(M, V, S)
    mu = 0.7
    Un = method.rcd_update(U, G, R, mu)
    k = U.shape[1]
    for j in range(k):
        Zj = np.concatenate([Un[:, :j], U[:, j:]], axis=1)
        # row-wise residual of the sketched objective with column j free
        others = np.delete(np.arange(k), j)
        Zo = Zj[:, others]
        x = Un[:, j]
        # d/dx [ ||A - x B_j - Zo B_o||^2 + mu (x - U_j)^2 ] / 2
        grad = x * (B[j] @ B[j]) - (A - Zo @ B[others]) @ B[j] + mu * (x - U[:, j])
        scale = np.max(np.abs(A @ B[j])) + 1.0
        assert np.all(np.abs(grad[x > 0]) <= 1e-9 * scale)
        assert np.all(grad[x == 0] >= -1e-9 * scale)


def test_half_step_is_row_independent():
    M, U, V = _problem(30, 24, 4, 9)
    S = method.Sketch(method.GAUSSIAN, 4, 0, 0, 24, 10)
    full = method.half_step(M, V, U, S, method.PGD, 1.0)
    rows = np.array([0, 7, 29])
    part = method.half_step(M, V, U, S, method.PGD, 1.0, rows=rows)
    assert np.allclose(full[rows], part, rtol=0, atol=1e-13)
    full = method.half_step(M, V, U, S, method.RCD, 1.0)
    part = method.half_step(M, V, U, S, method.RCD, 1.0, rows=rows)
    assert np.allclose(full[rows], part, rtol=0, atol=1e-13)


@pytest.mark.parametrize("solver", [method.PGD, method.RCD])
@pytest.mark.parametrize("kind", [method.GAUSSIAN, method.SUBSAMPLE])
def test_factors_stay_nonnegative(solver, kind):
    M, U, V = _problem(30, 24, 4, 3)
    opt = method.Options(sketch=kind, d=8, solver=solver)
    MT = M.T.copy()
    for t in range(10):
        U, V = method.outer_iteration(M, MT, U, V, 0, t, opt)
        assert U.min() >= 0 and V.min() >= 0


def test_rescaling_invariance_lemma1():
    M, U, V = _problem()
    D = np.diag([0.5, 2.0, 3.0, 0.25])
    assert abs(method.rel_error(M, U @ D, V @ np.linalg.inv(D)) - method.rel_error(M, U, V)) < 1e-13


def test_rel_error_of_an_exact_factorisation_is_zero():
    """M = U0 V0^T with small-integer factors (every product and sum exact in
    FP64): the relative error of Section 5.1 is exactly 0, dense and sparse."""
    g = np.random.default_rng(3)
    U0 = g.integers(0, 4, size=(37, 5)).astype(np.float64)
    V0 = g.integers(0, 4, size=(23, 5)).astype(np.float64)
    M = U0 @ V0.T
    assert method.rel_error(M, U0, V0) == 0.0
    assert method.rel_error(sp.csr_matrix(M), U0, V0) == 0.0


def test_rel_error_hand_computed_2x2():
    """M = [[1, 2], [3, 4]], U = [[1], [1]], V = [[1], [2]]: U V^T = [[1, 2],
    [1, 2]], M - U V^T = [[0, 0], [2, 2]], so the error is sqrt(8 / 30)."""
    M = np.array([[1.0, 2.0], [3.0, 4.0]])
    U = np.array([[1.0], [1.0]])
    V = np.array([[1.0], [2.0]])
    assert method.rel_error(M, U, V) == pytest.approx(np.sqrt(8.0 / 30.0), rel=1e-15)
    assert method.rel_error(sp.csr_matrix(M), U, V) == pytest.approx(np.sqrt(8.0 / 30.0), rel=1e-14)
    # a wrong normalisation (by ||U V^T|| or squared) would give another number
    assert abs(method.rel_error(M, U, V) - 8.0 / 30.0) > 0.1


def test_sparse_error_expansion_equals_direct():
    g = np.random.default_rng(0)
    D = g.random((40, 30))
    D[D < 0.7] = 0.0
    U, V = g.random((40, 5)), g.random((30, 5))
    direct = np.linalg.norm(D - U @ V.T) / np.linalg.norm(D)
    assert abs(method.rel_error(sp.csr_matrix(D), U, V) - direct) < 1e-12


def test_sketch_subsample_matches_dense_definition():
    M, U, V = _problem(10, 20, 3, 0)
    S = method.Sketch(method.SUBSAMPLE, 7, 3, 0, 20, 6)
    Sd = S.dense()
    assert np.allclose(S.right_multiply(M), M @ Sd, rtol=0, atol=1e-13)
    assert np.allclose(Sd.sum(axis=0), float(S.scale))
    assert math.isclose(float(S.scale) ** 2, 20 / 6, rel_tol=1e-6)


def test_sketched_run_reduces_error():
    M, U0, V0 = planted_dense(120, 90, 5, 0)
    U, V = method.default_init(0, 120, 90, 5)
    opt = method.Options(sketch=method.GAUSSIAN, d=30, solver=method.PGD)
    _, _, errs = method.run(M, U, V, 0, 30, opt)
    assert errs[-1] < 0.75 * errs[0]
    opt = method.Options(sketch=method.SUBSAMPLE, d=30, solver=method.RCD)
    _, _, errs = method.run(M, U, V, 0, 30, opt)
    assert errs[-1] < 0.5 * errs[0]


def test_default_init_is_uniform_field():
    U, V = method.default_init(3, 17, 9, 4)
    assert U.shape == (17, 4) and V.shape == (9, 4)
    assert np.array_equal(U, rng.uniform_field(3, 2, 0, 17, 4))
    assert U.min() >= 0 and U.max() < 1


# --------------------------------------------------------------------------
# planted mistakes: a mutated copy of the oracle must fail at least one pin
# --------------------------------------------------------------------------

class _Mutant:
    def __init__(self, **over):
        self.__dict__.update({k: getattr(method, k) for k in dir(method) if not k.startswith("__")})
        self.__dict__.update(over)



def test_mutant_dropped_R_term_is_caught():
    def bad_pgd(Z, G, R, eta, bound=None):
        return method.project(Z - eta * (Z @ G))
    mut = _Mutant(pgd_update=bad_pgd)
    assert pin_pgd_identity(mut) > 1e-3 or pin_identity_pgd(mut) > 1e-3


def test_mutant_wrong_sign_in_rcd_is_caught():
    def bad_rcd(Z, G, R, mu, bound=None):
        Zold, Znew = Z, Z.copy()
        for j in range(Z.shape[1]):
            T = mu * Zold[:, j] + R[:, j]
            for l in range(j):
                T = T + G[l, j] * Znew[:, l]
            for l in range(j + 1, Z.shape[1]):
                T = T - G[l, j] * Zold[:, l]
            Znew[:, j] = method.project(T / (G[j, j] + mu))
        return Znew
    mut = _Mutant(rcd_update=bad_rcd)
    assert pin_identity_rcd_is_hals(mut) > 1e-3


def test_mutant_old_columns_in_rcd_is_caught():
    """Jacobi instead of Gauss-Seidel sweep (all l use U^t)."""
    def jacobi(Z, G, R, mu, bound=None):
        Znew = Z.copy()
        for j in range(Z.shape[1]):
            T = mu * Z[:, j] + R[:, j] - Z @ G[:, j] + G[j, j] * Z[:, j]
            Znew[:, j] = method.project(T / (G[j, j] + mu))
        return Znew
    mut = _Mutant(rcd_update=jacobi)
    assert pin_identity_rcd_is_hals(mut) > 1e-3


def test_mutant_unscaled_subsample_is_caught():
    class BadSketch(method.Sketch):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            if self.kind == method.SUBSAMPLE:
                self.scale = np.float32(1.0)
    mut = _Mutant(Sketch=BadSketch)
    assert pin_unbiased_gradient(mut, method.SUBSAMPLE, trials=1500) > 0.2


def test_mutant_missing_gaussian_scale_is_caught():
    """Entries N(0,1) instead of N(0,1/d) give E[S S^T] = d I."""
    class BadSketch(method.Sketch):
        def __init__(self, kind, seed, t, side, n, d):
            super().__init__(kind, seed, t, side, n, d)
            if kind == method.GAUSSIAN:
                self.dense32 = rng.gaussian_field(seed, side, t, n, d, 1.0)
    mut = _Mutant(Sketch=BadSketch)
    assert pin_unbiased_gradient(mut, method.GAUSSIAN, trials=300) > 0.2


def test_round_bf16_matches_torch():
    """The oracle's bf16 rounding equals torch's float32 -> bfloat16 conversion."""
    import torch
    g = np.random.default_rng(0)
    x = np.concatenate([g.standard_normal(20000).astype(np.float32) * 100,
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.0078125, 3.0e38, 1e-40], np.float32)])
    # exact ties in the 16 dropped bits
    x = np.concatenate([x, (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(method.round_bf16(x), want)


def test_round_e4m3_matches_torch():
    """The oracle's E4M3 rounding equals torch's float32 -> float8_e4m3fn conversion (in range)."""
    import torch
    g = np.random.default_rng(1)
    x = np.concatenate([g.standard_normal(20000).astype(np.float32) * 20,
                        g.uniform(-448, 448, 2000).astype(np.float32),
                        np.array([0.0, 1.0, 1.0625, 1.1875, 0.001953125, 0.0029296875, 447.9, 448.0, -3.0e-3],
                                 np.float32)])
    x = x[np.abs(x) <= 448.0]
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(method.round_e4m3(x), want)


def test_rowblock_quantisation_error_bound():
    """Per-block scaling keeps every entry within half an E4M3 quantum of its block."""
    g = np.random.default_rng(2)
    X = (g.random((300, 50)) * np.repeat([1.0, 100.0, 0.01], 100)[:, None]).astype(np.float32)
    Xd = method.quantise_rowblocks_e4m3(X)
    for r0 in range(0, 300, 128):
        blk = X[r0:r0 + 128].astype(np.float64)
        sc = blk.max() / 448.0
        assert np.all(np.abs(Xd[r0:r0 + 128] - blk) <= np.maximum(np.abs(blk) * 2.0 ** -4, sc * 2.0 ** -9) * 1.0001)


# --------------------------------------------------------------------------
# the reassociated order R = X (S B^T) and the rounding points of the bf16
# models
# --------------------------------------------------------------------------

class _FixedSketch:
    """A Gaussian-kind sketch with given binary32 values (for exact cases)."""

    def __init__(self, values):
        self.kind = method.GAUSSIAN
        self.dense32 = np.asarray(values, dtype=np.float32)
        self.n, self.d = self.dense32.shape
        self.scale = np.float32(1.0)
        self.J = None

    def dense(self):
        return self.dense32.astype(np.float64)

    def right_multiply(self, X):
        return np.asarray(X @ self.dense(), dtype=np.float64)


@pytest.mark.parametrize("kind", [method.GAUSSIAN, method.SUBSAMPLE, method.IDENTITY])
@pytest.mark.parametrize("sparse", [False, True])
def test_reassociated_order_equals_paper_order(kind, sparse):
    """(X S) B^T = X (S B^T): both orders give the same B, G and R."""
    M, U, V = _problem(40, 32, 5, 3)
    d = 32 if kind == method.IDENTITY else 12
    S = method.Sketch(kind, 11, 2, 0, 32, d)
    X = sp.csr_matrix(np.where(M > 0.6, M, 0.0)) if sparse else M
    _, B1, G1, R1 = method.sketched_terms(X, V, S)
    _, B2, G2, R2 = method.sketched_terms_reassociated(X, V, S)
    for a, b in ((B1, B2), (G1, G2), (R1, R2)):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("model", ["paper", "reassociated"])
def test_bf16_models_are_exact_on_representable_inputs(model):
    """Small integers are bf16 values and their products stay exact: the bf16
    models then equal the exact terms bit for bit."""
    g = np.random.default_rng(4)
    X = g.integers(0, 3, (9, 7)).astype(np.float64)
    Y = g.integers(0, 3, (7, 2)).astype(np.float64)
    S = _FixedSketch(g.integers(-1, 2, (7, 3)))
    f = method.sketched_terms_bf16 if model == "paper" else method.sketched_terms_reassociated_bf16
    _, B, G, R = f(X, Y, S)
    _, Be, Ge, Re = method.sketched_terms(X, Y, S)
    assert np.array_equal(B, Be) and np.array_equal(G, Ge) and np.array_equal(R, Re)


def test_reassociated_bf16_rounding_points():
    """Where the reassociated bf16 model rounds: X, Y, S on entry, B where it
    enters P (not in G), and P where it enters R.  Hand-computed: with
    S = [[1],[1]], Y = [[128],[129]]: B = 257 (G = 257^2 exact), round(B) = 256
    (tie to even), P = [[256],[256]], R = X P."""
    X = np.array([[1.0, 0.0]])
    _, B, G, R = method.sketched_terms_reassociated_bf16(X, np.array([[128.0], [129.0]]), _FixedSketch([[1.0], [1.0]]))
    assert B[0, 0] == 257.0 and G[0, 0] == 257.0 ** 2 and R[0, 0] == 256.0
    # P rounded: S = [[7],[1]], Y = [[0],[43]]: B = 43, P = [[301],[43]] -> 301 rounds to 300
    _, B, _, R = method.sketched_terms_reassociated_bf16(X, np.array([[0.0], [43.0]]), _FixedSketch([[7.0], [1.0]]))
    assert B[0, 0] == 43.0 and R[0, 0] == 300.0
    # X, Y and S rounded on entry: 1 + 2^-9 is not a bf16 value (rounds to 1)
    e = 1.0 + 2.0 ** -9
    _, B, _, R = method.sketched_terms_reassociated_bf16(np.array([[e, 0.0]]), np.array([[e], [0.0]]),
                                                         _FixedSketch([[e], [0.0]]))
    assert B[0, 0] == 1.0 and R[0, 0] == 1.0


def test_paper_order_bf16_rounding_points():
    """Where the paper-order bf16 model rounds: A = X S where it enters R, B
    where it enters R (not in G).  X = [[128, 129]], S = [[1],[1]]: A = 257 ->
    256; Y = [[1],[0]]: B = 1, R = 256."""
    _, B, G, R = method.sketched_terms_bf16(np.array([[128.0, 129.0]]), np.array([[1.0], [0.0]]),
                                            _FixedSketch([[1.0], [1.0]]))
    assert B[0, 0] == 1.0 and R[0, 0] == 256.0
    _, B, G, R = method.sketched_terms_bf16(np.array([[1.0, 0.0]]), np.array([[128.0], [129.0]]),
                                            _FixedSketch([[1.0], [1.0]]))
    assert B[0, 0] == 257.0 and G[0, 0] == 257.0 ** 2 and R[0, 0] == 256.0


def test_reassociated_bf16_error_is_small_but_nonzero():
    """On Gaussian data the bf16 reassociated R is within a few bf16 units of
    the exact R (relative Frobenius error between 1e-5 and 2e-2)."""
    M, U, V = _problem(64, 48, 6, 5)
    S = method.Sketch(method.GAUSSIAN, 3, 0, 0, 48, 16)
    _, _, _, Re = method.sketched_terms(M, V, S)
    _, _, _, Rb = method.sketched_terms_reassociated_bf16(M, V, S)
    rel = np.linalg.norm(Rb - Re) / np.linalg.norm(Re)
    assert 1e-5 < rel < 2e-2


def test_reassociated_half_step_matches_paper_order():
    """A full PGD half-step in either order agrees to rounding."""
    M, U, V = _problem(30, 24, 4, 6)
    S = method.Sketch(method.GAUSSIAN, 1, 4, 0, 24, 10)
    a = method.half_step(M, V, U, S, method.PGD, 2.0)
    b = method.half_step(M, V, U, S, method.PGD, 2.0, reassociate=True)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_identity_bf16_model_rounding_points():
    """S = I in bf16: R = round(X) round(Y), G from the unrounded Y.  With
    X = [[1, 1]] and Y = [[1 + 2^-9], [1]]: R = 2 (Y rounded), G = (1 + 2^-9)^2 + 1."""
    e = 1.0 + 2.0 ** -9
    S = method.Sketch(method.IDENTITY, 0, 0, 0, 2, 2)
    _, B, G, R = method.sketched_terms_bf16(np.array([[1.0, 1.0]]), np.array([[e], [1.0]]), S)
    assert R[0, 0] == 2.0 and G[0, 0] == e * e + 1.0 and B[0, 0] == e
    _, _, _, R = method.sketched_terms_bf16(np.array([[e, 0.0]]), np.array([[1.0], [0.0]]), S)
    assert R[0, 0] == 1.0


def test_identity_bf16_model_is_exact_on_representable_inputs():
    g = np.random.default_rng(8)
    X = g.integers(0, 4, (7, 6)).astype(np.float64)
    Y = g.integers(0, 4, (6, 3)).astype(np.float64)
    S = method.Sketch(method.IDENTITY, 0, 0, 0, 6, 6)
    _, B, G, R = method.sketched_terms_bf16(X, Y, S)
    _, Be, Ge, Re = method.sketched_terms(X, Y, S)
    assert np.array_equal(B, Be) and np.array_equal(G, Ge) and np.array_equal(R, Re)


# --------------------------------------------------------------------------
# several projected-gradient steps on the proximal subproblem
# --------------------------------------------------------------------------

def _prox_problem(seed=3, rows=40, k=5):
    M, U, V = _problem(rows, 30, k, seed)
    S = method.Sketch(method.GAUSSIAN, seed, 2, 0, 30, 12)
    _, _, G, R = method.sketched_terms(M, V, S)
    mu = 0.7
    eta = 1.0 / (method.lambda_max(G) + mu)
    return U, G, R, mu, eta


def test_one_inner_step_is_the_paper_step():
    U, G, R, mu, eta = _prox_problem()
    a = method.pgd_inner(U, G, R, eta, mu, 1)
    b = method.pgd_update(U, G, R, eta)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_inner_steps_reach_the_exact_proximal_minimiser():
    """Many steps converge to the minimiser of 1/2 x^T (G + mu I) x - (r + mu u)^T x
    over x >= 0, computed independently by the Lawson-Hanson active-set method."""
    from oracle import mlp as omlp
    U, G, R, mu, eta = _prox_problem()
    x = method.pgd_inner(U, G, R, eta, mu, 20000)
    xs = omlp.prox_exact(G, mu, R + mu * U)
    assert np.max(np.abs(x - xs)) <= 1e-7 * max(1.0, np.max(np.abs(xs)))


def test_inner_steps_descend():
    from oracle import mlp as omlp
    U, G, R, mu, eta = _prox_problem(5)
    b = R + mu * U
    f_prev = omlp.prox_objective(G, mu, b, U)
    for p in range(1, 12):
        f = omlp.prox_objective(G, mu, b, method.pgd_inner(U, G, R, eta, mu, p))
        assert np.all(f <= f_prev + 1e-9 * np.abs(f_prev))
        f_prev = f


def test_mutant_inner_prox_sign_is_caught():
    """b = r - mu u instead of r + mu u: no longer the minimiser of eq. reg_sub."""
    from oracle import mlp as omlp

    def bad_inner(Z, G, R, eta, mu, iters, bound=None):
        b = R - mu * Z
        x = Z
        for _ in range(iters):
            x = method.project(x - eta * (x @ G + mu * x - b), bound)
        return x
    U, G, R, mu, eta = _prox_problem()
    x = bad_inner(U, G, R, eta, mu, 20000)
    xs = omlp.prox_exact(G, mu, R + mu * U)
    assert np.max(np.abs(x - xs)) > 1e-3 * max(1.0, np.max(np.abs(xs)))


def test_row_quantisation_error_bound():
    """One scale per row: every entry within half an E4M3 quantum of its row
    (relative 2^-4 above the subnormal range, scale 2^-9 below)."""
    g = np.random.default_rng(13)
    X = (g.standard_normal((40, 300)) * np.repeat([1.0, 1e3, 1e-3, 0.0], 10)[:, None]).astype(np.float32)
    Xd = method.quantise_rows_e4m3(X)
    for r in range(X.shape[0]):
        row = X[r].astype(np.float64)
        sc = np.abs(row).max() / 448.0 if np.abs(row).max() > 0 else 1.0
        assert np.all(np.abs(Xd[r] - row) <= np.maximum(np.abs(row) * 2.0 ** -4, sc * 2.0 ** -9) * 1.0001)


def test_reassociated_fp8_model_error():
    """The fp8 reassociated model is within E4M3 accuracy of the exact terms:
    relative error of R between the bf16 model's and 0.1, and B, G unchanged
    from the bf16 model."""
    M, U, V = _problem(256, 96, 6, 9)
    S = method.Sketch(method.GAUSSIAN, 2, 1, 0, 96, 32)
    _, Be, _, Re = method.sketched_terms(M, V, S)
    _, Bb, Gb, Rb = method.sketched_terms_reassociated_bf16(M, V, S)
    _, B8, G8, R8 = method.sketched_terms_reassociated_fp8(M, V, S)
    assert np.array_equal(B8, Bb) and np.array_equal(G8, Gb)
    e8 = np.linalg.norm(R8 - Re) / np.linalg.norm(Re)
    eb = np.linalg.norm(Rb - Re) / np.linalg.norm(Re)
    assert eb < e8 < 0.1
