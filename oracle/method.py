"""Sketched ANLS in plain FP64 numpy -- the oracle (test infrastructure only).

Follows the paper's steps in its order and notation:

  Alg. 1 (two-block coordinate descent), with each block solved by one step
  of the sketched subproblem of Section 3.2 (eq. sketched_u, sketched_v):
      A^t = M S^t,  B^t = V^{t T} S^t                       (eq. def_A_B)
      PGD:  U^{t+1} = max{U^t - eta_t (U^t B B^T - A B^T), 0} (eq. gradient_descent,
            with the factor 2 folded into eta_t)
      RCD:  Alg. 3 column sweep with proximal weight mu_t     (eq. entry_sol)
  then the V-half with M^T, S'^t (m x d') and the freshly updated U^{t+1}.

Readings of the paper that the paper leaves open (each one is a stated
choice, the GPU library implements the same choice independently):
  * eta_t = 1 / (lambda_max(G) + mu_t), mu_t = alpha + beta t; lambda_max from
    a fixed number of power iterations in FP64 starting at the all-ones vector.
  * Subsampling columns carry the scale sqrt(n/d) so that E[S S^T] = I
    (Assumption 1); the paper's unscaled e_i give (d/n) I.
  * The V-half uses U^{t+1} (Alg. 1 line 4).
  * Projection max{x, 0} returns +0 for x <= 0.
  * The optional bound of eq. extra_con clamps entries at sqrt(2 ||M||_F).

All arithmetic is FP64.  The sketch values are the binary32 numbers of the
Philox field (``rng.py``), promoted exactly.  Matrix products use numpy's
``@`` (a library matmul) as single steps.
"""
import numpy as np

from . import rng

GAUSSIAN = 0
SUBSAMPLE = 1
IDENTITY = 2
RADEMACHER = 3
COUNT = 4
SRHT = 5
DENSE_KINDS = (GAUSSIAN, RADEMACHER, COUNT, SRHT)

PGD = 0
RCD = 1

SIDE_U = 0
SIDE_V = 1


class Sketch:
    """The random matrix S^t (n x d) of Section 3.4, in one of six kinds.

    kind GAUSSIAN: dense, entries N(0, 1/d) from the Philox field.
    kind RADEMACHER: dense, entries +-1/sqrt(d) with the sign of the entry's
        Philox word (one of Section 3.4's "other choices" of random matrix).
    kind COUNT: count sketch, one entry +-1 per row at a hashed column
        (another of those choices; E[S S^T] = I without scaling).
    kind SRHT: subsampled randomized Hadamard transform sqrt(p/d) D H R
        (the third of those choices), materialised as a dense +-1/sqrt(d) matrix.
    kind SUBSAMPLE: columns sqrt(n/d) e_{J_p}, J drawn without replacement.
    kind IDENTITY: S = I (requires d = n); the unsketched subproblem.
    """

    def __init__(self, kind, seed, t, side, n, d):
        self.kind, self.n, self.d = kind, n, d
        self.J = None
        self.scale = None
        if kind == GAUSSIAN:
            self.scale = rng.gaussian_scale(d)
            self.dense32 = rng.gaussian_field(seed, side, t, n, d, self.scale)
        elif kind == RADEMACHER:
            self.scale = rng.gaussian_scale(d)
            self.dense32 = rng.rademacher_field(seed, side, t, n, d, self.scale)
        elif kind == COUNT:
            self.scale = np.float32(1.0)
            self.dense32 = rng.count_field(seed, side, t, n, d)
        elif kind == SRHT:
            if d > rng.srht_pad(n):
                raise ValueError("SRHT needs d <= the padded order")
            self.scale = rng.gaussian_scale(d)
            self.dense32 = rng.srht_field(seed, side, t, n, d, self.scale)
        elif kind == SUBSAMPLE:
            if d > n:
                raise ValueError("subsampling needs d <= n")
            self.J = rng.subsample_indices(seed, side, t, n, d)
            self.scale = rng.subsample_scale(n, d)
        elif kind == IDENTITY:
            if d != n:
                raise ValueError("identity sketch needs d == n")
        else:
            raise ValueError("unknown sketch kind")

    def dense(self):
        """S as an n x d FP64 array."""
        if self.kind in DENSE_KINDS:
            return self.dense32.astype(np.float64)
        S = np.zeros((self.n, self.d))
        if self.kind == SUBSAMPLE:
            S[self.J, np.arange(self.d)] = np.float64(self.scale)
        else:
            S[np.arange(self.n), np.arange(self.n)] = 1.0
        return S

    def right_multiply(self, X):
        """X S for X with n columns (dense ndarray or scipy sparse)."""
        if self.kind in DENSE_KINDS:
            out = X @ self.dense32.astype(np.float64)
        elif self.kind == SUBSAMPLE:
            out = X[:, self.J] * np.float64(self.scale)
        else:
            out = X.copy() if isinstance(X, np.ndarray) else X
        if hasattr(out, "toarray"):
            out = out.toarray()
        return np.asarray(out, dtype=np.float64)


def mu_t(alpha, beta, t):
    """Proximal weight mu_t = alpha + beta t (Section 5.1 setup; eq. reg_sub)."""
    return float(alpha) + float(beta) * float(t)


def lambda_max(G, iters=32):
    """Largest eigenvalue of the symmetric PSD Gram G by power iteration from
    the all-ones vector, Rayleigh quotient at the end (FP64)."""
    k = G.shape[0]
    x = np.ones(k) / np.sqrt(k)
    for _ in range(iters):
        y = G @ x
        nrm = np.sqrt(y @ y)
        if nrm == 0.0:
            return 0.0
        x = y / nrm
    return float(x @ (G @ x))


def project(X, bound=None):
    """max{X, 0} (+0 for nonpositive entries); optional upper bound of eq. extra_con."""
    Y = np.where(X > 0.0, X, 0.0)
    if bound is not None:
        Y = np.minimum(Y, bound)
    return Y


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as FP64.  Models
    the reduced-precision form's operand rounding (1 sign, 8 exponent, 7
    fraction bits).  Goes through binary32 first, as the GPU operands do."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def sketched_terms_bf16(X, Y, S):
    """The sketched terms of the reduced-precision form: the operands X, Y and
    S rounded to bf16, products accumulated exactly; A = X S and B = Y^T S
    rounded to bf16 again where they enter R = A B^T; G = B B^T from the
    unrounded B.  For S = I: R = X Y from bf16 X and Y, G = Y^T Y from the
    unrounded Y (A is not formed)."""
    if S.kind == IDENTITY:
        Y = np.asarray(Y, dtype=np.float64)
        return None, Y.T.copy(), Y.T @ Y, round_bf16(X) @ round_bf16(Y)
    Sb = round_bf16(S.dense32)
    A = round_bf16(round_bf16(X) @ Sb)
    B = round_bf16(Y).T @ Sb
    G = B @ B.T
    R = A @ round_bf16(B).T
    return A, B, G, R


def round_e4m3(x):
    """Round binary32 values to the nearest fp8 E4M3 value (ties to even,
    saturating at +-448; 3 fraction bits, exponent bias 7, subnormal quantum
    2^-9), returned as FP64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.where(a > 0, a, 1.0))
    e = np.maximum(ex - 1, -6)                     # binade exponent, subnormals share 2^-6
    q = np.ldexp(1.0, e - 3)                       # spacing of E4M3 values in that binade
    r = np.rint(a / q) * q
    r = np.minimum(r, 448.0)
    return np.copysign(r, x)


def quantise_rowblocks_e4m3(X):
    """Per 128-row block: scale = max|x| / 448 (binary32, 1 if zero) and
    Xq = e4m3(x / scale) (binary32 division); returns the dequantised FP64 X."""
    X32 = np.asarray(X, dtype=np.float32)
    out = np.empty(X32.shape, dtype=np.float64)
    for r0 in range(0, X32.shape[0], 128):
        blk = X32[r0:r0 + 128]
        mx = np.float32(np.max(np.abs(blk))) if blk.size else np.float32(0.0)
        sc = np.float32(mx / np.float32(448.0)) if mx > 0 else np.float32(1.0)
        out[r0:r0 + 128] = round_e4m3(blk / sc) * np.float64(sc)
    return out


def sketched_terms_fp8(X, Y, S, seed, t, side):
    """The sketched terms of the fp8 form: X quantised per 128-row block to
    E4M3, the unit-variance draws z of S to E4M3, A = (Xq zq) / sqrt(d)
    rounded to bf16 where it enters R; B = Y^T S from bf16 operands as in the
    bf16 form."""
    if S.kind == COUNT:
        z = rng.count_field(seed, side, t, S.n, S.d)
    elif S.kind == SRHT:
        z = rng.srht_field(seed, side, t, S.n, S.d, np.float32(1.0))
    else:
        unit = rng.rademacher_field if S.kind == RADEMACHER else rng.gaussian_field
        z = unit(seed, side, t, S.n, S.d, np.float32(1.0))
    A = round_bf16((quantise_rowblocks_e4m3(X) @ round_e4m3(z)) * np.float64(S.scale))
    Sb = round_bf16(S.dense32)
    B = round_bf16(Y).T @ Sb
    G = B @ B.T
    R = A @ round_bf16(B).T
    return A, B, G, R


def quantise_rows_e4m3(X):
    """Per row: scale = max|x| / 448 (binary32, 1 if zero) and Xq = e4m3(x / scale)
    (binary32 division); returns the dequantised FP64 X."""
    X32 = np.asarray(X, dtype=np.float32)
    out = np.empty(X32.shape, dtype=np.float64)
    for r in range(X32.shape[0]):
        mx = np.float32(np.max(np.abs(X32[r]))) if X32.shape[1] else np.float32(0.0)
        sc = np.float32(mx / np.float32(448.0)) if mx > 0 else np.float32(1.0)
        out[r] = round_e4m3(X32[r] / sc) * np.float64(sc)
    return out


def sketched_terms_reassociated_fp8(X, Y, S):
    """The reassociated order with an fp8 streaming product: B and P^T = B S^T
    as in the bf16 model but P^T kept in binary32, then quantised per row of
    P^T (one scale per column of P) to E4M3; X quantised per 128-row block to
    E4M3; R = Xq P_q.  G = B B^T from the unrounded B."""
    Sb = round_bf16(S.dense32)
    B = round_bf16(Y).T @ Sb
    G = B @ B.T
    Pt = (round_bf16(B) @ Sb.T).astype(np.float32)
    R = quantise_rowblocks_e4m3(X) @ quantise_rows_e4m3(Pt).T
    return None, B, G, R


def sketched_terms(X, Y, S):
    """A = X S, B = Y^T S, G = B B^T, R = A B^T  (eq. def_A_B; gradient terms of
    eq. gradient_descent).  X: rows x n data (M or M^T), Y: n x k fixed factor."""
    A = S.right_multiply(X)
    if S.kind == SUBSAMPLE:
        B = (Y[S.J, :] * np.float64(S.scale)).T
    elif S.kind == IDENTITY:
        B = Y.T.copy()
    else:
        B = Y.T @ S.dense32.astype(np.float64)
    G = B @ B.T
    R = A @ B.T
    return A, B, G, R


def sketched_terms_reassociated(X, Y, S):
    """B, G and R of sketched_terms with R formed in the other order:
    P = S B^T (n x k) first, then R = X P.  In exact arithmetic R = (X S) B^T
    = X (S B^T) (associativity of the matrix product); the work is
    2 n d k + 2 rows n k instead of 2 rows n d + 2 rows d k.  A = X S is not
    formed (None)."""
    Sd = S.dense()
    B = Y.T @ Sd
    G = B @ B.T
    P = Sd @ B.T
    R = X @ P
    R = np.asarray(R.toarray() if hasattr(R, "toarray") else R, dtype=np.float64)
    return None, B, G, R


def sketched_terms_reassociated_bf16(X, Y, S):
    """The reassociated order with bf16 operands: S, Y rounded to bf16 for
    B = Y^T S (exact accumulation); P = S round(B)^T rounded to bf16 where it
    enters R = round(X) P; G = B B^T from the unrounded B."""
    Sb = round_bf16(S.dense32)
    B = round_bf16(Y).T @ Sb
    G = B @ B.T
    P = round_bf16(Sb @ round_bf16(B).T)
    R = round_bf16(X) @ P
    return None, B, G, R


def pgd_update(Z, G, R, eta, bound=None):
    """One projected-gradient step, eq. gradient_descent:
    Z <- max{Z - eta (Z G - R), 0} (the gradient's factor 2 is inside eta)."""
    return project(Z - eta * (Z @ G - R), bound)


def pgd_inner(Z, G, R, eta, mu, iters, bound=None):
    """``iters`` projected-gradient steps on the proximal row objective of eq.
    reg_sub (halved), f(x) = 1/2 x^T (G + mu I) x - (r + mu u)^T x with u the
    current row of Z, starting at x = u with step eta:
        x <- max{x - eta ((G + mu I) x - (R + mu Z)), 0}.
    At x = u the mu terms cancel, so the first step is eq. gradient_descent
    (pgd_update); more steps approach the exact minimiser of the subproblem."""
    b = R + mu * Z
    x = Z
    for _ in range(iters):
        x = project(x - eta * (x @ G + mu * x - b), bound)
    return x


def rcd_update(Z, G, R, mu, bound=None):
    """Proximal coordinate descent, Alg. 3 / eq. entry_sol: for j = 1..k,
    T = mu Z^t_j + R_j - sum_{l<j} G_lj Z^{t+1}_l - sum_{l>j} G_lj Z^t_l,
    Z^{t+1}_j = max{T / (G_jj + mu), 0}."""
    Zold = Z
    Znew = Z.copy()
    k = Z.shape[1]
    for j in range(k):
        T = mu * Zold[:, j] + R[:, j]
        for l in range(j):
            T = T - G[l, j] * Znew[:, l]
        for l in range(j + 1, k):
            T = T - G[l, j] * Zold[:, l]
        Znew[:, j] = project(T / (G[j, j] + mu), bound)
    return Znew


def half_step(X, Y, Z, S, solver, mu, power_iters=32, bound=None, rows=None, bf16=False, fp8=None,
              reassociate=False, inner_iters=1):
    """Update of the factor Z (rows x k) against data X (rows x n) with the
    other factor Y (n x k) fixed and sketch S (n x d): one solver step on the
    sketched subproblem (eq. sketched_sub), or ``inner_iters`` projected
    gradient steps on its proximal form (PGD).  ``rows`` restricts the result
    to a subset of rows (the subproblem is row-independent, eq. u_block)."""
    if rows is not None:
        X = X[rows]
        Z = Z[rows]
    if reassociate and fp8 is not None:
        A, B, G, R = sketched_terms_reassociated_fp8(X, Y, S)
    elif reassociate:
        A, B, G, R = (sketched_terms_reassociated_bf16 if bf16 else sketched_terms_reassociated)(X, Y, S)
    elif fp8 is not None:  # fp8 = (seed, t, side) of the sketch, to redraw its unit-variance values
        A, B, G, R = sketched_terms_fp8(X, Y, S, *fp8)
    elif bf16:
        A, B, G, R = sketched_terms_bf16(X, Y, S)
    else:
        A, B, G, R = sketched_terms(X, Y, S)
    if solver == PGD:
        eta = 1.0 / (lambda_max(G, power_iters) + mu)
        if inner_iters > 1:
            return pgd_inner(Z, G, R, eta, mu, inner_iters, bound)
        return pgd_update(Z, G, R, eta, bound)
    if solver == RCD:
        return rcd_update(Z, G, R, mu, bound)
    raise ValueError("unknown solver")


class Options:
    def __init__(self, sketch=GAUSSIAN, d=None, d_v=None, solver=PGD, alpha=1.0, beta=1.0,
                 power_iters=32, bound_clamp=False, inner_iters=1):
        self.sketch, self.d, self.d_v = sketch, d, d_v
        self.solver, self.alpha, self.beta = solver, alpha, beta
        self.inner_iters = inner_iters
        self.power_iters, self.bound_clamp = power_iters, bound_clamp


def frob(M):
    if hasattr(M, "multiply"):
        return float(np.sqrt(M.multiply(M).sum()))
    return float(np.linalg.norm(M))


def outer_iteration(M, MT, U, V, seed, t, opt, bound=None):
    """One iteration t of Alg. 1 with sketched subproblems: U-half with S^t
    (n x d, side 0), then V-half with S'^t (m x d', side 1) and U^{t+1}."""
    m, n = M.shape
    d = opt.d
    d_v = opt.d_v if opt.d_v is not None else d
    mu = mu_t(opt.alpha, opt.beta, t)
    S = Sketch(opt.sketch, seed, t, SIDE_U, n, d)
    U = half_step(M, V, U, S, opt.solver, mu, opt.power_iters, bound, inner_iters=opt.inner_iters)
    Sp = Sketch(opt.sketch, seed, t, SIDE_V, m, d_v)
    V = half_step(MT, U, V, Sp, opt.solver, mu, opt.power_iters, bound, inner_iters=opt.inner_iters)
    return U, V


def rel_error(M, U, V):
    """||M - U V^T||_F / ||M||_F (Section 5.1), FP64."""
    if hasattr(M, "tocsr"):
        return rel_error_sparse(M, U, V)
    return float(np.linalg.norm(M - U @ V.T) / np.linalg.norm(M))


def rel_error_sparse(M, U, V):
    """Same quantity for sparse M through the expansion
    ||M||^2 - 2 sum_{ij in nnz} M_ij <U_i, V_j> + <U^T U, V^T V>."""
    M = M.tocoo()
    mm = float(np.dot(M.data, M.data))
    cross = float(np.sum(M.data * np.einsum("ij,ij->i", U[M.row], V[M.col])))
    gram = float(np.sum((U.T @ U) * (V.T @ V)))
    return float(np.sqrt(max(mm - 2.0 * cross + gram, 0.0)) / np.sqrt(mm))


def run(M, U0, V0, seed, T, opt, t0=0, log_error=True):
    """T outer iterations from (U0, V0), returns (U, V, errors)."""
    M64 = M.astype(np.float64) if isinstance(M, np.ndarray) else M.astype(np.float64).tocsr()
    MT = M64.T.copy() if isinstance(M64, np.ndarray) else M64.T.tocsr()
    U = np.asarray(U0, dtype=np.float64).copy()
    V = np.asarray(V0, dtype=np.float64).copy()
    bound = np.sqrt(2.0 * frob(M64)) if opt.bound_clamp else None
    errs = []
    for t in range(t0, t0 + T):
        U, V = outer_iteration(M64, MT, U, V, seed, t, opt, bound)
        if log_error:
            errs.append(rel_error(M64, U, V))
    return U, V, errs


def default_init(seed, m, n, k):
    """U^0, V^0 ~ Uniform[0,1) from Philox streams 2 and 3 (Alg. 2 line 1)."""
    U0 = rng.uniform_field(seed, rng.STREAM_INIT_U, 0, m, k)
    V0 = rng.uniform_field(seed, rng.STREAM_INIT_V, 0, n, k)
    return U0, V0


# ---------------------------------------------------------------------------
# Unsketched relatives used as pins (Section 2.1, Alg. 1 with exact or HALS
# subproblem solvers).
# ---------------------------------------------------------------------------

def hals_update(Z, X, Y):
    """Textbook HALS column update for min_Z ||X - Z Y^T||, Z >= 0
    (Cichocki et al.; Gillis 2014): Z_j <- max{Z_j + ((X Y)_j - Z (Y^T Y)_j)/(Y^T Y)_jj, 0},
    columns in order, each using the already updated earlier columns."""
    Z = Z.copy()
    XY = X @ Y
    YY = Y.T @ Y
    for j in range(Z.shape[1]):
        Z[:, j] = project(Z[:, j] + (XY[:, j] - Z @ YY[:, j]) / YY[j, j])
    return Z


def plain_pg_update(Z, X, Y, eta):
    """Unsketched projected gradient step on min_Z ||X - Z Y^T||^2 / 2:
    Z <- max{Z - eta (Z Y^T Y - X Y), 0}."""
    return project(Z - eta * (Z @ (Y.T @ Y) - X @ Y))
