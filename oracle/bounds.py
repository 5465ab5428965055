"""Acceptance bounds of the reduced-precision forms against the exact FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The exact oracle (``method.py``) is the reference of every form of the
library.  A form that rounds its operands to bf16 or fp8 E4M3 cannot match it
to 1e-5; it is accepted when its half-step lies within a bound derived here
from the unit roundoff of the formats it uses and the data of the step, with
no knowledge of any kernel beyond which operands the form is defined to round
(the rounding points of each form are fixed once, in the library's header and
design notes).

Rounding model (the standard model of floating-point arithmetic with the
probabilistic reading of Higham and Mary, SIAM J. Sci. Comput. 41(5), 2019):
rounding a real v to a format returns v (1 + delta) + eps with |delta| <= u
(unit roundoff: bf16 2^-8, E4M3 2^-4, binary32 2^-24) and |eps| <= a (half
the subnormal spacing of the format times the scale in use: E4M3 2^-10; zero
for bf16 at the magnitudes here), and different roundings are independent
with mean zero.  For C = fl(X) fl(Y) accumulated in binary32 this gives

  E ||C - X Y||_F^2 <= sum_l [ ex_l r_l + c_l ey_l + ex_l ey_l ]
                       + K v^2 || |X| |Y| ||_F^2,
  ex_l = u_X^2 c_l + n a_X^2,   ey_l = u_Y^2 r_l + p a_Y^2,

with c_l = ||X[:, l]||^2, r_l = ||Y[l, :]||^2, n rows of X, p columns of Y,
K the inner dimension and v = 2^-24 (each partial sum bounded by |X| |Y|).
The same entrywise form carries the error of a computed product into the
next product (E ||dA B^T||_F^2 = sum_j (sum_i Var dA_ij) ||B[:, j]||^2 for
independent entries), the rms of a sum of error terms is bounded by the sum
of their rms (Minkowski), and an error is bounded by 3 times its rms (the
Frobenius norm of a sum of thousands of independent terms concentrates near
its rms).  With e_G >= ||dG||_F >= ||dG||_2 and e_R >= ||dR||_F:

  |eta' - eta| <= eta eta' |d lambda|, d lambda = 2 v^T dB B^T v + O(dB^2)
                                           (v the top eigenvector of G),
  PGD (eq. gradient_descent, projection 1-Lipschitz):
  ||Z'_form - Z'_exact||_F <= eta' (eta' |d lambda| ||Z G - R||_F + ||Z dG||_F
                                    + e_R) + 4 v (||Z|| + eta' (||Z G|| + ||R||)),
  eta' = 1 / (lambda_max(G) - |d lambda| + mu) >= both step sizes,
  (entries of dB in one column share the rounding of S: sums over them are
  bounded for any correlation, Var sum a_c e_c <= (sum |a_c| sigma_c)^2),

and for P inner steps on the proximal objective (each step map is
nonexpansive for eta <= 1 / (lambda_max + mu)) the per-step terms add up.
For the coordinate-descent sweep (Alg. 3) no usable worst-case bound exists
(the sweep's perturbation bound grows like (1 + G_lj / G_jj)^k); there the
bound is 3 times the rms deviation of the exact sweep over 8 draws of the
rounding model itself (every rounding point of the form perturbed by
+-u relative and +-a absolute with random signs, the terms recomputed in
FP64).
"""
import numpy as np

from . import method

U_BF16 = 2.0 ** -8
U_E4M3 = 2.0 ** -4
A_E4M3 = 2.0 ** -10
V_F32 = 2.0 ** -24

FORMS = ("bf16", "fp8", "bf16_reassociated", "fp8_reassociated", "bf16_identity")


def _fro(A):
    return float(np.linalg.norm(A))


def spectral_norm(A):
    """||A||_2 from the eigenvalues of the smaller Gram matrix (exact up to
    FP64 rounding), or the Frobenius norm (an upper bound) when both sides
    exceed 2048."""
    A = np.asarray(A, dtype=np.float64)
    if A.size == 0:
        return 0.0
    if min(A.shape) > 2048:
        return _fro(A)
    Gm = A.T @ A if A.shape[1] <= A.shape[0] else A @ A.T
    return float(np.sqrt(max(np.linalg.eigvalsh(Gm)[-1], 0.0))) * (1.0 + 1e-9)


def product_rms(X, Y, ux=0.0, uy=0.0, ax=0.0, ay=0.0):
    """Root mean square of ||fl(X) fl(Y) - X Y||_F under the model above:
    X (n x K) rounded with (ux, ax), Y (K x p) with (uy, ay), products summed
    in binary32."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n, K = X.shape
    p = Y.shape[1]
    c = np.einsum("il,il->l", X, X)
    r = np.einsum("lj,lj->l", Y, Y)
    ex = ux * ux * c + n * ax * ax
    ey = uy * uy * r + p * ay * ay
    var = float(np.sum(ex * r + c * ey + ex * ey))
    acc = K * V_F32 * V_F32 * float(np.sum((np.abs(X) @ np.abs(Y)) ** 2))
    return float(np.sqrt(var + acc))


class Terms:
    """Exact sketched terms with the error bounds of a reduced-precision form:
    eR >= ||dR||_F, and what the step bound needs to carry dG (the operands
    of B = Y^T S and their entry variances)."""

    def __init__(self, B, G, R, eR, Y=None, Sd=None, vY=None, vS=None):
        self.B, self.G, self.R, self.eR = B, G, R, eR
        self.Y, self.Sd, self.vY, self.vS = Y, Sd, vY, vS


def _var(W, u, a=0.0):
    """Entrywise variance bound of rounding W with unit u and floor a."""
    return u * u * W * W + a * a


def _acc_var(X, Y):
    """Entrywise variance bound of the binary32 accumulation of X Y (every
    partial sum bounded by |X| |Y|, one rounding per product)."""
    return X.shape[1] * V_F32 * V_F32 * (np.abs(X) @ np.abs(Y)) ** 2


def _sum_sd(*variances):
    """sqrt(E ||sum_t E_t||_F^2) <= sqrt(sum_ic (sum_t sigma_t,ic)^2) for error
    terms of entry variances V_t (any correlation between the terms)."""
    tot = sum(np.sqrt(np.maximum(V, 0.0)) for V in variances)
    return float(np.sqrt(np.sum(tot * tot)))


def terms_bound(X, Y, S, form):
    """Exact B, G, R of the sketched subproblem (``method.sketched_terms``) and
    the bound e_R of the given reduced-precision form (3 times the rms of
    ||dR||_F under the model).

    Each error term is linear in the independent rounding errors, so its
    entry variances follow exactly from the operands; e.g. for dA B^T with
    A = X S rounded at X and S,
      Var (dA B^T)_ic <= sum_l vX_il (S B^T)_lc^2 + sum_l X_il^2 sum_j vS_lj B_cj^2.
    Terms sharing a rounding (X dS B^T and A dB^T share that of S) are
    combined entrywise by Minkowski's inequality.

    Rounding points of each form (fixed by the form's definition):
      bf16              X, S, Y rounded to bf16; B = Y^T S and A = X S summed in
                        binary32; A and B rounded to bf16 for R = A B^T;
                        G = B B^T from the unrounded B.
      fp8               X in E4M3 with block scales s = max|x| / 448 (absolute
                        floor 2^-10 s), the unit draws z of S in E4M3 (S = z /
                        sqrt(d)); A rounded to bf16 for R; B and G as in bf16.
      bf16_reassociated B, G as in bf16; P = S B^T from bf16 S and B, rounded
                        to bf16; R = X P from bf16 X.
      fp8_reassociated  B, G as in bf16; P = S B^T from bf16 S and B in binary32,
                        then in E4M3 with one scale per column of P; R = X P with
                        X in E4M3 (block scales).
      bf16_identity     S = I: R = X Y from bf16 X and Y; G = Y^T Y unrounded.
    """
    if form not in FORMS:
        raise ValueError("unknown form")
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    vY = _var(Y, U_BF16)
    if form == "bf16_identity":
        G = Y.T @ Y
        R = X @ Y
        vX = _var(X, U_BF16)
        VR = vX @ (Y * Y) + (X * X) @ vY + vX @ vY + _acc_var(X, Y)
        return Terms(Y.T.copy(), G, R, 3.0 * float(np.sqrt(VR.sum())))
    Sd = S.dense()
    fp8 = form.startswith("fp8")
    ax = A_E4M3 * float(np.max(np.abs(X))) / 448.0 if X.size else 0.0
    vX = _var(X, U_E4M3, ax) if fp8 else _var(X, U_BF16)
    vSb = _var(Sd, U_BF16)
    B = Y.T @ Sd
    G = B @ B.T
    P = Sd @ B.T
    A = X @ Sd
    X2, A2, B2, Y2 = X * X, A * A, B * B, Y * Y
    # A dB'^T: the roundings of Y and S inside B, and of B itself (bf16)
    AS = A @ Sd.T
    V_AdB = (AS * AS) @ vY + ((A2 @ vSb.T) @ Y2) + U_BF16 * U_BF16 * (A2 @ B2.T) + A2 @ _acc_var(Y.T, Sd).T
    if form in ("bf16", "fp8"):
        R = A @ B.T
        vS = _var(Sd, U_E4M3, A_E4M3 * float(S.scale)) if fp8 else vSb
        # dA B^T: the roundings of X and S inside A, and of A itself (bf16)
        V_dAB = vX @ (P * P) + X2 @ (vS @ B2.T) + U_BF16 * U_BF16 * (A2 @ B2.T) + _acc_var(X, Sd) @ B2.T
        second = float(np.sqrt(np.dot((vX @ (Sd * Sd) + X2 @ vS).sum(axis=0), (vY.T @ (Sd * Sd)).sum(axis=0))))
        eR = 3.0 * (_sum_sd(V_dAB, V_AdB, _acc_var(A, B.T)) + second)
        return Terms(B, G, R, eR, Y, Sd, vY, vSb)
    R = X @ P
    accP = _acc_var(Sd, B.T)
    if form == "bf16_reassociated":
        vP = _var(P, U_BF16) + accP
    else:
        sc = np.max(np.abs(P), axis=0) / 448.0
        vP = U_E4M3 * U_E4M3 * P * P + (A_E4M3 * sc[None, :]) ** 2 + accP
    V_dXP = vX @ (P * P)
    V_XdSB = X2 @ (vSb @ B2.T)
    V_XdP = X2 @ vP
    second = float(np.sqrt(np.dot(vX.sum(axis=0), vP.sum(axis=1) + vSb @ B2.sum(axis=0))))
    eR = 3.0 * (_sum_sd(V_dXP, V_XdSB, V_AdB, V_XdP, _acc_var(X, P)) + second)
    return Terms(B, G, R, eR, Y, Sd, vY, vSb)


def _zdg_sd(x, T):
    """rms of ||x dG||_F, dG = dB B^T + B dB^T for dB = (Y^T S)_computed - Y^T S
    (roundings of Y and S, entry variances vY, vS; B rounded nowhere: G is
    taken from the binary32 B), with the correlation of dB's entries through
    the shared roundings carried exactly; plus the second order ||dB||^2."""
    if T.Sd is None:
        return 0.0
    Y, Sd, B, vY, vS = T.Y, T.Sd, T.B, T.vY, T.vS
    P = Sd @ B.T
    B2 = B * B
    ZY = x @ Y.T
    V1 = ((x * x) @ vY.T) @ (P * P) + (ZY * ZY) @ (vS @ B2.T)          # x dB B^T
    W = x @ B
    WS = W @ Sd.T
    V2 = (WS * WS) @ vY + ((W * W) @ vS.T) @ (Y * Y)                     # x B dB^T
    VB = vY.T @ (Sd * Sd) + (Y * Y).T @ vS
    return _sum_sd(V1, V2) + _fro(x) * float(VB.sum())


def _dlam_sd(T):
    """rms of the change of lambda_max(G) to first order, 2 v^T dB B^T v for
    the top eigenvector v (correlations through the shared roundings exact),
    plus the second order ||dB||_F^2."""
    if T.Sd is None:
        return 0.0
    Y, Sd, B, vY, vS = T.Y, T.Sd, T.B, T.vY, T.vS
    v = np.linalg.eigh(T.G)[1][:, -1]
    w = B.T @ v
    Sw = Sd @ w
    Yv = Y @ v
    var = float(np.sum(Sw * Sw * (vY @ (v * v))) + np.sum(Yv * Yv * (vS @ (w * w))))
    VB = vY.T @ (Sd * Sd) + (Y * Y).T @ vS
    return 2.0 * float(np.sqrt(var)) + float(VB.sum())


def _pgd_step_term(x, Gm, b, eta_hi, dlam, T):
    """One projected-gradient step's deviation bound at the point x for the
    objective with Hessian Gm and linear term b (eq. gradient_descent, or its
    proximal form with Gm = G + mu I and b = R + mu Z): the step-size change
    (3 rms), x dG (3 rms) and dR (e_R), plus binary32 arithmetic."""
    g = x @ Gm - b
    rnd = 4.0 * V_F32 * (_fro(x) + eta_hi * (_fro(x @ Gm) + _fro(b)))
    return eta_hi * (eta_hi * 3.0 * dlam * _fro(g) + 3.0 * _zdg_sd(x, T) + T.eR) + rnd


MC_DRAWS = 8


def _pert(W, u, g, a=0.0):
    """W (1 + delta) + eps with delta = +-u and eps = +-a, random signs: a draw
    of the rounding model at its largest magnitudes."""
    out = W * (1.0 + u * g.choice((-1.0, 1.0), size=W.shape))
    if a:
        out = out + a * g.choice((-1.0, 1.0), size=W.shape)
    return out


def perturbed_terms(X, Y, S, form, g):
    """G and R of the given form computed in FP64 from operands perturbed by
    one draw of the rounding model at the form's rounding points (the same
    points as terms_bound)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Yb = _pert(Y, U_BF16, g)
    if form == "bf16_identity":
        return Y.T @ Y, _pert(X, U_BF16, g) @ Yb
    Sd = S.dense()
    fp8 = form.startswith("fp8")
    ax = A_E4M3 * float(np.max(np.abs(X))) / 448.0 if X.size else 0.0
    Xq = _pert(X, U_E4M3, g, ax) if fp8 else _pert(X, U_BF16, g)
    Sb = _pert(Sd, U_BF16, g)
    Bc = Yb.T @ Sb
    Gp = Bc @ Bc.T
    Br = _pert(Bc, U_BF16, g)
    if form in ("bf16", "fp8"):
        Sq = _pert(Sd, U_E4M3, g, A_E4M3 * float(S.scale)) if fp8 else Sb
        return Gp, _pert(Xq @ Sq, U_BF16, g) @ Br.T
    P = Sb @ Br.T
    if form == "bf16_reassociated":
        P = _pert(P, U_BF16, g)
    else:
        sc = np.max(np.abs(P), axis=0) / 448.0
        P = P * (1.0 + U_E4M3 * g.choice((-1.0, 1.0), size=P.shape)) + A_E4M3 * sc[None, :] * g.choice(
            (-1.0, 1.0), size=P.shape)
    return Gp, Xq @ P


def half_step_bound(X, Y, Z, S, solver, mu, form, inner_iters=1, power_iters=32, seed=0):
    """(Z' exact, bound on ||Z'_form - Z'_exact||_F) for one half-step of the
    given solver and reduced-precision form (eq. gradient_descent / Alg. 3)."""
    Z = np.asarray(Z, dtype=np.float64)
    T = terms_bound(X, Y, S, form)
    G, R = T.G, T.R
    if solver == method.PGD:
        lam = method.lambda_max(G, power_iters)
        eta = 1.0 / (lam + mu)
        dlam = _dlam_sd(T)
        eta_hi = 1.0 / (max(lam - 3.0 * dlam, 0.0) + mu)
        if inner_iters <= 1:
            exact = method.pgd_update(Z, G, R, eta)
            return exact, _pgd_step_term(Z, G, R, eta_hi, dlam, T)
        Gm = G + mu * np.eye(G.shape[0])
        b = R + mu * Z
        x = Z
        total = 0.0
        for _ in range(inner_iters):
            total += _pgd_step_term(x, Gm, b, eta_hi, dlam, T)
            x = method.project(x - eta * (x @ Gm - b))
        return x, total
    if solver == method.RCD:
        exact = method.rcd_update(Z, G, R, mu)
        g = np.random.default_rng(seed)
        sq = 0.0
        for _ in range(MC_DRAWS):
            Gp, Rp = perturbed_terms(X, Y, S, form, g)
            sq += _fro(method.rcd_update(Z, Gp, Rp, mu) - exact) ** 2
        rnd = 4.0 * V_F32 * (_fro(Z) + _fro(exact))
        return exact, 3.0 * float(np.sqrt(sq / MC_DRAWS)) + rnd
    raise ValueError("unknown solver")


def check(got, X, Y, Z, S, solver, mu, form, inner_iters=1):
    """(relative deviation of got from the exact half-step, relative bound)."""
    exact, bnd = half_step_bound(X, Y, Z, S, solver, mu, form, inner_iters)
    den = max(_fro(exact), 1e-300)
    return _fro(np.asarray(got, dtype=np.float64) - exact) / den, bnd / den
