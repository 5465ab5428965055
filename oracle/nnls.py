"""Exact nonnegative least squares for the oracle (test infrastructure only).

The NNLS subproblems of Section 2.1 (eq. subproblem) split by rows
(eq. u_block): each row solves  min_{x >= 0} 1/2 x^T G x - b^T x  with
G = Y^T Y (k x k, PSD) and b = Y^T m_i.  Two independent exact solvers:

  * brute force over all 2^k supports (k <= ~12): for each support P solve
    the equality-constrained system G_PP x_P = b_P and keep the feasible point
    with the smallest objective;
  * the active-set method of Lawson and Hanson (1974, ch. 23), written from
    the book's description.

plus a KKT checker: x >= 0, g = G x - b >= -tol, |x_i g_i| <= tol.
"""
import itertools

import numpy as np


def objective(G, b, x):
    return 0.5 * float(x @ G @ x) - float(b @ x)


def brute_force(G, b):
    """Exact minimiser over all supports (small k)."""
    k = G.shape[0]
    best_x = np.zeros(k)
    best_f = 0.0
    for r in range(1, k + 1):
        for P in itertools.combinations(range(k), r):
            P = list(P)
            try:
                xp = np.linalg.solve(G[np.ix_(P, P)], b[P])
            except np.linalg.LinAlgError:
                continue
            if np.any(xp < 0):
                continue
            x = np.zeros(k)
            x[P] = xp
            f = objective(G, b, x)
            if f < best_f - 1e-15 * max(1.0, abs(best_f)):
                best_f, best_x = f, x
    return best_x


def active_set(G, b, tol=1e-12, max_iter=None):
    """Lawson-Hanson active set for min 1/2 x^T G x - b^T x, x >= 0."""
    k = G.shape[0]
    max_iter = max_iter or 10 * k + 50
    x = np.zeros(k)
    passive = np.zeros(k, dtype=bool)
    w = b - G @ x
    it = 0
    while (~passive).any() and np.max(np.where(~passive, w, -np.inf)) > tol and it < max_iter:
        it += 1
        j = int(np.argmax(np.where(~passive, w, -np.inf)))
        passive[j] = True
        while True:
            P = np.flatnonzero(passive)
            z = np.zeros(k)
            z[P] = np.linalg.solve(G[np.ix_(P, P)], b[P])
            if np.all(z[P] > 0):
                x = z
                break
            neg = P[z[P] <= 0]
            alpha = np.min(x[neg] / (x[neg] - z[neg]))
            x = x + alpha * (z - x)
            passive &= ~(x <= tol)
            x[~passive] = 0.0
        w = b - G @ x
    return x


def kkt_ok(G, b, x, tol=1e-8):
    """x >= 0, gradient g = Gx - b >= -tol, complementarity |x_i g_i| <= tol."""
    g = G @ x - b
    scale = max(1.0, float(np.max(np.abs(b))))
    return bool(np.all(x >= 0) and np.all(g >= -tol * scale)
                and np.all(np.abs(x * g) <= tol * scale * max(1.0, float(np.max(np.abs(x))))))


def nnls_rows(X, Y, solver=active_set):
    """Exact NNLS solution of min_{Z>=0} ||X - Z Y^T||_F, row by row."""
    G = Y.T @ Y
    Bm = X @ Y
    return np.stack([solver(G, Bm[i]) for i in range(X.shape[0])])


def anls(M, U0, V0, T, solver=active_set):
    """Exact ANLS (Alg. 1 with exact NNLS per block)."""
    U, V = U0.copy(), V0.copy()
    for _ in range(T):
        U = nnls_rows(M, V, solver)
        V = nnls_rows(M.T, U, solver)
    return U, V
