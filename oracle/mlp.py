"""Learned warm start for the proximal row subproblem -- FP64 oracle
(test infrastructure only).

The row subproblem of the proximal coordinate-descent form (eq. reg_sub,
halved):   f(x) = 1/2 x^T (G + mu I) x - (r + mu u)^T x,   x >= 0,
with G = B B^T, r = the row of R = A B^T, u = the row of U^t, mu = mu_t.

Learned form of one half-step (the same choices the GPU library makes):
  * inputs normalised: s = tr(G + mu I) / k, Gn = (G + mu I) / s,
    beta = ||r + mu u|| / sqrt(k) (1 if zero), bn = (r + mu u) / beta;
    then the solution of the normalised problem is y = x s / beta;
  * MLP y0 = ReLU(W3 h2 + b3), h2 = GELU(W2 h1 + b2),
    h1 = GELU(W1g vec(Gn) + W1b bn + b1)  (W1g vec(Gn) is shared by all rows);
  * x0 = y0 beta / s, then P projected-gradient steps on f with step
    eta = 1/(lambda_max(G) + mu): x <- max(0, x - eta ((G + mu I) x - (r + mu u)));
  * fallback: the plain path's update x_pgd -- the projected-gradient step
    max(0, u - eta (u G - r)), or the same number of steps on f from u as the
    plain path takes -- is kept whenever f(x_pgd) < f(x_mlp).
Training: squared error against the normalised exact minimiser y* (one-sided
below zero, see loss_and_grads), Adam.  GELU is the exact x Phi(x).
"""
import math

import numpy as np

from . import nnls as _nnls


def param_shapes(k, hidden):
    return [("W1g", (hidden, k * k)), ("W1b", (hidden, k)), ("b1", (hidden,)), ("W2", (hidden, hidden)),
            ("b2", (hidden,)), ("W3", (k, hidden)), ("b3", (k,))]


def unflatten(theta, k, hidden):
    out, off = {}, 0
    for name, shape in param_shapes(k, hidden):
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def flatten(params, k, hidden):
    return np.concatenate([params[name].ravel() for name, _ in param_shapes(k, hidden)])


def gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def normalise(G, mu, b):
    """(Gn, bn, s, beta) for one subproblem; b = r + mu u (rows x k)."""
    k = G.shape[0]
    Gm = G + mu * np.eye(k)
    s = np.trace(Gm) / k
    beta = np.linalg.norm(b, axis=1) / math.sqrt(k)
    beta = np.where(beta > 0.0, beta, 1.0)
    return Gm / s, b / beta[:, None], s, beta


def forward(P, Gn, bn):
    """Rows of bn (N x k) with one shared Gn; returns y (N x k) and the cache."""
    zg = P["W1g"] @ Gn.ravel() + P["b1"]
    z1 = bn @ P["W1b"].T + zg[None, :]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    o = h2 @ P["W3"].T + P["b3"]
    y = np.maximum(o, 0.0)
    return y, (Gn, bn, z1, h1, z2, h2, o)


def loss_and_grads(P, groups):
    """groups: list of (Gn, bn, ystar).  Loss = 1/2 mean over all rows of
    sum_j e_j^2 with e_j = o_j - y*_j where y*_j > 0 and e_j = max(o_j, 0)
    where y*_j = 0 (o the output before the ReLU).  This equals the squared
    error of the ReLU output y = max(o, 0) except where o_j < 0 < y*_j, where
    it keeps a gradient pulling o_j up: an output unit negative on every row
    can then not stay dead."""
    N = sum(g[1].shape[0] for g in groups)
    grads = {name: np.zeros_like(v) for name, v in P.items()}
    loss = 0.0
    for Gn, bn, ys in groups:
        y, (Gn, bn, z1, h1, z2, h2, o) = forward(P, Gn, bn)
        e = np.where(ys > 0.0, o - ys, np.maximum(o, 0.0))
        loss += 0.5 * float(np.sum(e * e))
        do = e / N
        grads["W3"] += do.T @ h2
        grads["b3"] += do.sum(axis=0)
        dz2 = (do @ P["W3"]) * gelu_grad(z2)
        grads["W2"] += dz2.T @ h1
        grads["b2"] += dz2.sum(axis=0)
        dz1 = (dz2 @ P["W2"]) * gelu_grad(z1)
        grads["W1b"] += dz1.T @ bn
        g1 = dz1.sum(axis=0)
        grads["b1"] += g1
        grads["W1g"] += np.outer(g1, Gn.ravel())
    return loss / N, grads


def adam(P, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) on every parameter; state holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for name in P:
        m = state.setdefault("m_" + name, np.zeros_like(P[name]))
        v = state.setdefault("v_" + name, np.zeros_like(P[name]))
        g = grads[name]
        m[:] = b1 * m + (1 - b1) * g
        v[:] = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[name] = P[name] - lr * mh / (np.sqrt(vh) + eps)
    return P


def prox_objective(G, mu, b, x):
    """f(x) = 1/2 x^T (G + mu I) x - b^T x per row (b = r + mu u)."""
    Gm = G + mu * np.eye(G.shape[0])
    return 0.5 * np.einsum("ij,jk,ik->i", x, Gm, x) - np.einsum("ij,ij->i", b, x)


def prox_exact(G, mu, b):
    """Exact minimiser of f per row (Lawson-Hanson active set)."""
    Gm = G + mu * np.eye(G.shape[0])
    return np.stack([_nnls.active_set(Gm, bi) for bi in b])


def learned_candidates(P, G, mu, R, Z, eta, pg_iters, plain_iters=1):
    """Both candidates of the learned form and their proximal objectives:
    (x_mlp, x_pgd, f_mlp, f_pgd).  x_pgd is the plain path's update: one
    projected gradient step from u (eq. gradient_descent), or ``plain_iters``
    steps on the proximal objective."""
    b = R + mu * Z
    Gn, bn, s, beta = normalise(G, mu, b)
    y0, _ = forward(P, Gn, bn)
    x = y0 * (beta / s)[:, None]
    Gm = G + mu * np.eye(G.shape[0])
    for _ in range(pg_iters):
        x = np.where(x - eta * (x @ Gm - b) > 0.0, x - eta * (x @ Gm - b), 0.0)
    if plain_iters > 1:
        x_pgd = Z
        for _ in range(plain_iters):
            x_pgd = np.where(x_pgd - eta * (x_pgd @ Gm - b) > 0.0, x_pgd - eta * (x_pgd @ Gm - b), 0.0)
    else:
        x_pgd = np.where(Z - eta * (Z @ G - R) > 0.0, Z - eta * (Z @ G - R), 0.0)
    return x, x_pgd, prox_objective(G, mu, b, x), prox_objective(G, mu, b, x_pgd)


def learned_update(P, G, mu, R, Z, eta, pg_iters, plain_iters=1):
    """The learned form of one half-step for rows R (N x k), current rows Z."""
    x, x_pgd, f_mlp, f_pgd = learned_candidates(P, G, mu, R, Z, eta, pg_iters, plain_iters)
    keep = f_mlp <= f_pgd
    return np.where(keep[:, None], x, x_pgd), keep
