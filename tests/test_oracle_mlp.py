"""Pins of the oracle's learned warm start (CPU only): backpropagation against
central finite differences, GELU against its erf definition via scipy, the
exact proximal row solution against brute force and its KKT conditions, the
scale invariance the normalisation relies on, and the fallback guarantee
(never a worse proximal objective than the plain step)."""
import math

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import mlp, nnls


def _params(k, h, seed):
    g = np.random.default_rng(seed)
    theta = np.concatenate([g.standard_normal(int(np.prod(s))) / math.sqrt(s[-1])
                            for _, s in mlp.param_shapes(k, h)])
    return mlp.unflatten(theta, k, h)


def _groups(k, seed, n_groups=2, rows=5):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n_groups):
        B = g.standard_normal((k, 3 * k))
        G = B @ B.T
        b = g.standard_normal((rows, k)) + 1.0
        Gn, bn, _, _ = mlp.normalise(G, 0.3, b)
        ys = np.abs(g.standard_normal((rows, k)))
        ys[g.random((rows, k)) < 0.4] = 0.0  # NNLS minimisers have zero entries
        out.append((Gn, bn, ys))
    return out


def test_gelu_is_x_times_normal_cdf():
    x = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(x), x * ndtr(x), rtol=0, atol=1e-14)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def test_backprop_matches_finite_differences():
    k, h = 3, 7
    P = _params(k, h, 0)
    groups = _groups(k, 1)
    _, grads = mlp.loss_and_grads(P, groups)
    eps = 1e-6
    for name in P:
        flat = P[name].ravel()
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = mlp.loss_and_grads(P, groups)
            flat[idx] = old - eps
            lm, _ = mlp.loss_and_grads(P, groups)
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            assert abs(num - grads[name].ravel()[idx]) <= 1e-6 * max(1.0, abs(num)), name


def test_adam_reduces_the_loss():
    k, h = 4, 16
    P = _params(k, h, 3)
    groups = _groups(k, 4, n_groups=3, rows=20)
    state = {}
    l0, _ = mlp.loss_and_grads(P, groups)
    for _ in range(200):
        _, g = mlp.loss_and_grads(P, groups)
        P = mlp.adam(P, g, state, 1e-2)
    l1, _ = mlp.loss_and_grads(P, groups)
    assert l1 < 0.2 * l0


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_prox_exact_against_brute_force(k):
    g = np.random.default_rng(k)
    for _ in range(20):
        B = g.standard_normal((k, 2 * k + 1))
        G = B @ B.T
        mu = float(g.uniform(0.01, 2.0))
        b = g.standard_normal((3, k))
        x = mlp.prox_exact(G, mu, b)
        Gm = G + mu * np.eye(k)
        for i in range(3):
            assert np.allclose(x[i], nnls.brute_force(Gm, b[i]), atol=1e-9)
            assert nnls.kkt_ok(Gm, b[i], x[i])


def test_normalised_problem_is_scale_invariant():
    """y* of (Gn, bn) times beta / s is x* of the original problem."""
    g = np.random.default_rng(5)
    k = 6
    B = g.standard_normal((k, 20))
    G = 37.0 * (B @ B.T)
    mu = 2.5
    b = g.standard_normal((4, k)) * 11.0 + 3.0
    Gn, bn, s, beta = mlp.normalise(G, mu, b)
    ystar = np.stack([nnls.active_set(Gn, bi) for bi in bn])
    assert np.allclose(ystar * (beta / s)[:, None], mlp.prox_exact(G, mu, b), rtol=1e-8, atol=1e-10)


def test_learned_update_never_worse_than_plain_step():
    g = np.random.default_rng(7)
    k, h = 8, 32
    P = _params(k, h, 8)
    B = g.random((k, 40))
    G = B @ B.T
    mu = 0.5
    lam = np.linalg.eigvalsh(G)[-1]
    eta = 1.0 / (lam + mu)
    Z = g.random((50, k))
    R = g.random((50, k)) * 5
    x, keep = mlp.learned_update(P, G, mu, R, Z, eta, 3)
    b = R + mu * Z
    x_pgd = np.maximum(Z - eta * (Z @ G - R), 0.0)
    assert np.all(mlp.prox_objective(G, mu, b, x) <= mlp.prox_objective(G, mu, b, x_pgd) + 1e-12)
    assert x.min() >= 0


def test_perfect_warm_start_is_a_fixed_point():
    """If the network returned y*, the corrected solution is the exact minimiser."""
    g = np.random.default_rng(9)
    k = 5
    B = g.random((k, 30))
    G = B @ B.T
    mu = 0.2
    Z = g.random((6, k))
    R = g.random((6, k)) * 4
    b = R + mu * Z
    xs = mlp.prox_exact(G, mu, b)
    eta = 1.0 / (np.linalg.eigvalsh(G)[-1] + mu)
    Gm = G + mu * np.eye(k)
    x = xs.copy()
    for _ in range(5):
        x = np.maximum(x - eta * (x @ Gm - b), 0.0)
    assert np.allclose(x, xs, atol=1e-9)


def test_learned_fallback_with_plain_inner_steps():
    """With plain_iters = p the fallback candidate is the plain path's p-step
    update (method.pgd_inner) and the learned update is never worse than it."""
    from oracle import method
    g = np.random.default_rng(12)
    k, hidden = 6, 16
    theta = g.standard_normal(sum(int(np.prod(s)) for _, s in mlp.param_shapes(k, hidden))) * 0.1
    P = mlp.unflatten(theta, k, hidden)
    B = g.random((k, 3 * k))
    G = B @ B.T
    R = g.random((30, k)) * 3.0
    Z = g.random((30, k))
    mu = 0.4
    eta = 1.0 / (method.lambda_max(G) + mu)
    _, xp, fm, fp = mlp.learned_candidates(P, G, mu, R, Z, eta, 3, plain_iters=5)
    assert np.allclose(xp, method.pgd_inner(Z, G, R, eta, mu, 5), rtol=1e-12, atol=1e-12)
    x, keep = mlp.learned_update(P, G, mu, R, Z, eta, 3, plain_iters=5)
    b = R + mu * Z
    assert np.all(mlp.prox_objective(G, mu, b, x) <= mlp.prox_objective(G, mu, b, xp) + 1e-12)


def test_one_sided_loss_equals_relu_error_where_outputs_are_nonnegative():
    """With every pre-activation output o >= 0 the training loss is the plain
    1/2 mean ||max(o, 0) - y*||^2."""
    k, h = 3, 7
    P = _params(k, h, 1)
    P["b3"] = P["b3"] + 50.0  # pushes every o above zero
    groups = _groups(k, 2)
    loss, _ = mlp.loss_and_grads(P, groups)
    N = sum(g[1].shape[0] for g in groups)
    ref = sum(0.5 * float(np.sum((mlp.forward(P, Gn, bn)[0] - ys) ** 2)) for Gn, bn, ys in groups) / N
    assert abs(loss - ref) <= 1e-12 * max(1.0, ref)


def test_dead_outputs_still_get_a_gradient_from_positive_targets():
    """All outputs below zero: the ReLU error has no gradient, the training loss
    still pulls the biases of outputs with positive targets up (negative
    gradient) and leaves those whose targets are all zero alone."""
    k, h = 3, 7
    P = _params(k, h, 2)
    P["b3"] = P["b3"] - 50.0
    Gn, bn, ys = _groups(k, 3)[0]
    ys = ys.copy()
    ys[:, 0] = 0.0
    ys[:, 1:] = np.abs(ys[:, 1:]) + 0.5
    _, grads = mlp.loss_and_grads(P, [(Gn, bn, ys)])
    assert grads["b3"][0] == 0.0
    assert np.all(grads["b3"][1:] < 0.0)
