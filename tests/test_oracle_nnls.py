"""Pins of the oracle's exact NNLS solvers and the planted-recovery check.

The NNLS subproblems (Section 2.1, eq. subproblem) are pinned by: agreement
of brute-force support enumeration with the active-set solver and with
scipy's independent NNLS routine for k <= 4; KKT conditions; and exact ANLS
recovering a noise-free planted factorisation M = U0 V0^T to relative error
< 1e-6 (Alg. 1 with exact subproblem solves).
"""
import numpy as np
import pytest
from scipy.optimize import nnls as scipy_nnls

from oracle import nnls


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_brute_force_active_set_and_scipy_agree(k):
    g = np.random.default_rng(k)
    for trial in range(40):
        Y = g.standard_normal((12, k))
        y = g.standard_normal(12) + (trial % 3)
        G, b = Y.T @ Y, Y.T @ y
        xb = nnls.brute_force(G, b)
        xa = nnls.active_set(G, b)
        xs, _ = scipy_nnls(Y, y)
        assert np.allclose(xb, xs, atol=1e-9)
        assert np.allclose(xa, xs, atol=1e-9)
        assert nnls.kkt_ok(G, b, xb) and nnls.kkt_ok(G, b, xa)


def test_kkt_rejects_wrong_points():
    G = np.array([[2.0, 0.5], [0.5, 1.0]])
    b = np.array([1.0, -1.0])
    x = nnls.brute_force(G, b)
    assert nnls.kkt_ok(G, b, x)
    assert not nnls.kkt_ok(G, b, x + np.array([0.1, 0.0]))
    assert not nnls.kkt_ok(G, b, np.array([0.0, 0.3]))


def test_planted_recovery_by_exact_anls():
    g = np.random.default_rng(0)
    m, n, k = 40, 30, 3
    U0, V0 = g.random((m, k)), g.random((n, k))
    M = U0 @ V0.T
    best = np.inf
    for restart in range(3):
        U, V = g.random((m, k)), g.random((n, k))
        U, V = nnls.anls(M, U, V, 300)
        best = min(best, np.linalg.norm(M - U @ V.T) / np.linalg.norm(M))
        if best < 1e-6:
            break
    assert best < 1e-6
