"""Pins of the acceptance bounds of the reduced-precision forms (oracle/bounds.py).

The bound must (1) hold for every deterministic rounding model of the oracle
(round_bf16 / round_e4m3 at the form's rounding points, themselves pinned to
torch's conversions in test_oracle_method.py) against the exact FP64 step,
(2) not be vacuous -- within a fixed factor of the error it bounds and below a
few units of the format's unit roundoff -- and (3) reject plausible mistakes
in a step: a dropped rounding-free term, a wrong step size, a missing 1/sqrt(d).
Its product-error formula is checked against a direct Monte-Carlo simulation of
the rounding model.
"""
import numpy as np
import pytest

from oracle import bounds, method
from synthdata import initial_factors, planted_dense

CASES = [(256, 128, 16, 256, 256), (1000, 808, 10, 104, 96), (640, 528, 64, 520, 264)]
FORM_KW = {
    "bf16": dict(bf16=True),
    "bf16_reassociated": dict(bf16=True, reassociate=True),
    "bf16_identity": dict(bf16=True),
}


def _setup(case, side, form, t=2, seed=21):
    m, n, k, d, d_v = case
    M, _, _ = planted_dense(m, n, min(k, 16), 2)
    U, V = initial_factors(m, n, k, 3)
    M64 = M.astype(np.float64)
    X = M64 if side == 0 else M64.T
    Y = (V if side == 0 else U).astype(np.float64)
    Z = (U if side == 0 else V).astype(np.float64)
    dd = d if side == 0 else d_v
    if form == "bf16_identity":
        S = method.Sketch(method.IDENTITY, seed, t, side, X.shape[1], X.shape[1])
    else:
        S = method.Sketch(method.GAUSSIAN, seed, t, side, X.shape[1], dd)
    return X, Y, Z, S, method.mu_t(1.0, 1.0, t)


def _model(X, Y, Z, S, solver, mu, form, side, t=2, seed=21, inner=1):
    if form == "fp8":
        return method.half_step(X, Y, Z, S, solver, mu, fp8=(seed, t, side), inner_iters=inner)
    if form == "fp8_reassociated":
        return method.half_step(X, Y, Z, S, solver, mu, fp8=(seed, t, side), reassociate=True, inner_iters=inner)
    return method.half_step(X, Y, Z, S, solver, mu, inner_iters=inner, **FORM_KW[form])


UNIT = {"bf16": bounds.U_BF16, "bf16_reassociated": bounds.U_BF16, "bf16_identity": bounds.U_BF16,
        "fp8": bounds.U_E4M3, "fp8_reassociated": bounds.U_E4M3}


@pytest.mark.parametrize("form", bounds.FORMS)
@pytest.mark.parametrize("solver", [method.PGD, method.RCD])
@pytest.mark.parametrize("case", CASES)
def test_bound_holds_for_the_rounding_models_and_is_not_vacuous(case, solver, form):
    for side in (0, 1):
        X, Y, Z, S, mu = _setup(case, side, form)
        got = _model(X, Y, Z, S, solver, mu, form, side)
        rel, rb = bounds.check(got, X, Y, Z, S, solver, mu, form)
        assert rel <= rb, (side, rel, rb)
        assert rb <= 64.0 * rel, (side, rel, rb)       # within a fixed factor of the real deviation
        assert rb <= 32.0 * UNIT[form], (side, rb)       # a few units of the format's roundoff


def test_bound_with_inner_steps_holds():
    case = (640, 528, 64, 520, 264)
    for side in (0, 1):
        X, Y, Z, S, mu = _setup(case, side, "bf16_reassociated")
        got = _model(X, Y, Z, S, method.PGD, mu, "bf16_reassociated", side, inner=8)
        rel, rb = bounds.check(got, X, Y, Z, S, method.PGD, mu, "bf16_reassociated", inner_iters=8)
        assert rel <= rb <= 0.1, (rel, rb)


@pytest.mark.parametrize("form", ["bf16", "fp8", "bf16_reassociated"])
def test_bound_rejects_plausible_mistakes(form):
    """Steps with a mistake the bound must catch: R without its 1/sqrt(d)
    scaling of S, a step size 2 % off, and the gradient's sign flipped."""
    X, Y, Z, S, mu = _setup((640, 528, 64, 520, 264), 0, form)
    _, _, G, R = method.sketched_terms(X, Y, S)
    eta = 1.0 / (method.lambda_max(G) + mu)
    _, rb = bounds.check(Z, X, Y, Z, S, method.PGD, mu, form)
    d = S.d
    mistakes = [
        method.pgd_update(Z, G, R * np.sqrt(d), eta),
        method.pgd_update(Z, G, R, 1.02 * eta),
        method.project(Z + eta * (Z @ G - R)),
    ]
    for bad in mistakes:
        rel, _ = bounds.check(bad, X, Y, Z, S, method.PGD, mu, form)
        assert rel > rb, (rel, rb)


def test_product_rms_matches_a_simulation_of_the_model():
    """E ||fl(X) fl(Y) - X Y||_F^2 from the formula against the mean over 200
    draws of the model at its largest magnitudes (|delta| = u, random signs),
    for which the formula is exact up to the second-order term."""
    g = np.random.default_rng(0)
    X = g.random((40, 300))
    Y = g.standard_normal((300, 30))
    u = bounds.U_BF16
    want = bounds.product_rms(X, Y, u, u) ** 2 - 300 * bounds.V_F32 ** 2 * float(
        np.sum((np.abs(X) @ np.abs(Y)) ** 2))
    sims = []
    for _ in range(200):
        Xp = X * (1 + u * g.choice((-1.0, 1.0), size=X.shape))
        Yp = Y * (1 + u * g.choice((-1.0, 1.0), size=Y.shape))
        sims.append(float(np.sum((Xp @ Yp - X @ Y) ** 2)))
    assert abs(np.mean(sims) / want - 1.0) < 0.05


def test_entry_variance_of_the_right_hand_side_matches_a_simulation():
    """The propagated bound e_R / 3 (the rms of ||dR||_F, Minkowski over the
    error terms) is at least the simulated rms of the bf16 form's ||dR||_F
    under the model and at most 2.5 times it."""
    X, Y, Z, S, mu = _setup((256, 128, 16, 256, 256), 0, "bf16")
    T = bounds.terms_bound(X, Y, S, "bf16")
    g = np.random.default_rng(1)
    sq = [float(np.sum((bounds.perturbed_terms(X, Y, S, "bf16", g)[1] - T.R) ** 2)) for _ in range(40)]
    rms = float(np.sqrt(np.mean(sq)))
    assert rms <= T.eR / 3.0 <= 2.5 * rms, (rms, T.eR / 3.0)
