"""The bf16-factor form of sparse data (subsampling sketch, BF16 precision): U
and V are stored in bf16, halving the bytes of the HBM-bound row update.

Rounding points (the form's definition): the factors are bf16 values; each
half-step computes B, G, R and the projected-gradient step in binary32 /
FP64 from those exact values and rounds the updated factor to bf16 when it
is stored.  Against the exact oracle run from the same (bf16) factors, the
step therefore differs only by that final rounding: |z_gpu - z_exact| <=
2^-8 |z_exact| per entry (plus binary32 arithmetic, 1e-5), so the norm-wise
deviation is at most 2^-8 + 1e-5; and most entries equal the bf16 rounding
of the exact value (the others sit at a rounding boundary).  A 20-iteration
run ends within 2e-3 of the oracle's relative error.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import method
from synthdata import initial_factors, sparse_text

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _csr(m, n, seed, mean_len):
    rp, col, val = sparse_text(m, n, seed, mean_len=mean_len)
    return rp, col, val, sp.csr_matrix((val.astype(np.float64), col, rp), shape=(m, n))


@pytest.mark.parametrize("case", [
    (3000, 1200, 48, 300, 400, 20.0),
    (2000, 5000, 100, 500, 300, 40.0),
    # several 128-row tiles per CTA, ragged last tiles whose bytes are not a multiple
    # of 16 (k = 66 also takes the scalar row slices)
    (70001, 700, 66, 300, 2000, 20.0),
    (60001, 900, 100, 400, 3000, 20.0),
])
def test_bf16_factor_half_steps(pkg, case):
    m, n, k, d, d_v, mean_len = case
    rp, col, val, Msp = _csr(m, n, 7, mean_len)
    U, V = initial_factors(m, n, k, 8)
    Ub, Vb = method.round_bf16(U), method.round_bf16(V)
    for side, dd in ((0, d), (1, d_v)):
        h = pkg.DSANLS(m, n, k, d, pkg.SUBSAMPLE, seed=5, d_v=d_v, precision=pkg.BF16, t=3)
        h.set_csr(rp, col, val)
        h.set_factors(U, V)
        h.half_step(side)
        Ug, Vg = h.factors()
        h.close()
        got = (Ug if side == 0 else Vg).astype(np.float64)
        X = Msp if side == 0 else Msp.T.tocsr()
        Y, Z = (Vb, Ub) if side == 0 else (Ub, Vb)
        S = method.Sketch(method.SUBSAMPLE, 5, 3, side, X.shape[1], dd)
        exact = method.half_step(X, Y, Z, S, method.PGD, method.mu_t(1.0, 1.0, 3))
        assert np.array_equal(got, method.round_bf16(got)), "stored factors are bf16 values"
        rel = np.linalg.norm(got - exact) / np.linalg.norm(exact)
        assert rel <= U_BF16 + 1e-5, (side, rel)
        assert np.mean(got != method.round_bf16(exact)) <= 0.01, side


def test_bf16_factor_run_final_error(pkg):
    m, n, k, d = 3000, 1200, 48, 300
    rp, col, val, Msp = _csr(m, n, 9, 20.0)
    U0, V0 = method.default_init(2, m, n, k)
    h = pkg.DSANLS(m, n, k, d, pkg.SUBSAMPLE, seed=2, precision=pkg.BF16, use_graph=1)
    h.set_csr(rp, col, val)
    h.step(20)
    err = h.rel_error()
    h.close()
    _, _, errs = method.run(Msp, method.round_bf16(U0), method.round_bf16(V0), 2, 20,
                            method.Options(sketch=method.SUBSAMPLE, d=d))
    assert abs(err - errs[-1]) <= 2e-3, (err, errs[-1])


def test_bf16_factor_form_rejects_other_solvers(pkg):
    h = pkg.DSANLS(300, 200, 48, 40, pkg.SUBSAMPLE, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(precision=pkg.BF16, solver=pkg.RCD)
    h.close()
    h = pkg.DSANLS(300, 200, 16, 40, pkg.SUBSAMPLE, seed=0)
    with pytest.raises(pkg.DSANLSError):
        h.set_options(precision=pkg.BF16)  # k <= 32: the CUDA-core update keeps binary32 factors
    h.close()
