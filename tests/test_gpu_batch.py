"""Parity of the batched form with the FP64 oracle, instance by instance.

Each instance of a batch follows the single-problem method (Alg. 1 with the
sketched subproblems, Gaussian sketch, its own seed, d and d').  After one
outer iteration from the default factors: U within 1e-5 and V within 2e-5
(norm-wise relative; V inherits U's rounding through the V-half).  After 20
iterations the relative errors agree to 1e-4.
"""
import numpy as np
import pytest

from oracle import bounds, method
from synthdata import batch_specs, planted_dense

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(m=130, n=70, k=8, d=32, d_v=32, seed=0),
    dict(m=1000, n=333, k=16, d=64, d_v=125, seed=1),
    dict(m=257, n=1024, k=32, d=128, d_v=128, seed=2),
    dict(m=64, n=64, k=32, d=128, d_v=128, seed=3),
    dict(m=4096, n=512, k=8, d=64, d_v=512, seed=4),
    dict(m=700, n=2048, k=16, d=256, d_v=87, seed=5),
]


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _inputs(shapes):
    return [planted_dense(s["m"], s["n"], s["k"], 100 + i)[0] for i, s in enumerate(shapes)]


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_one_iteration(pkg, solver, use_graph):
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, solver=solver, use_graph=use_graph)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(1)
    assert b.tuned_blocks() > 0
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U, V = b.factors(i)
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        opt = method.Options(sketch=method.GAUSSIAN, d=s["d"], d_v=s["d_v"], solver=solver)
        Uo, Vo, _ = method.run(M, U0, V0, s["seed"], 1, opt, log_error=False)
        assert _rel(U, Uo) <= 1e-5, (i, _rel(U, Uo))
        assert _rel(V, Vo) <= 2e-5, (i, _rel(V, Vo))
        assert U.min() >= 0 and V.min() >= 0
    b.close()


def test_batch_run_errors(pkg):
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, use_graph=1)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(20)
    errs = b.rel_errors()
    b.close()
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        opt = method.Options(sketch=method.GAUSSIAN, d=s["d"], d_v=s["d_v"])
        _, _, eo = method.run(M, U0, V0, s["seed"], 20, opt)
        assert abs(errs[i] - eo[-1]) <= 1e-4, (i, errs[i], eo[-1])


def test_batch_matches_single_problem_handle(pkg):
    """The batched kernels and the single-problem kernels agree (same method)."""
    s = SHAPES[1]
    M = _inputs([s])[0]
    b = pkg.Batch([s], use_graph=1)
    b.set_dense(0, M)
    b.step(3)
    Ub, Vb = b.factors(0)
    b.close()
    h = pkg.DSANLS(s["m"], s["n"], s["k"], s["d"], pkg.GAUSSIAN, seed=s["seed"], d_v=s["d_v"])
    h.set_dense(M)
    h.step(3)
    Uh, Vh = h.factors()
    h.close()
    assert _rel(Ub, Uh.astype(np.float64)) <= 1e-4 and _rel(Vb, Vh.astype(np.float64)) <= 1e-4


def test_batch_uneven_specs_sampled(pkg):
    """64 instances from the uneven recipe (m in [128, 4096], n in [64, 2048],
    k in {8, 16, 32}); every 8th instance checked after one iteration."""
    specs = batch_specs(64, 0)
    Ms = [planted_dense(s["m"], s["n"], s["k"], s["seed"])[0] for s in specs]
    b = pkg.Batch(specs, use_graph=1)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(1)
    for i in range(0, 64, 8):
        s = specs[i]
        U, V = b.factors(i)
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        opt = method.Options(sketch=method.GAUSSIAN, d=s["d"], d_v=s["d_v"])
        Uo, Vo, _ = method.run(Ms[i], U0, V0, s["seed"], 1, opt, log_error=False)
        assert _rel(U, Uo) <= 1e-5 and _rel(V, Vo) <= 2e-5, i
    b.close()


def test_batch_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.DSANLSError):
        pkg.Batch([dict(m=10, n=10, k=33, d=4, d_v=4, seed=0)])
    b = pkg.Batch([dict(m=10, n=12, k=4, d=4, d_v=4, seed=0)])
    with pytest.raises(pkg.DSANLSError) as e:
        b.step(1)
    assert e.value.code == -4
    with pytest.raises(pkg.DSANLSError):
        b.set_options(precision=pkg.FP8)
    with pytest.raises(pkg.DSANLSError):
        b.set_options(inner_iters=4)
    with pytest.raises(pkg.DSANLSError):
        b.set_options(order=2)
    b.close()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_reassociated_one_iteration(pkg, use_graph):
    """The batched reassociated order R_i = X_i (S_i B_i^T) against the FP64
    oracle of the same order, per instance (1e-5)."""
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, use_graph=use_graph, order=pkg.ORDER_REASSOCIATED)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(1)
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U, V = b.factors(i)
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        M64 = M.astype(np.float64)
        mu = method.mu_t(1.0, 1.0, 0)
        S = method.Sketch(method.GAUSSIAN, s["seed"], 0, 0, s["n"], s["d"])
        Uo = method.half_step(M64, V0.astype(np.float64), U0.astype(np.float64), S, 0, mu, reassociate=True)
        Sp = method.Sketch(method.GAUSSIAN, s["seed"], 0, 1, s["m"], s["d_v"])
        Vo = method.half_step(M64.T, Uo, V0.astype(np.float64), Sp, 0, mu, reassociate=True)
        assert _rel(U, Uo) <= 1e-5, (i, _rel(U, Uo))
        assert _rel(V, Vo) <= 1e-5, (i, _rel(V, Vo))
    b.close()


@pytest.mark.parametrize("order", [0, 1])
def test_batch_bf16_one_iteration(pkg, order):
    """The bf16 batched form per instance: against the exact oracle within the
    derived bound of the form (oracle/bounds.py), and (diagnostic) the
    oracle's bf16 model of the same order (<= 3e-4: fp32 accumulation order
    and the rare bf16 rounding flip of an fp32-accumulated A or P entry)."""
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, use_graph=1, order=order, precision=pkg.BF16)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(1)
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U, V = b.factors(i)
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        M64 = M.astype(np.float64)
        mu = method.mu_t(1.0, 1.0, 0)
        S = method.Sketch(method.GAUSSIAN, s["seed"], 0, 0, s["n"], s["d"])
        Uo = method.half_step(M64, V0.astype(np.float64), U0.astype(np.float64), S, 0, mu, bf16=True,
                              reassociate=order == 1)
        Sp = method.Sketch(method.GAUSSIAN, s["seed"], 0, 1, s["m"], s["d_v"])
        Vo = method.half_step(M64.T, U.astype(np.float64), V0.astype(np.float64), Sp, 0, mu, bf16=True,
                              reassociate=order == 1)
        assert _rel(U, Uo) <= 3e-4, (i, _rel(U, Uo))
        assert _rel(V, Vo) <= 3e-4, (i, _rel(V, Vo))
        form = "bf16_reassociated" if order == 1 else "bf16"
        rel, rb = bounds.check(U, M64, V0.astype(np.float64), U0.astype(np.float64), S, 0, mu, form)
        assert rel <= rb, (i, rel, rb)
        rel, rb = bounds.check(V, M64.T, U.astype(np.float64), V0.astype(np.float64), Sp, 0, mu, form)
        assert rel <= rb, (i, rel, rb)
    b.close()


TILES = [(64, 4, 1), (128, 3, 1), (128, 4, 1), (256, 4, 1), (64, 2, 1),
         (64, 4, 2), (128, 3, 2), (128, 4, 2), (192, 3, 2), (64, 2, 2)]
TILES_LOADERS = ([t + (2,) for t in [(256, 3, 2), (192, 3, 2), (128, 4, 2), (64, 5, 2)]] +
                 [t + (p,) for p in (1, 0) for t in TILES])


def _check_bf16_batch(b, Ms, tag):
    """Every instance of a bf16 batch after one outer iteration within the derived
    bound of the exact oracle."""
    mu = method.mu_t(1.0, 1.0, 0)
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U, V = b.factors(i)
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        M64 = M.astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, s["seed"], 0, 0, s["n"], s["d"])
        rel, rb = bounds.check(U, M64, V0.astype(np.float64), U0.astype(np.float64), S, 0, mu, "bf16")
        assert rel <= rb, (tag, i, rel, rb)
        Sp = method.Sketch(method.GAUSSIAN, s["seed"], 0, 1, s["m"], s["d_v"])
        rel, rb = bounds.check(V, M64.T, U.astype(np.float64), V0.astype(np.float64), Sp, 0, mu, "bf16")
        assert rel <= rb, (tag, i, rel, rb)


def test_batch_tile_per_side(pkg):
    """Each half-step has its own tile: pinned differently for the U- and the
    V-half, both are reported as pinned and the results stay within the bound."""
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, use_graph=1, precision=pkg.BF16)
    b.set_tile(192, 3, 2, 2, side=0)
    b.set_tile(128, 3, 1, 1, side=1)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(1)
    assert b.tuned_tile(0)[0::2] == (192, 2) and b.tuned_tile(0)[3] == 2
    assert b.tuned_tile(1)[0::2] == (128, 1) and b.tuned_tile(1)[3] == 1
    _check_bf16_batch(b, Ms, "per side")
    b.close()


@pytest.mark.parametrize("tile", TILES_LOADERS)
def test_batch_bf16_every_tile(pkg, tile):
    """Each tile of the tensor-core product pinned in turn (chunk of sketch columns,
    ring stages, one or two 128-row tiles per work item, operand ring fed by TMA or
    by cp.async, the chunk epilogue off the copy path or not): every instance within the
    derived bound of the exact oracle.  The
    shapes give pairs of row tiles whose second tile is ragged or empty (257 and 64
    rows), sketches of several chunks (d' = 512, d = 256) and K not a multiple of
    64 (the TMA boxes past K read zeros)."""
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, use_graph=1, precision=pkg.BF16)
    b.set_tile(*tile)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(1)
    for side in (0, 1):
        chunk, ctas, row_tiles, pipeline = b.tuned_tile(side)
        assert (chunk, row_tiles, pipeline) == (tile[0], tile[2], tile[3]) and ctas > 0
    mu = method.mu_t(1.0, 1.0, 0)
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U, V = b.factors(i)
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        M64 = M.astype(np.float64)
        S = method.Sketch(method.GAUSSIAN, s["seed"], 0, 0, s["n"], s["d"])
        rel, rb = bounds.check(U, M64, V0.astype(np.float64), U0.astype(np.float64), S, 0, mu, "bf16")
        assert rel <= rb, (tile, i, rel, rb)
        Sp = method.Sketch(method.GAUSSIAN, s["seed"], 0, 1, s["m"], s["d_v"])
        rel, rb = bounds.check(V, M64.T, U.astype(np.float64), V0.astype(np.float64), Sp, 0, mu, "bf16")
        assert rel <= rb, (tile, i, rel, rb)
    b.close()


def test_batch_set_tile_rejects_unbuilt_tiles(pkg):
    b = pkg.Batch(SHAPES[:2], precision=pkg.BF16)
    for bad in [(96, 3, 2, 1), (256, 4, 2, 1), (128, 2, 1, 0), (64, 4, 3, 1), (64, 4, 1, 3), (192, 4, 2, 2),
                (192, 3, 1, 2)]:
        with pytest.raises(pkg.DSANLSError):
            b.set_tile(*bad)
    b.set_tile(0, 0, 0)  # back to the autotuner
    b.close()


def test_batch_bf16_tensor_core_tile_is_tuned(pkg):
    """The bf16 paper order runs R_i = (X_i S_i) B_i^T on tensor cores; the
    autotuner times the candidate tiles (64- to 256-column chunks of the sketch,
    one or two 128-row tiles per work item, each with its CTAs per SM) on the real batch -- every candidate
    runs a full iteration, with the factors restored after each -- and keeps
    one; the first iteration then matches a second handle that reuses the
    cached choice bit for bit."""
    Ms = _inputs(SHAPES)
    out = []
    for _ in range(2):
        b = pkg.Batch(SHAPES, use_graph=1, precision=pkg.BF16)
        for i, M in enumerate(Ms):
            b.set_dense(i, M)
        b.step(1)
        for side in (0, 1):
            chunk, ctas, row_tiles, pipeline = b.tuned_tile(side)
            assert (chunk, row_tiles) in ((64, 1), (128, 1), (256, 1), (64, 2), (128, 2), (192, 2), (256, 2))
            assert ctas > 0 and pipeline in (0, 1, 2)
        out.append([b.factors(i) for i in range(len(SHAPES))])
        b.close()
    for (u0, v0), (u1, v1) in zip(*out):
        assert np.array_equal(u0, u1) and np.array_equal(v0, v1)


def test_batch_bf16_run_final_errors(pkg):
    """20 outer iterations of every instance, bf16 tensor-core form with the last
    three in binary32: each instance's final relative error within 2e-3 of the
    exact oracle's (the acceptance of the reduced-precision forms)."""
    Ms = _inputs(SHAPES)
    b = pkg.Batch(SHAPES, use_graph=1, precision=pkg.BF16)
    for i, M in enumerate(Ms):
        b.set_dense(i, M)
    b.step(17)
    b.set_options(precision=pkg.FP32, t=17)
    b.step(3)
    errs = b.rel_errors()
    b.close()
    for i, (s, M) in enumerate(zip(SHAPES, Ms)):
        U0, V0 = method.default_init(s["seed"], s["m"], s["n"], s["k"])
        opt = method.Options(sketch=method.GAUSSIAN, d=s["d"], d_v=s["d_v"])
        _, _, eo = method.run(M, U0, V0, s["seed"], 20, opt)
        assert abs(errs[i] - eo[-1]) <= 2e-3, (i, errs[i], eo[-1])
