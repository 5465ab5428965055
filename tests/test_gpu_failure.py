"""Failure paths, tested without faulting, trapping or hanging the GPU.

  * Allocation failure: the C API's test switch makes the n-th device
    allocation of a handle fail as if the device were out of memory; create
    and set_dense return DSANLS_ENOMEM, give back what they had allocated,
    and the library works normally once the switch is off.
  * Bounded device waits: the test switch makes the tensor-core GEMM's TMA
    producer issue no copy (nothing is in flight) and shortens the wait
    limit to 50 ms; the consumers' waits run out, the kernel frees its tensor
    memory and returns, the next synchronising call reports DSANLS_ETIMEOUT,
    and the same handle then computes a correct half-step.
"""
import numpy as np
import pytest

from oracle import bounds, method
from synthdata import initial_factors, planted_dense

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT = -2, -6


@pytest.fixture(scope="module")
def pkg():
    import paper_2009_02845_gb300 as p
    return p


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("budget", [0, 1, 3, 7])
def test_create_out_of_memory_is_clean(pkg, budget):
    import torch
    torch.cuda.init()
    h0 = pkg.DSANLS(512, 256, 16, 64, pkg.GAUSSIAN, seed=0)  # primes the device outside the measurement
    h0.close()
    free0 = _free_bytes()
    pkg.debug_fail_alloc_after(budget)
    try:
        with pytest.raises(pkg.DSANLSError) as e:
            pkg.DSANLS(4096, 2048, 64, 256, pkg.GAUSSIAN, seed=0)
        assert e.value.code == ENOMEM
    finally:
        pkg.debug_fail_alloc_after(-1)
    assert abs(_free_bytes() - free0) <= 4 << 20  # everything allocated before the failure was released


def test_set_dense_out_of_memory_then_recovers(pkg):
    m, n, k, d = 1024, 512, 16, 64
    M, _, _ = planted_dense(m, n, k, 0)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=0)
    pkg.debug_fail_alloc_after(0)
    try:
        with pytest.raises(pkg.DSANLSError) as e:
            h.set_dense(M)
        assert e.value.code == ENOMEM
    finally:
        pkg.debug_fail_alloc_after(-1)
    h.set_dense(M)  # the handle is still usable
    h.step(2)
    assert 0.0 < h.rel_error() < 1.0
    h.close()


def test_tensor_core_wait_runs_out_and_the_handle_recovers(pkg):
    m, n, k, d = 512, 256, 32, 256
    M, _, _ = planted_dense(m, n, 16, 1)
    U, V = initial_factors(m, n, k, 2)
    h = pkg.DSANLS(m, n, k, d, pkg.GAUSSIAN, seed=3, precision=pkg.BF16, t=1)
    h.set_dense(M)
    h.set_factors(U, V)
    pkg.debug_tc_wait(50_000_000, starve=True)
    try:
        h.half_step(0)
        with pytest.raises(pkg.DSANLSError) as e:
            h.sync()
        assert e.value.code == ETIMEOUT
    finally:
        pkg.debug_tc_wait(0, starve=False)
    # the context is intact: the same handle, from the same factors, gives the right step
    h.set_factors(U, V)
    h.half_step(0)
    Ug, _ = h.factors()
    h.close()
    S = method.Sketch(method.GAUSSIAN, 3, 1, 0, n, d)
    rel, rb = bounds.check(Ug, M.astype(np.float64), V.astype(np.float64), U.astype(np.float64), S, method.PGD,
                           method.mu_t(1.0, 1.0, 1), "bf16")
    assert rel <= rb, (rel, rb)


def test_tc_wait_switch_rejects_a_starve_without_limit(pkg):
    with pytest.raises(pkg.DSANLSError):
        pkg.debug_tc_wait(0, starve=True)
