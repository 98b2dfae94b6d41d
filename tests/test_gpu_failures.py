"""Error paths of the C ABI, all made on the host (no GPU fault): Algorithm 4.1's iteration cap
(SEXPM_ENOCONV), an unreachable tolerance (SEXPM_ENOPARAM), and a device allocation that fails
(SEXPM_ENOMEM, injected on the host by SEXPM_FAIL_ALLOC_AT before the allocation is made).  After
each failure nothing stays allocated and the plan still computes the same result."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from tests._compare import to_scipy, torch_csr
from workloads import CSR, dirichlet_laplacian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


def test_filter_iteration_cap_returns_enoconv(sx):
    """The hand-trace input 1, -2, 3, 4 with eps_g = 3 needs two Algorithm 4.1 passes."""
    A = CSR.from_scipy(sp.csr_matrix(np.array([[1.0, -2.0], [3.0, 4.0]])))
    with pytest.raises(sx.SexpmError) as ei:
        sx.filter_csr(torch_csr(A), 3.0, 0.1, max_iters=1)
    assert ei.value.code == -4 and "did not converge" in str(ei.value)
    (rp, ci, v), t, it, b = sx.filter_csr(torch_csr(A), 3.0, 0.1, max_iters=2)
    assert it == 2 and t == pytest.approx(9 / math.sqrt(14))


def test_unreachable_tolerance_returns_enoparam(sx):
    H = dirichlet_laplacian(6, 2)
    plan = sx.Plan(torch_csr(H), 1e-300, n_extra=0, max_taylor=3)
    try:
        with pytest.raises(sx.SexpmError) as ei:
            plan.compute(1e-2)
        assert ei.value.code == -5
    finally:
        plan.close()


@pytest.mark.parametrize("k", [1, 3, 8, 20, 60])
def test_injected_allocation_failure_returns_enomem_and_leaks_nothing(sx, monkeypatch, k):
    H = dirichlet_laplacian(24, 2)
    tau = 2.253 / 25 ** 2
    plan = sx.Plan(torch_csr(H), 1e-12)
    try:
        ref = plan.compute(tau)
        r_rp, r_ci, r_v = ref.to_numpy()
        ref.free()
        live0, _ = sx.pool_stats()
        monkeypatch.setenv("SEXPM_FAIL_ALLOC_AT", str(k))
        with pytest.raises(sx.SexpmError) as ei:
            plan.compute(tau)
        assert ei.value.code == -2 and "injected" in str(ei.value)
        assert sx.pool_stats()[0] == live0
        monkeypatch.delenv("SEXPM_FAIL_ALLOC_AT")
        again = plan.compute(tau)
        a_rp, a_ci, a_v = again.to_numpy()
        again.free()
        assert np.array_equal(a_rp, r_rp) and np.array_equal(a_ci, r_ci) and np.array_equal(a_v, r_v)
        assert sx.pool_stats()[0] == live0
    finally:
        plan.close()
