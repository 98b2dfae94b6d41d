"""Applying a computed e^{tau H} to vectors (sexpm_result_spmm, sexpm_spmm) and time stepping with
it (sexpm_propagate, Eq. 2.2), through the C ABI."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

from tests._compare import torch_csr
from workloads import CSR, dirichlet_laplacian, random_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


@pytest.mark.parametrize("r", [1, 2, 3, 8, 11])
def test_spmm_matches_scipy(sx, r):
    """Ragged random matrix with empty rows; r vectors (several chunks of 8 when r > 8)."""
    import torch
    A = random_csr(3000, 0.003, seed=r, scale=2.0)
    X = np.random.default_rng(r).standard_normal((A.n, r))
    Y = sx.spmm(torch_csr(A), torch.from_numpy(X).cuda()).cpu().numpy()
    ref = A.to_scipy() @ X
    assert np.abs(Y - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0)


def _sine_basis_expm(m, tau):
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam = -(4.0 / h ** 2) * np.sin(j * np.pi * h / 2) ** 2
    V = np.sqrt(2 * h) * np.sin(np.outer(j, j) * np.pi * h)
    return (V * np.exp(tau * lam)) @ V.T


def test_propagate_matches_the_closed_form(sx):
    """Ten steps U_k = E U_{k-1} with E = e^{tau L} (32 x 32 grid, tau = 1e-3) against
    e^{10 tau L} U_0 = (E_1 (x) E_1) U_0 from the sine eigenbasis with 10 tau."""
    import torch
    m, tau, steps = 32, 1e-3, 10
    H = dirichlet_laplacian(m, 2)
    plan = sx.Plan(torch_csr(H), 1e-14)
    try:
        E = plan.compute(tau)
        U0 = np.random.default_rng(3).uniform(-1, 1, (H.n, 4))
        dU0 = torch.from_numpy(U0).cuda()
        U = E.propagate(dU0, steps).cpu().numpy()
        # the C entry point with U aliasing U0
        alias = dU0.clone()
        sx._check(sx.load().sexpm_propagate(E._h, alias.data_ptr(), 4, steps, alias.data_ptr(), sx._stream_ptr()))
        assert np.array_equal(alias.cpu().numpy(), U)
        one = E.spmm(dU0).cpu().numpy()
        assert np.array_equal(E.propagate(dU0, 1).cpu().numpy(), one)
        assert np.array_equal(E.propagate(dU0, 0).cpu().numpy(), U0)
        E.free()
    finally:
        plan.close()
    E1 = _sine_basis_expm(m, steps * tau)
    exact = np.stack([(E1 @ U0[:, c].reshape(m, m) @ E1.T).ravel() for c in range(4)], axis=1)
    assert np.abs(U - exact).max() <= 1e-11
