"""Complex H through the C ABI (sexpm_plan_z / sexpm_compute / sexpm_result_copy_z): parity with
the complex oracle at the same bar as the real path (1e-12 ||e^H||_1 element-wise; entries stored
by one side only at most 2 t), the Schroedinger propagator of a grid Laplacian against its
closed form, unitarity, and edge cases."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sexpm_oracle as O
from tests._compare import expm_parity
from workloads import dirichlet_laplacian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


def _dev(Z, device="cuda"):
    import torch
    Z = sp.csr_matrix(Z, dtype=np.complex128)
    Z.sort_indices()
    return (torch.from_numpy(Z.indptr.astype(np.int64)).to(device), torch.from_numpy(Z.indices.astype(np.int32)).to(device),
            torch.from_numpy(Z.data.astype(np.complex128)).to(device), Z.shape[0])


def _to_scipy(rp, ci, v, n):
    return sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))


def _rand_complex(n, seed, density=0.08, scale=1.0, empty_rows=0):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=rng, format="csr")
    A.data = rng.standard_normal(A.nnz) + 1j * rng.standard_normal(A.nnz)
    A = sp.csr_matrix(A * scale)
    if empty_rows:
        A = A.tolil()
        for i in rng.choice(n, size=empty_rows, replace=False):
            A.rows[i] = []
            A.data[i] = []
        A = A.tocsr()
    return A


def _parity(sx, Z, tau, eps, **opts):
    (rp, ci, v), st = sx.expm_complex(_dev(Z), tau, eps, **opts)
    G = _to_scipy(rp, ci, v, Z.shape[0])
    E, so = O.expm(sp.csr_matrix(Z, dtype=np.complex128), tau, eps)
    assert (st["M"], st["N"]) == (so.M, so.N)
    assert bool(st["normal"]) == bool(so.normal)
    ts = [r["t"] for r in st["steps"]] + [s.t for s in so.steps] + [t.t for t in so.taylor]
    expm_parity(G, E, max(ts) if ts else 0.0)
    return G, st


@pytest.mark.parametrize("kind", ["general", "hermitian_times_i", "skew_hermitian", "non_normal_scaled"])
def test_complex_matches_oracle(sx, kind):
    Z = _rand_complex(120, seed={"general": 1, "hermitian_times_i": 2, "skew_hermitian": 3, "non_normal_scaled": 4}[kind],
                      empty_rows=5)
    if kind == "hermitian_times_i":
        Z = sp.csr_matrix(1j * (Z + Z.conj().T))
    elif kind == "skew_hermitian":
        Z = sp.csr_matrix(Z - Z.conj().T)
    elif kind == "non_normal_scaled":
        Z = sp.csr_matrix(Z * 3.0)
    _parity(sx, Z, 1.0, 1e-12)


def test_schroedinger_propagator_of_a_grid_laplacian(sx):
    """e^{i tau L} of the 2-D Dirichlet Laplacian (24 x 24 grid): parity with the oracle and
    element-wise agreement with V e^{i tau Lambda} V^T (x) itself from the sine eigenbasis."""
    m, tau = 24, 2e-4
    L = dirichlet_laplacian(m, 2).to_scipy()
    Z = sp.csr_matrix(1j * L)
    G, st = _parity(sx, Z, tau, 1e-12)
    assert st["normal"] == 1
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam = -(4.0 / h ** 2) * np.sin(j * np.pi * h / 2) ** 2
    V = np.sqrt(2 * h) * np.sin(np.outer(j, j) * np.pi * h)
    E1 = (V * np.exp(1j * tau * lam)) @ V.T
    X = np.kron(E1, E1)
    assert np.abs(G.toarray() - X).max() <= 1e-12 * np.abs(X).sum(axis=0).max()
    # unitary (up to the filter's bound)
    U = G.toarray()
    assert np.abs(U @ U.conj().T - np.eye(m * m)).max() <= 1e-11


def test_real_input_through_the_complex_path(sx):
    """A real matrix given as complex: the same (M, N) and, to the parity bar, the same e^H as the
    real path; every imaginary part is zero."""
    L = dirichlet_laplacian(16, 2).to_scipy()
    G, st = _parity(sx, sp.csr_matrix(L, dtype=np.complex128), 1e-3, 1e-12)
    assert not np.any(G.data.imag)
    (rp, ci, v), st_r = sx.expm((L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data, L.shape[0]), 1e-3, 1e-12)
    R = sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=L.shape)
    assert (st["M"], st["N"]) == (st_r["M"], st_r["N"])
    assert abs(G.real - R).max() <= 1e-12 * float(np.abs(R).sum(axis=0).max())


def test_complex_edge_cases(sx):
    # scalar phase e^{i theta}: the oracle's result, and the closed form within the tolerance
    G, _ = _parity(sx, sp.csr_matrix(np.array([[0.7j]])), 1.0, 1e-14)
    assert abs(complex(G[0, 0]) - np.exp(0.7j)) <= 1e-14
    # all-zero stored matrix: e^0 = I
    Z = sp.csr_matrix((np.zeros(2, dtype=np.complex128), np.array([1, 2]), np.array([0, 1, 2, 2])), shape=(3, 3))
    (rp, ci, v), st = sx.expm_complex(_dev(Z), 1.0, 1e-12)
    assert (st["M"], st["N"]) == (0, 0)
    assert np.array_equal(_to_scipy(rp, ci, v, 3).toarray(), np.eye(3))
    # host input arrays, a 2 x 2 non-normal complex matrix
    A = np.array([[1 + 1j, 2.0], [0.0, -1 + 0.5j]])
    S = sp.csr_matrix(A)
    Gh, _ = sx.expm_complex((S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data, 2), 1.0, 1e-13)
    import scipy.linalg as sla
    X = sla.expm(A)
    assert np.abs(_to_scipy(*Gh, 2).toarray() - X).max() <= 1e-12 * np.abs(X).sum(axis=0).max()


def test_complex_rejects_invalid_input_and_real_only_calls(sx):
    S = sp.csr_matrix(np.array([[1j, 2.0], [0.0, np.nan]]))
    with pytest.raises(sx.SexpmError):
        sx.ComplexPlan((S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data, 2), 1e-12)
    P = sx.ComplexPlan(_dev(sp.csr_matrix(np.array([[1j, 0.5], [0.5, 0.0]]))), 1e-12)
    try:
        r = P.compute(1.0)
        with pytest.raises(sx.SexpmError):
            sx.Result.to_torch(r, "cpu")  # the real copy refuses a complex result
        r.free()
        with pytest.raises(sx.SexpmError):
            P.forward_keep(1.0)
    finally:
        P.close()
