"""Pins of the oracle for complex H (the method is stated for C^{n x n}): dense Pade on small
matrices of every kind, the Schroedinger propagator e^{i tau L} of a grid Laplacian from the sine
eigenbasis, unitarity of e^{iA} for Hermitian A, Algorithm 4.1 deciding by the modulus, the
normality test with the conjugate transpose, and real input taking exactly the real path."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import sexpm_oracle as O
from workloads import dirichlet_laplacian


def _rand_complex(n, seed, density=0.4, scale=1.0):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=rng, format="csr")
    B = sp.random(n, n, density=density, random_state=rng, format="csr")
    A.data = rng.standard_normal(A.nnz)
    B.data = rng.standard_normal(B.nnz)
    return sp.csr_matrix((A + 1j * B) * scale)


@pytest.mark.parametrize("kind", ["general", "hermitian", "skew_hermitian", "scaled_up"])
def test_complex_oracle_matches_dense_pade(kind):
    Z = _rand_complex(14, seed={"general": 1, "hermitian": 2, "skew_hermitian": 3, "scaled_up": 4}[kind])
    if kind == "hermitian":
        Z = sp.csr_matrix(Z + Z.conj().T)
    elif kind == "skew_hermitian":
        Z = sp.csr_matrix(Z - Z.conj().T)
    elif kind == "scaled_up":
        Z = Z * 6.0
    E, st = O.expm(Z, 1.0, 1e-14)
    X = sla.expm(Z.toarray())
    assert np.abs(E.toarray() - X).max() <= 1e-12 * np.abs(X).sum(axis=0).max()
    assert st.normal == (kind in ("hermitian", "skew_hermitian"))


def _sine_basis(m):
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam = -(4.0 / h ** 2) * np.sin(j * np.pi * h / 2) ** 2
    V = np.sqrt(2 * h) * np.sin(np.outer(j, j) * np.pi * h)
    return lam, V


def test_schroedinger_propagator_matches_sine_basis():
    """e^{i tau L} for the 2-D Dirichlet Laplacian on a 12x12 grid: the 1-D factor
    V diag(e^{i tau lambda}) V^T and the Kronecker product (node x + m y)."""
    m, tau = 12, 2e-4
    L = dirichlet_laplacian(m, 2).to_scipy()
    E, st = O.expm(sp.csr_matrix(1j * L), tau, 1e-14)
    lam, V = _sine_basis(m)
    E1 = (V * np.exp(1j * tau * lam)) @ V.T
    X = np.kron(E1, E1)
    assert st.normal
    assert np.abs(E.toarray() - X).max() <= 1e-12 * np.abs(X).sum(axis=0).max()


def test_exponential_of_i_times_hermitian_is_unitary():
    A = _rand_complex(16, seed=7)
    A = sp.csr_matrix((A + A.conj().T) * 0.8)
    U, _ = O.expm(sp.csr_matrix(1j * A), 1.0, 1e-14)
    U = U.toarray()
    assert np.abs(U @ U.conj().T - np.eye(16)).max() <= 1e-12


def test_scalar_phase():
    """e^{i theta I} = e^{i theta} I."""
    theta = 0.7
    E, _ = O.expm(sp.csr_matrix(1j * theta * sp.identity(5)), 1.0, 1e-15)
    assert np.abs(E.toarray() - np.exp(1j * theta) * np.eye(5)).max() <= 2e-16 * 8


def test_algorithm_41_decides_by_the_modulus():
    """|3+4i| = 5 is kept at eps_f = 4.8 although its real and imaginary parts are below it;
    the dropped part is {4.5, 0.1i}: b^2 = 20.25 + 0.01 (one pass, b <= 4.8 (1 + 0.1))."""
    vals = np.array([3 + 4j, 4.5 + 0j, 0.1j])
    t, iters, b = O.alg41_threshold(vals, 4.8, 0.1)
    assert (t, iters) == (4.8, 1)
    assert abs(b * b - 20.26) <= 1e-13
    A = sp.csr_matrix(np.array([[3 + 4j, 4.5, 0.1j]]))
    B, info = O.filter_csr(A, 4.8, 0.1)
    assert B.nnz == 1 and B[0, 0] == 3 + 4j


def test_normality_uses_the_conjugate_transpose():
    """[[1, i], [i, -1]] equals its transpose but is not normal (H H^* != H^* H); [[1, i], [i, 1]]
    is normal without being Hermitian."""
    assert not O.is_normal(sp.csr_matrix(np.array([[1, 1j], [1j, -1]])))
    assert O.is_normal(sp.csr_matrix(np.array([[1, 1j], [1j, 1]])))


def test_real_input_takes_the_real_path_exactly():
    """A real matrix stored as complex gives the real oracle's result bit for bit (zero imaginary
    parts) and the same thresholds."""
    L = dirichlet_laplacian(10, 2).to_scipy()
    Er, sr = O.expm(L, 1e-3, 1e-12)
    Ec, sc = O.expm(sp.csr_matrix(L.astype(np.complex128)), 1e-3, 1e-12)
    assert (sr.M, sr.N) == (sc.M, sc.N)
    assert [s.t for s in sr.steps] == [s.t for s in sc.steps]
    assert np.array_equal(Er.indptr, Ec.indptr) and np.array_equal(Er.indices, Ec.indices)
    assert np.array_equal(Er.data, Ec.data.real) and not Ec.data.imag.any()


def test_pins_catch_filtering_by_the_real_part(monkeypatch):
    """A filter that compared the real part instead of the modulus would drop 3+4i."""
    real_abs = np.abs

    def wrong_abs(x, *a, **k):
        x = np.asarray(x)
        return real_abs(x.real, *a, **k) if np.iscomplexobj(x) else real_abs(x, *a, **k)

    monkeypatch.setattr(O.np, "abs", wrong_abs)
    t, iters, b = O.alg41_threshold(np.array([3 + 4j, 4.5 + 0j, 0.1j]), 4.8, 0.1)
    assert (t, iters) != (4.8, 1) or abs(b * b - 20.26) > 1e-13
