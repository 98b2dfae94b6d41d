"""Pins of the oracle's adjoint (reverse pass of Algorithm 4.2 with the filter masks frozen)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import sexpm_oracle as O
from workloads import dirichlet_laplacian, rgg_adjacency


def _loss(E, W):
    return float(E.multiply(W).sum())


def _masks(tr):
    return [S.copy() for S in tr["S"]], [T.copy() for T in tr["T"]]


@pytest.mark.parametrize("case", ["grid", "graph", "nonsym"])
def test_adjoint_matches_central_differences_with_frozen_masks(case):
    rng = np.random.default_rng(7)
    if case == "grid":
        H, tau = dirichlet_laplacian(7, 2).to_scipy(), 4e-3
    elif case == "graph":
        H, tau = rgg_adjacency(150, seed=5).to_scipy(), 0.5
    else:
        A = sp.random(40, 40, density=0.1, random_state=np.random.RandomState(3), format="csr")
        H, tau = (A - sp.diags(np.asarray(A.sum(axis=1)).ravel())).tocsr(), 0.8
    n = H.shape[0]
    W = sp.csr_matrix((rng.uniform(-1, 1, 3 * n), (rng.integers(0, n, 3 * n), rng.integers(0, n, 3 * n))),
                      shape=(n, n))
    G, E, st, tr = O.adjoint(H, tau, 1e-12, W)
    Sm, Tm = _masks(tr)
    H = O._canon(H)
    for p in rng.choice(H.nnz, size=12, replace=False):
        d = 1e-5 * max(abs(H.data[p]), 1e-3)
        Hp, Hm = H.copy(), H.copy()
        Hp.data[p] += d
        Hm.data[p] -= d
        fd = (_loss(O.forward_frozen(Hp, tau, st.N, Sm, Tm), W) - _loss(O.forward_frozen(Hm, tau, st.N, Sm, Tm), W)) / (2 * d)
        r, c = np.searchsorted(H.indptr, p, side="right") - 1, H.indices[p]
        assert G[r, c] == pytest.approx(fd, rel=1e-6, abs=1e-9 * max(1.0, abs(fd)))


def test_forward_frozen_reproduces_the_filtered_result():
    H = dirichlet_laplacian(6, 2).to_scipy()
    G, E, st, tr = O.adjoint(H, 0.01, 1e-12, sp.identity(36, format="csr"))
    Sm, Tm = _masks(tr)
    E2 = O.forward_frozen(H, 0.01, st.N, Sm, Tm)
    assert abs(E - E2).max() <= 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_matches_block_frechet_identity(seed):
    """For L = <W, e^H>, dL/dH = L_exp(H^T, W), the upper-right block of
    exp([[H^T, W], [0, H^T]]); with a tolerance near u the filter drops almost nothing."""
    rng = np.random.default_rng(seed)
    n = 12
    H = sp.random(n, n, density=0.3, random_state=np.random.RandomState(seed), format="csr") * 2.0
    W = rng.uniform(-1, 1, (n, n))
    G, E, st, tr = O.adjoint(H, 1.0, 1e-16, sp.csr_matrix(W))
    Hd = H.toarray()
    Z = np.block([[Hd.T, W], [np.zeros((n, n)), Hd.T]])
    F = sla.expm(Z)[:n, n:]
    Hc = O._canon(H)
    rows = np.repeat(np.arange(n), np.diff(Hc.indptr))
    ref = F[rows, Hc.indices]
    got = np.asarray(G[rows, Hc.indices]).ravel()
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(F).max()


def test_adjoint_of_trace_is_transposed_exponential():
    """L = trace(e^H): dL/dH = (e^H)^T on the pattern of H."""
    H = (dirichlet_laplacian(5, 2).to_scipy() * 3e-3).tocsr()
    H = H + sp.triu(H, 1) * 0.3  # break the symmetry
    G, E, st, tr = O.adjoint(H, 1.0, 1e-15, sp.identity(25, format="csr"))
    Hc = O._canon(H)
    rows = np.repeat(np.arange(25), np.diff(Hc.indptr))
    Ed = sla.expm(Hc.toarray())
    assert np.abs(np.asarray(G[rows, Hc.indices]).ravel() - Ed.T[rows, Hc.indices]).max() <= 1e-10


def test_adjoint_pins_catch_a_missing_transpose(monkeypatch):
    """Planting Y T + T Y (transposes dropped) in the oracle's reverse pass breaks the
    finite-difference pin on a non-symmetric matrix."""
    monkeypatch.setattr(O, "square_adjoint", lambda Y, Tp: O.restrict(2.0 * Y + Y @ Tp + Tp @ Y, Tp))
    H = dirichlet_laplacian(5, 2).to_scipy()
    H = ((H + sp.triu(H, 1) * 0.5) * 5e-3).tocsr()
    W = sp.csr_matrix(np.random.default_rng(1).uniform(-1, 1, (25, 25)))
    G, E, st, tr = O.adjoint(H, 1.0, 1e-12, W)
    assert st.N > 0
    Sm, Tm = _masks(tr)
    Hc = O._canon(H)
    worst = 0.0
    for p in range(0, Hc.nnz, 7):
        d = 1e-5 * abs(Hc.data[p])
        Hp, Hm = Hc.copy(), Hc.copy()
        Hp.data[p] += d
        Hm.data[p] -= d
        fd = (_loss(O.forward_frozen(Hp, 1.0, st.N, Sm, Tm), W) - _loss(O.forward_frozen(Hm, 1.0, st.N, Sm, Tm), W)) / (2 * d)
        r, c = np.searchsorted(Hc.indptr, p, side="right") - 1, Hc.indices[p]
        worst = max(worst, abs(G[r, c] - fd) / max(abs(fd), 1e-12))
    assert worst > 1e-3


def test_oracle_adjoint_zero_branch_matches_first_order_term():
    """At ||tau H|| = 0 the oracle's adjoint returns tau W on the pattern of H (the first-order term
    of e^{tau H} = I + tau H + ...).  Pinned against central differences of the oracle's forward at
    H = 0 along each stored entry (diagonal and off-diagonal): e^{tau d E_ij} = I + tau d E_ij
    (i != j) or differs from I by e^{tau d} - 1 at (i, i)."""
    import scipy.sparse as sp
    n, tau, eps = 5, 0.7, 1e-14
    rows = np.array([0, 1, 2, 3, 4, 4])
    cols = np.array([0, 3, 2, 1, 0, 4])
    H0 = sp.csr_matrix((np.zeros(6), (rows, cols)), shape=(n, n))
    H0.sort_indices()
    rng = np.random.default_rng(4)
    W = sp.csr_matrix(rng.uniform(-1, 1, (n, n)))
    G, E, st, tr = O.adjoint(H0, tau, eps, W)
    G = sp.csr_matrix(G)
    d = 1e-6
    for i, j in zip(rows, cols):
        def loss(x):
            Hx = H0.copy().tolil()
            Hx[i, j] = x
            Ex, _ = O.expm(sp.csr_matrix(Hx), tau, eps)
            return float(sp.csr_matrix(Ex).multiply(W).sum())
        fd = (loss(d) - loss(-d)) / (2 * d)
        assert G[i, j] == pytest.approx(tau * W[i, j], rel=1e-14)
        assert fd == pytest.approx(G[i, j], rel=1e-8, abs=1e-12)
