"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: exact equality for the integer choices (M, N, normality) and the pattern of
sparse products; element-wise |GPU - oracle| <= 1e-12 ||e^H||_1 for e^{tau H};
entries stored by only one side must lie within a factor 2 of the drop threshold.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sexpm_oracle as O
from tests._compare import expm_parity, to_scipy, torch_csr
from workloads import (
    CSR,
    diag_scale,
    dirichlet_laplacian,
    get_config,
    paper_table1_matrices,
    random_csr,
    rgg_adjacency,
    toeplitz_trid,
)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


def _csr(M) -> CSR:
    return CSR.from_scipy(sp.csr_matrix(M))


# ------------------------------------------------------------------ the sparse product

def _sprand(n, per_row, seed):
    """About per_row uniformly placed U[0,1) entries per row (seeded; duplicates summed)."""
    rng = np.random.default_rng(seed)
    k = max(1, int(round(per_row * n)))
    A = sp.csr_matrix((rng.uniform(0.0, 1.0, k), (rng.integers(0, n, k), rng.integers(0, n, k))), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A


def _ragged(n, seed, dense_rows=(), empty_rows=(), dense_size=3000):
    rng = np.random.default_rng(seed + 1000)
    A = _sprand(n, min(6.0, n), seed).tolil()
    for r in dense_rows:
        cols = rng.choice(n, size=min(n, dense_size), replace=False)
        A[r, cols] = rng.uniform(-1, 1, size=len(cols))
    for r in empty_rows:
        A[r, :] = 0
    A = sp.csr_matrix(A)
    A.eliminate_zeros()
    A.sort_indices()
    return A


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (300, 2), (5000, 3)])
def test_spgemm_taylor_term_matches_scipy(sx, n, seed):
    """S~ = S H_0 / i with a thin right operand (Eq. 4.10)."""
    S = _ragged(n, seed, empty_rows=[0] if n > 1 else [])
    H0 = _ragged(n, seed + 100)
    (rp, ci, v), prod = sx.spgemm(torch_csr(_csr(S)), torch_csr(_csr(H0)), div=7.0)
    G = to_scipy(rp, ci, v, n)
    R = (S @ H0).tocsr()
    R.data = R.data / 7.0
    assert prod == int(sum(np.diff(H0.indptr)[S.indices]))
    _assert_product_parity(G, R)


@pytest.mark.parametrize("n,seed,dense", [(64, 4, ()), (2000, 5, (3, 1500)), (40000, 6, (17, 20000, 39999))])
def test_spgemm_squaring_matches_scipy(sx, n, seed, dense):
    """T~ = 2T + T T (Eq. 4.15), including rows wide enough for the global-scratch class (rows of
    30000 entries make product rows of nearly all 40000 columns: 320 KB of accumulators)."""
    T = _ragged(n, seed, dense_rows=dense, empty_rows=[1], dense_size=30000)
    tt = torch_csr(_csr(T))
    (rp, ci, v), prod = sx.spgemm(tt, tt, tt, div=1.0, beta=2.0)
    G = to_scipy(rp, ci, v, n)
    R = O.square_raw(T)
    _assert_product_parity(G, R)


def _assert_product_parity(G, R):
    G.sort_indices()
    # every stored entry of the oracle is stored by the GPU; extra GPU entries are exact zeros
    Gp = sp.csr_matrix((np.ones(G.nnz), G.indices, G.indptr), shape=G.shape)
    Rp = sp.csr_matrix((np.ones(R.nnz), R.indices, R.indptr), shape=R.shape)
    assert (Rp - Rp.multiply(Gp)).nnz == 0
    extra = (Gp - Gp.multiply(Rp)).tocoo()
    if extra.nnz:
        assert np.all(np.asarray(G[extra.row, extra.col]).ravel() == 0.0)
    D = (G - R)
    scale = np.abs(R).max() if R.nnz else 1.0
    assert (np.abs(D.data).max() if D.nnz else 0.0) <= 1e-13 * max(scale, 1e-300)
    # rows are sorted with unique columns
    for i in range(0, G.shape[0], max(1, G.shape[0] // 50)):
        c = G.indices[G.indptr[i]:G.indptr[i + 1]]
        assert np.all(np.diff(c) > 0)


# ------------------------------------------------------------------ Algorithm 4.1

@pytest.mark.parametrize("seed", range(4))
def test_filter_matches_oracle(sx, seed):
    rng = np.random.default_rng(seed)
    n = [50, 400, 3000, 20000][seed]
    A = _sprand(n, min(30.0, n), seed)
    A.data = rng.standard_normal(A.nnz) * np.exp(rng.uniform(-45, 0, A.nnz))
    eps_g = float(np.exp(rng.uniform(-35, -15)))
    (rp, ci, v), t, iters, b = sx.filter_csr(torch_csr(_csr(A)), eps_g, 0.1)
    t_o, it_o, b_o = O.alg41_threshold(A.data, eps_g, 0.1)
    assert iters == it_o
    assert t == pytest.approx(t_o, rel=1e-12)
    assert b == pytest.approx(b_o, rel=1e-12)
    G = to_scipy(rp, ci, v, n)
    keep = np.abs(A.data) > t_o
    near = np.abs(np.abs(A.data) - t_o) <= 1e-12 * t_o
    Rk = A.copy(); Rk.data = np.where(keep, Rk.data, 0.0); Rk.eliminate_zeros()
    diff = (G - Rk).tocsr()
    assert diff.nnz == 0 or near.any()


def test_filter_hand_trace(sx):
    """Algorithm 4.1 on 1,2,3,4 with eps_g=3: two passes, t = 9/sqrt(14), keeps {3, 4}."""
    A = sp.csr_matrix(np.array([[1.0, -2.0], [3.0, 4.0]]))
    (rp, ci, v), t, iters, b = sx.filter_csr(torch_csr(_csr(A)), 3.0, 0.1)
    assert iters == 2 and t == pytest.approx(9 / math.sqrt(14))
    assert to_scipy(rp, ci, v, 2).toarray().tolist() == [[0.0, 0.0], [3.0, 4.0]]


# ------------------------------------------------------------------ the whole method

def _run_both(sx, H: CSR, tau, eps, **opts):
    (rp, ci, v), st = sx.expm(torch_csr(H), tau, eps, **opts)
    G = to_scipy(rp, ci, v, H.n)
    kw = {}
    if opts.get("square_scale", 1) == 0:
        kw["square_scale"] = "abs"
    E, so = O.expm(H.to_scipy(), tau, eps, **kw)
    return G, st, E, so


def _t_drop(st, so):
    ts = [r["t"] for r in st["steps"]] + [s.t for s in so.steps] + [t.t for t in so.taylor]
    return max(ts) if ts else 0.0


def _check_method(sx, H, tau, eps, **opts):
    G, st, E, so = _run_both(sx, H, tau, eps, **opts)
    assert (st["M"], st["N"]) == (so.M, so.N)
    assert bool(st["normal"]) == bool(so.normal)
    assert st["norm_H"] == pytest.approx(so.normH, rel=1e-13)
    if so.M:
        assert st["a"] == pytest.approx(so.a, rel=1e-14)
        assert st["r0"] == pytest.approx(so.r0, rel=1e-12)
    res = expm_parity(G, E, _t_drop(st, so))
    return res, st, so


@pytest.mark.parametrize("symmetric", [1, 0])
def test_expm_config_small_grid(sx, symmetric):
    """The 32x32 grid (n = 1024), with and without the symmetric (upper-triangle) products."""
    c = get_config("lap2d_m32")
    res, st, so = _check_method(sx, c.build(), c.tau, c.eps, symmetric=symmetric)
    assert st["symmetric"] == symmetric
    # the per-step record: same number of squarings, kept counts within the flip allowance
    sq = [r for r in st["steps"] if r["phase"] == 1]
    assert len(sq) == so.N
    for r, s in zip(sq, so.steps):
        assert r["nnz"] == pytest.approx(s.nnz, rel=2e-3)
        assert r["eps_g"] == pytest.approx(s.eps_g, rel=1e-10)


@pytest.mark.parametrize("symmetric", [1, 0])
def test_expm_paper_toeplitz(sx, symmetric):
    H = toeplitz_trid(10_000, 1.0, -2.0, 1.0)
    res, st, so = _check_method(sx, H, 1.0, 1e-16, symmetric=symmetric)
    assert (st["M"], st["N"]) == (20, 8)


def test_expm_heat_toeplitz(sx):
    n = 10_000
    H = toeplitz_trid(n, -1.0 / (n + 1), 2.0 / (n + 1), -1.0 / (n + 1))
    _check_method(sx, H, 1.0, 1e-16)


def test_expm_3d_grid_and_nonnormal_variant(sx):
    L = dirichlet_laplacian(12, 3)
    tau = 2.1125 / 13 ** 2
    _check_method(sx, L, tau, 1e-12)
    DL, _ = diag_scale(L, seed=1)
    res, st, so = _check_method(sx, DL, tau, 1e-12)
    assert not st["normal"] and not st["symmetric"]


def test_expm_absolute_threshold_option(sx):
    c = get_config("lap2d_m32")
    _check_method(sx, c.build(), c.tau, c.eps, square_scale=0)


def test_expm_random_graph(sx):
    A = rgg_adjacency(3000, seed=7)
    _check_method(sx, A, 0.5, 1e-12)


@pytest.mark.parametrize("k", range(5))
def test_expm_paper_table1(sx, k):
    H = CSR.from_dense(paper_table1_matrices()[k])
    _check_method(sx, H, 1.0, 1e-16)


def test_expm_edge_cases(sx):
    # n = 1 scalar exponential
    H = CSR.from_dense([[-3.5]])
    res, st, so = _check_method(sx, H, 0.7, 1e-14)
    # zero matrix (explicitly stored zeros) -> identity
    Z = CSR(3, np.array([0, 1, 1, 2], dtype=np.int64), np.array([1, 2], dtype=np.int32), np.zeros(2))
    (rp, ci, v), st = sx.expm(torch_csr(Z), 1.0, 1e-12)
    assert (st["M"], st["N"]) == (0, 0)
    assert np.array_equal(to_scipy(rp, ci, v, 3).toarray(), np.eye(3))
    # empty rows and a ragged random matrix
    R = random_csr(700, 0.004, seed=9, scale=3.0)
    _check_method(sx, R, 1.0, 1e-12)


def test_expm_rejects_invalid_input(sx):
    bad = CSR(2, np.array([0, 2, 3], dtype=np.int64), np.array([1, 0, 1], dtype=np.int32), np.ones(3))
    with pytest.raises(sx.SexpmError) as ei:
        sx.expm(torch_csr(bad), 1.0, 1e-12)
    assert ei.value.code == -1
    nanm = CSR(1, np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([np.nan]))
    with pytest.raises(sx.SexpmError):
        sx.expm(torch_csr(nanm), 1.0, 1e-12)
    with pytest.raises(sx.SexpmError):
        sx.expm(torch_csr(CSR.from_dense([[1.0]])), 1.0, 0.0)


def test_row_schedule_does_not_change_results(sx):
    """The strip schedule of grid-numbered matrices only reorders work: results are identical."""
    H = dirichlet_laplacian(80, 2)
    tau = 2.253 / 81 ** 2
    (a_rp, a_ci, a_v), st1 = sx.expm(torch_csr(H), tau, 1e-12, row_order=1)
    (b_rp, b_ci, b_v), st0 = sx.expm(torch_csr(H), tau, 1e-12, row_order=0)
    assert np.array_equal(a_rp.cpu().numpy(), b_rp.cpu().numpy())
    assert np.array_equal(a_ci.cpu().numpy(), b_ci.cpu().numpy())
    assert np.array_equal(a_v.cpu().numpy(), b_v.cpu().numpy())


@pytest.mark.parametrize("ks_bytes", ["0", "32768", "1048576"])
def test_accumulation_modes_match_oracle(sx, monkeypatch, ks_bytes):
    """The accumulation layouts of the numeric pass against the oracle: pure column split
    (SEXPM_KSPLIT_BYTES=0), groups of 1, 2, 4 or 8 k-splitting members chosen row by row (a
    32 KB per-SM budget), and the pure k split wherever it fits (a 1 MB budget); on products
    with long rows (the k split's upper-mode search) and on the method, symmetric and not."""
    monkeypatch.setenv("SEXPM_KSPLIT_BYTES", ks_bytes)
    T = _ragged(2000, 21, dense_rows=(5, 1999), empty_rows=[2])
    tt = torch_csr(_csr(T))
    (rp, ci, v), _ = sx.spgemm(tt, tt, tt, div=1.0, beta=2.0)
    _assert_product_parity(to_scipy(rp, ci, v, 2000), O.square_raw(T))
    H = dirichlet_laplacian(40, 2)
    _check_method(sx, H, 2.253 / 41 ** 2, 1e-12, symmetric=1)
    _check_method(sx, H, 2.253 / 41 ** 2, 1e-12, symmetric=0)


def test_expm_takes_and_returns_torch_sparse_csr(sx):
    """sexpm.expm on a torch.sparse_csr tensor returns e^{tau H} as one, identical to the result
    of the (row_ptr, col, val) path."""
    import warnings
    import torch
    H = dirichlet_laplacian(16, 2)
    tau = 2.253 / 17 ** 2
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        Hs = torch.sparse_csr_tensor(torch.from_numpy(H.row_ptr.astype(np.int64)),
                                     torch.from_numpy(H.col.astype(np.int64)),
                                     torch.from_numpy(H.val.astype(np.float64)), size=(H.n, H.n)).cuda()
        E, st = sx.expm(Hs, tau, 1e-12)
        assert E.layout == torch.sparse_csr and tuple(E.shape) == (H.n, H.n)
        (rp, ci, v), _ = sx.expm(torch_csr(H), tau, 1e-12)
        assert torch.equal(E.crow_indices().cpu(), rp.cpu())
        assert torch.equal(E.col_indices().cpu(), ci.cpu().to(torch.int64))
        assert torch.equal(E.values().cpu(), v.cpu())


# ------------------------------------------------------------------ chunked squaring

def _chunk_case(variant):
    if variant.startswith("lap3d"):
        H = dirichlet_laplacian(12, 3)
        if variant.endswith("DL"):
            H, _ = diag_scale(H, seed=1)
        return H, 2.1125 / 13 ** 2, 1e-12
    c = get_config("lap2d_m32")
    return c.build(), c.tau, c.eps


@pytest.mark.parametrize("variant", ["lap3d", "lap3d_DL", "lap2d"])
def test_chunked_squaring_matches_oracle(sx, variant):
    """Squaring products formed in row chunks of at most 64 KB with Algorithm 4.1 streamed exactly
    (entries below eps_g / (2 sqrt(nnz)) folded into one sum of squares): the 3-D grid (symmetric
    mode, lower entries from earlier chunks' pieces), its non-normal D L variant (every entry
    formed) and the 2-D grid, at the same parity bar against the oracle as the whole products."""
    H, tau, eps = _chunk_case(variant)
    res, st, so = _check_method(sx, H, tau, eps, chunk_bytes=65536)
    sq = [r for r in st["steps"] if r["phase"] == 1]
    assert max(r["chunks"] for r in sq) > 4
    for r in sq:
        if r["chunks"] > 1:
            assert r["nnz"] <= r["nnz_stream"] <= r["nnz_raw"]
    # the same decisions as the whole product up to the rounding of the sums: equal pass counts,
    # thresholds within 1e-12 relative
    (rp, ci, v), st_w = sx.expm(torch_csr(H), tau, eps)
    for a, b in zip([r for r in st_w["steps"] if r["phase"] == 1], sq):
        assert a["iters"] == b["iters"] and a["t"] == pytest.approx(b["t"], rel=1e-12)
        assert a["nnz_raw"] == b["nnz_raw"]


def test_spgemm_reaches_every_size_class(sx):
    """The wide-row product of the squaring test really runs rows in the global-memory class (and in
    the shared-memory classes): per-class row counts from the step record of sexpm_spgemm."""
    T = _ragged(40000, 6, dense_rows=(17, 20000, 39999), empty_rows=[1], dense_size=30000)
    tt = torch_csr(_csr(T))
    rows = sx.spgemm_rows_per_class(tt, tt, tt, div=1.0, beta=2.0)
    assert rows[5] >= 1, rows          # global-memory accumulators
    assert rows[0] > 0, rows
    assert 39000 < sum(rows) <= 40000, rows  # every non-empty product row is in exactly one class


# ------------------------------------------------------------------ structural vibration (Eq. 2.1-2.2)

def test_expm_structural_vibration_theta(sx):
    """H = Theta dt for a damped 12 x 12 spring lattice (Rayleigh C = 0.02 M + 0.01 K): non-normal and
    non-symmetric (a = 1/||H||_F, every product entry formed), at the parity bar against the oracle."""
    from workloads import theta_lattice
    H = theta_lattice(12, 2, seed=4, dt=0.7, alpha=0.02, beta=0.01)
    res, st, so = _check_method(sx, H, 1.0, 1e-12)
    assert not st["normal"] and not st["symmetric"]


def test_expm_theta_chain_closed_form(sx):
    """The undamped chain's propagator against its closed form (cos/sin of (K/m)^(1/2) dt)."""
    from tests.test_oracle_pins import _chain_exact, _chain_theta
    m, k, m0, dt = 40, 1.3, 0.7, 0.9
    H = _chain_theta(m, k, m0, dt)
    (rp, ci, v), st = sx.expm(torch_csr(_csr(H)), 1.0, 1e-14)
    G = to_scipy(rp, ci, v, 2 * m).toarray()
    X = _chain_exact(m, k, m0, dt)
    assert np.abs(G - X).max() <= 1e-12 * np.abs(X).sum(axis=0).max()


# ------------------------------------------------------------------ refined norm (Sec. 4.2, Eq. 4.9)

def test_power_norms_match_the_oracle(sx):
    """||H^k||_F, k = 1..41, from the GPU's sparse powers against scipy's."""
    H = dirichlet_laplacian(20, 2)
    Hs = H.to_scipy() * (2.253 / 21 ** 2)
    Hd = CSR.from_scipy(Hs)
    got = sx.power_norms(torch_csr(Hd), 41)
    ref = O.power_norms(Hs, 41)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("case", ["toeplitz", "grid"])
def test_refined_scaling_matches_oracle(sx, case):
    """scaling = 1: (M, N) from the refined norm h_{M,N} (fewer squarings than Eq. 4.20 on the
    F-norm), r_0 = rho(M, h), the rest of Algorithm 4.2 unchanged; same (M, N) as the oracle's
    reading and the parity bar on e^{tau H}."""
    if case == "toeplitz":
        H, tau, eps = toeplitz_trid(10_000, 1.0, -2.0, 1.0), 1.0, 1e-16
    else:
        H, tau, eps = dirichlet_laplacian(30, 2), 2.253 / 31 ** 2, 1e-12
    (rp, ci, v), st = sx.expm(torch_csr(H), tau, eps, scaling=1)
    E, MN = O.expm_refined(H.to_scipy(), tau, eps)
    assert (st["M"], st["N"]) == MN
    assert st["N"] < O.choose_MN(O.fro_norm(H.to_scipy() * tau), eps)[1]
    ts = [r["t"] for r in st["steps"]]
    expm_parity(to_scipy(rp, ci, v, H.n), E, max(ts) if ts else 0.0)
