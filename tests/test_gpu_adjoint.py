"""Adjoint form: dL/dH through sexpm_adjoint (reverse pass with the filter masks frozen)
against the oracle's adjoint, checkpoint strides, finite differences of the GPU forward,
and the autograd wrapper."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sexpm_oracle as O
from tests._compare import to_scipy, torch_csr
from workloads import CSR, dirichlet_laplacian, rgg_adjacency

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


def _cases():
    A = sp.random(40, 40, density=0.1, random_state=np.random.RandomState(3), format="csr")
    Q = (A - sp.diags(np.asarray(A.sum(axis=1)).ravel())).tocsr()
    return {
        "grid": (dirichlet_laplacian(9, 2), 4e-3),
        "graph": (rgg_adjacency(400, seed=5), 0.5),
        "nonsym": (CSR.from_scipy(Q), 0.8),
    }


def _W(n, seed, count=None):
    rng = np.random.default_rng(seed)
    k = count or 3 * n
    return CSR.from_scipy(sp.csr_matrix((rng.uniform(-1, 1, k), (rng.integers(0, n, k), rng.integers(0, n, k))),
                                        shape=(n, n)))


@pytest.mark.parametrize("case", ["grid", "graph", "nonsym"])
def test_adjoint_matches_oracle(sx, case):
    H, tau = _cases()[case]
    W = _W(H.n, 11)
    rp, ci, v = sx.adjoint(torch_csr(H), tau, 1e-12, torch_csr(W))
    G = to_scipy(rp, ci, v, H.n)
    Go, E, st, tr = O.adjoint(H.to_scipy(), tau, 1e-12, W.to_scipy())
    assert np.array_equal(G.indptr, H.row_ptr) and np.array_equal(G.indices, H.col)
    scale = max(abs(Go).max(), 1e-300)
    assert abs(G - Go).max() <= 1e-9 * scale


def test_adjoint_checkpoint_strides_agree(sx):
    H, tau = _cases()["grid"]
    W = _W(H.n, 12)
    outs = [sx.adjoint(torch_csr(H), tau, 1e-12, torch_csr(W), ckpt_stride=k) for k in (1, 0, 3)]
    for rp, ci, v in outs[1:]:
        assert np.array_equal(v.cpu().numpy(), outs[0][2].cpu().numpy())


def test_adjoint_against_finite_differences_of_the_gpu_forward(sx):
    """Central differences of L(H) = <W, e^{tau H}> computed by the GPU forward (filter live)."""
    H, tau = _cases()["graph"]
    W = _W(H.n, 13)
    Ws = W.to_scipy()
    rp, ci, v = sx.adjoint(torch_csr(H), tau, 1e-12, torch_csr(W))
    g = v.cpu().numpy()
    rng = np.random.default_rng(3)

    def loss(vals):
        Hx = CSR(H.n, H.row_ptr, H.col, vals)
        (erp, eci, ev), _ = sx.expm(torch_csr(Hx), tau, 1e-12, symmetric=0)
        return float(to_scipy(erp, eci, ev, H.n).multiply(Ws).sum())

    for p in rng.choice(H.nnz, size=8, replace=False):
        d = 1e-4 * abs(H.val[p])
        vp, vm = H.val.copy(), H.val.copy()
        vp[p] += d
        vm[p] -= d
        fd = (loss(vp) - loss(vm)) / (2 * d)
        assert g[p] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_autograd_function(sx):
    import torch
    H, tau = _cases()["nonsym"]
    W = _W(H.n, 14)
    rp, ci, hv = (torch.from_numpy(H.row_ptr).cuda(), torch.from_numpy(H.col).cuda(),
                  torch.from_numpy(H.val).cuda().requires_grad_(True))
    ev, erp, eci = sx.expm_autograd(hv, rp, ci, H.n, tau, 1e-12)
    # weights of W on the pattern of E, in E's storage order
    Wd = W.to_scipy().tocsr()
    erp_h = np.array(erp.cpu().numpy(), dtype=np.int64, copy=True)
    eci_h = np.array(eci.cpu().numpy(), dtype=np.int64, copy=True)
    rows = np.repeat(np.arange(H.n), np.diff(erp_h))
    w_on_E = torch.from_numpy(np.asarray(Wd[rows, eci_h]).ravel().copy()).cuda()
    loss = (ev * w_on_E).sum()
    loss.backward()
    Go, E, st, tr = O.adjoint(H.to_scipy(), tau, 1e-12, W.to_scipy())
    ref = np.asarray(Go[np.repeat(np.arange(H.n), np.diff(H.row_ptr)), np.array(H.col, dtype=np.int64)]).ravel()
    assert np.abs(hv.grad.cpu().numpy() - ref).max() <= 1e-9 * max(np.abs(ref).max(), 1e-300)


def test_forward_keep_tape_matches_adjoint(sx):
    """sexpm_forward_keep + sexpm_adjoint_tape return exactly what sexpm_adjoint returns (same
    forward, same checkpoints), and one kept forward serves two loss weights."""
    H, tau = _cases()["graph"]
    W1, W2 = _W(H.n, 21), _W(H.n, 22)
    plan = sx.Plan(torch_csr(H), 1e-12)
    try:
        tape, res = plan.forward_keep(tau)
        res.free()
        g1 = tape.adjoint(torch_csr(W1))
        g2 = tape.adjoint(torch_csr(W2))
        tape.free()
        r1 = sx.adjoint(plan, tau, 1e-12, torch_csr(W1))
        r2 = sx.adjoint(plan, tau, 1e-12, torch_csr(W2))
    finally:
        plan.close()
    for g, r in ((g1, r1), (g2, r2)):
        assert np.array_equal(g[0].cpu().numpy(), r[0].cpu().numpy())
        assert np.array_equal(g[2].cpu().numpy(), r[2].cpu().numpy())


def test_autograd_edge_parameterisation(sx):
    """SexpmFn in the edge form: H = beta A for the symmetric weighted adjacency A of a graph
    given by its edge list and one weight per edge; dL/dw_e = beta (dL/dH_uv + dL/dH_vu) against
    the oracle's adjoint."""
    import torch
    A = rgg_adjacency(500, seed=9)
    beta, tau = 0.5, 1.0
    Au = sp.triu(A.to_scipy(), 1).tocoo()
    edges = np.vstack([Au.row, Au.col])
    w = torch.from_numpy(Au.data.copy()).cuda().requires_grad_(True)
    ev, erp, eci = sx.expm_edges(w, edges, A.n, beta, tau, 1e-12)
    W = _W(A.n, 23)
    Wd = W.to_scipy().tocsr()
    erp_h = np.array(erp.cpu().numpy(), dtype=np.int64, copy=True)
    eci_h = np.array(eci.cpu().numpy(), dtype=np.int64, copy=True)
    rows = np.repeat(np.arange(A.n), np.diff(erp_h))
    w_on_E = torch.from_numpy(np.asarray(Wd[rows, eci_h]).ravel().copy()).cuda()
    (ev * w_on_E).sum().backward()
    Go, E, st, tr = O.adjoint(beta * A.to_scipy(), tau, 1e-12, W.to_scipy())
    Go = sp.csr_matrix(Go)
    ref = beta * (np.asarray(Go[Au.row, Au.col]).ravel() + np.asarray(Go[Au.col, Au.row]).ravel())
    got = w.grad.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-9 * max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("long_len", [5000, 30000])
def test_transpose_with_long_rows_matches_scipy(sx, long_len):
    """The transpose behind the reverse pass: rows of the result longer than the 4096 entries a
    block sorts in shared memory (a column of 5000 or 30000 entries) are merged from sorted runs;
    the result equals scipy's transpose entry for entry."""
    rng = np.random.default_rng(long_len)
    n = 40000
    # about 4 random entries per row (positions drawn independently; repeats are summed)
    br, bc = rng.integers(0, n, 4 * n), rng.integers(0, n, 4 * n)
    keep = (bc != 5) & (bc != 777)  # columns 5 and 777 are set below
    rows = rng.choice(n, size=long_len, replace=False)
    half = rows[:long_len // 2]
    r = np.concatenate([br[keep], rows, half])
    c = np.concatenate([bc[keep], np.full(long_len, 5), np.full(half.size, 777)])
    v = np.concatenate([rng.uniform(-1, 1, int(keep.sum())), rng.uniform(-1, 1, long_len),
                        rng.uniform(-1, 1, half.size)])
    A = sp.csr_matrix((v, (r, c)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    rp, ci, v = sx.transpose(torch_csr(CSR.from_scipy(A)))
    G = to_scipy(rp, ci, v, n)
    R = sp.csr_matrix(A.T)
    R.sort_indices()
    assert np.array_equal(G.indptr, R.indptr)
    assert np.array_equal(G.indices, R.indices)
    assert np.array_equal(G.data, R.data)
    assert np.diff(G.indptr).max() >= long_len
