"""Checks at the full sizes of the benchmark workloads, where the CPU oracle cannot run:
sampled outputs against closed forms, and e^H R against an independent time stepper."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from tests._compare import taylor_time_stepper, torch_csr
from workloads import CSR, dirichlet_laplacian, get_config, rgg_adjacency, sparse_loss_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


def _sine_basis_expm(m, tau):
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam = -(4.0 / h ** 2) * np.sin(j * np.pi * h / 2) ** 2
    V = np.sqrt(2 * h) * np.sin(np.outer(j, j) * np.pi * h)
    return (V * np.exp(tau * lam)) @ V.T


def _rows(rp, ci, v, rows):
    """Dense copies of the given rows of a device CSR (col, val) pairs."""
    rph = rp.cpu().numpy()
    out = []
    for i in rows:
        a, b = int(rph[i]), int(rph[i + 1])
        out.append((ci[a:b].cpu().numpy(), v[a:b].cpu().numpy()))
    return out


def test_lap2d_m1500_rows_match_kronecker_closed_form(sx):
    """The bench workload (n = 2.25M): 48 sampled full rows of e^{tau L} against
    e^{tau L_1} (x) e^{tau L_1} (1-D sine eigenbasis), max-abs <= 1e-12 ||e^H||_1 (<= 1e-12)."""
    c = get_config("lap2d_m1500")
    H = c.build()
    (rp, ci, v), st = sx.expm(torch_csr(H), c.tau, c.eps)
    m = 1500
    E1 = _sine_basis_expm(m, c.tau)
    rng = np.random.default_rng(5)
    rows = list(rng.integers(0, H.n, size=40)) + [0, m - 1, H.n - 1, H.n // 2, 37 * m + 3, 750 * m + 750, m * (m - 1), 1]
    for i, (cols, vals) in zip(rows, _rows(rp, ci, v, rows)):
        xi, yi = i % m, i // m
        exact = np.outer(E1[yi], E1[xi]).ravel()
        got = np.zeros(H.n)
        got[cols] = vals
        assert np.abs(got - exact).max() <= 1e-12, i
    assert (st["M"], st["N"]) == (18, 14)


def _free_cached():
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_lap3d_m64_rows_match_kronecker_closed_form(sx):
    """The 3-D workload at full size (64^3 grid, n = 262,144, tau = 5e-4, eps = 1e-12): its
    last unfiltered products do not fit in memory whole, so they are formed in row chunks with
    Algorithm 4.1 streamed exactly.  Sampled full rows against
    e^{tau L_1} (x) e^{tau L_1} (x) e^{tau L_1}, max-abs <= 1e-12 ||e^H||_1 (<= 1e-12)."""
    _free_cached()
    c = get_config("lap3d_m64")
    H = c.build()
    (rp, ci, v), st = sx.expm(torch_csr(H), c.tau, c.eps)
    m = 64
    E1 = _sine_basis_expm(m, c.tau)
    rng = np.random.default_rng(6)
    rows = list(rng.integers(0, H.n, size=40)) + [0, m - 1, H.n - 1, H.n // 2, 32 + 64 * 32 + 4096 * 32,
                                                   5 + 64 * 63 + 4096 * 10]
    for i, (cols, vals) in zip(rows, _rows(rp, ci, v, rows)):
        x, y, z = i % m, (i // m) % m, i // (m * m)
        exact = np.einsum("a,b,c->abc", E1[z], E1[y], E1[x]).ravel()
        got = np.zeros(H.n)
        got[cols] = vals
        assert np.abs(got - exact).max() <= 1e-12, i
    sq = [r for r in st["steps"] if r["phase"] == 1]
    print(f"lap3d_m64: M={st['M']} N={st['N']} nnz(e^H)={st['nnz_out']} peak={st['peak_bytes'] / 2**30:.1f} GiB "
          f"chunks={[r['chunks'] for r in sq]} ms={st['ms_total']:.0f}")
    del rp, ci, v
    _free_cached()


@pytest.mark.skipif(os.environ.get("SEXPM_FULLSIZE_DL") != "1",
                    reason="about 17 minutes on one GB300; run with SEXPM_FULLSIZE_DL=1")
def test_lap3d_m64_DL_rows_match_time_stepper(sx):
    """The non-normal variant D L at full size (every product entry formed, a = 1/||H||_F, the
    last squarings in row chunks): eight full rows e_j^T e^H (interior, face, edge and corner
    nodes) against a Taylor time stepper for e^{tau H^T} e_j on cuSPARSE products,
    element-wise <= 1e-12 max_j ||e_j^T e^H||_1 (a lower bound of ||e^H||_inf, the bar of the
    transposed problem)."""
    import torch
    _free_cached()
    c = get_config("lap3d_m64_DL")
    H = c.build()
    (rp, ci, v), st = sx.expm(torch_csr(H), c.tau, c.eps)
    assert not st["normal"] and not st["symmetric"]
    m = 64
    rows = [0, m - 1, m * m * m - 1, 32 + 64 * 32 + 4096 * 32, 7 + 64 * 50 + 4096 * 20, 64 * 64 * 31, 4096 * 63 + 5,
            int(np.random.default_rng(8).integers(0, H.n))]
    got = np.zeros((H.n, len(rows)))
    for k, (cols, vals) in enumerate(_rows(rp, ci, v, rows)):
        got[cols, k] = vals
    del rp, ci, v
    _free_cached()
    Ht_s = sp.csr_matrix(H.to_scipy().T)
    Ht_s.sort_indices()
    Ht = torch.sparse_csr_tensor(torch.from_numpy(Ht_s.indptr.astype(np.int64)).cuda(),
                                 torch.from_numpy(Ht_s.indices.astype(np.int64)).cuda(),
                                 torch.from_numpy(Ht_s.data * c.tau).cuda(), size=(H.n, H.n))
    R = torch.zeros(H.n, len(rows), dtype=torch.float64, device="cuda")
    for k, j in enumerate(rows):
        R[j, k] = 1.0
    Y = taylor_time_stepper(Ht, R, substeps=128).cpu().numpy()
    n1 = float(np.abs(Y).sum(axis=0).max())
    err = float(np.abs(got - Y).max())
    sq = [r for r in st["steps"] if r["phase"] == 1]
    print(f"lap3d_m64_DL: M={st['M']} N={st['N']} nnz(e^H)={st['nnz_out']} max-abs={err:.2e} "
          f"||rows||_1={n1:.3f} peak={st['peak_bytes'] / 2**30:.1f} GiB ms={st['ms_total']:.0f} "
          f"chunks={[r['chunks'] for r in sq]}")
    assert err <= 1e-12 * n1


def test_rgg_1e5_columns_match_time_stepper(sx):
    """The differentiation workload's forward (RGG n = 1e5, H = 0.5 A, eps = 1e-12): sixteen
    columns e^H e_j (through sexpm_result_spmm) element-wise against a Taylor time stepper built
    on cuSPARSE products (64 substeps, terms until they fall below 1e-20 of the running sum), at
    1e-12 max_j ||e^H e_j||_1 (a lower bound of ||e^H||_1); and e^H R for four random vectors."""
    import torch
    A = rgg_adjacency(100_000, seed=3)
    Hv = 0.5 * A.val
    Hd = (torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(), torch.from_numpy(Hv).cuda(), A.n)
    plan = sx.Plan(Hd, 1e-12)
    E = plan.compute(1.0)
    cols = np.random.default_rng(7).choice(A.n, size=16, replace=False)
    R = torch.zeros(A.n, 20, dtype=torch.float64, device="cuda")
    for k, j in enumerate(cols):
        R[j, k] = 1.0
    R[:, 16:] = torch.from_numpy(np.random.default_rng(7).uniform(-1, 1, (A.n, 4))).cuda()
    ER = E.spmm(R)
    E.free()
    plan.close()
    Ht = torch.sparse_csr_tensor(Hd[0], Hd[1].to(torch.int64), Hd[2], size=(A.n, A.n))
    Y = taylor_time_stepper(Ht, R, substeps=64)
    n1 = float(Y[:, :16].abs().sum(dim=0).max())
    err_cols = float((ER[:, :16] - Y[:, :16]).abs().max())
    err_R = float((ER[:, 16:] - Y[:, 16:]).abs().max() / Y[:, 16:].abs().max())
    print(f"rgg_1e5 forward: columns max-abs {err_cols:.2e} (||cols||_1 {n1:.3f}); e^H R rel {err_R:.2e}")
    assert err_cols <= 1e-12 * n1
    assert err_R <= 1e-12


def _gather_loss_fn(W, n):
    """L(E) = sum_ij W_ij E_ij for a device CSR E, by locating W's entries in E's sorted keys."""
    import torch
    Ws = W.to_scipy().tocoo()
    wk = torch.from_numpy(Ws.row.astype(np.int64) * n + Ws.col.astype(np.int64)).cuda()
    wv = torch.from_numpy(Ws.data.astype(np.float64)).cuda()

    def loss(rp, ci, v, absolute=False):
        rows = torch.repeat_interleave(torch.arange(n, device="cuda"), rp[1:] - rp[:-1])
        keys = rows * n + ci.to(torch.int64)
        pos = torch.searchsorted(keys, wk).clamp(max=keys.numel() - 1)
        hit = keys[pos] == wk
        vals = torch.where(hit, v[pos], torch.zeros_like(wv))
        return float((wv.abs() * vals.abs()).sum()) if absolute else float((wv * vals).sum())

    return loss


def test_rgg_1e5_adjoint_against_finite_differences(sx):
    """dL/dw_e = 0.5 (dL/dH_uv + dL/dH_vu) for L = <W, e^H> on the 1e5-node graph against central
    differences of the GPU forward on 64 random edges, each with its plain relative error
    |adjoint - fd| / |fd| <= 1e-6 (no floor).  A difference quotient resolves a gradient only
    above its rounding noise, about 2^-52 sum|W_ij E_ij| / delta; the 64 edges are drawn from the
    edges whose adjoint gradient is at least 1e6 times that noise (a 1e-6 relative check is
    meaningful there), and the share of edges below it is printed: W has 1e5 entries at random
    positions, so most edges lie too far from every one of them to have a resolvable gradient."""
    import torch
    A = rgg_adjacency(100_000, seed=3)
    n = A.n
    W = sparse_loss_weights(n, 100_000, seed=3)
    dev = lambda vals: (torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col).cuda(),
                        torch.from_numpy(vals).cuda(), n)
    rp, ci, g = sx.adjoint(dev(0.5 * A.val), 1.0, 1e-12, torch_csr(W))
    G = sp.csr_matrix((g.cpu().numpy(), A.col, A.row_ptr), shape=(n, n))
    gather = _gather_loss_fn(W, n)

    def loss(vals, absolute=False):
        plan = sx.Plan(dev(0.5 * vals), 1e-12)
        try:
            E = plan.compute(1.0)
            try:
                erp, eci, ev = E.to_torch()
            finally:
                E.free()
        finally:
            plan.close()
        return gather(erp, eci, ev, absolute)

    Au = sp.triu(A.to_scipy(), 1).tocoo()
    ge = 0.5 * (np.asarray(G[Au.row, Au.col]).ravel() + np.asarray(G[Au.col, Au.row]).ravel())
    delta = 1e-4 * Au.data
    noise = 2.0 ** -52 * loss(A.val, absolute=True) / delta
    ok = np.abs(ge) >= 1e6 * noise
    print(f"rgg_1e5 adjoint: {ok.sum()} of {len(ge)} edges have a gradient resolvable at 1e-6 by central "
          f"differences (max |dL/dw| = {np.abs(ge).max():.3e})")
    assert ok.sum() >= 64
    pick = np.random.default_rng(3).choice(np.flatnonzero(ok), size=64, replace=False)
    worst = 0.0
    for e in pick:
        u, w = int(Au.row[e]), int(Au.col[e])
        puw = A.row_ptr[u] + np.searchsorted(A.col[A.row_ptr[u]:A.row_ptr[u + 1]], w)
        pwu = A.row_ptr[w] + np.searchsorted(A.col[A.row_ptr[w]:A.row_ptr[w + 1]], u)
        d = delta[e]
        vp, vm = A.val.copy(), A.val.copy()
        vp[[puw, pwu]] += d
        vm[[puw, pwu]] -= d
        fd = (loss(vp) - loss(vm)) / (2 * d)
        rel = abs(ge[e] - fd) / abs(fd)
        worst = max(worst, rel)
        print(f"  edge ({u}, {w}): adjoint {ge[e]: .12e}  fd {fd: .12e}  rel {rel:.2e}")
        assert rel <= 1e-6, (u, w, ge[e], fd)
    print(f"  worst relative error over 64 edges: {worst:.2e}")


def _diag_of(rp, ci, v, n):
    """Diagonal of a device CSR (torch tensors), 0 where absent."""
    import torch
    rows = torch.repeat_interleave(torch.arange(n, dtype=torch.int32, device=rp.device), rp[1:] - rp[:-1])
    on = ci == rows
    d = torch.zeros(n, dtype=torch.float64, device=rp.device)
    d[rows[on].long()] = v[on]
    return d


def test_lap2d_m1500_adjoint_of_trace(sx):
    """The bench workload's adjoint (n = 2.25M): L = trace(P e^{tau H}) through one kept forward
    (sexpm_forward_keep, checkpoints every ceil(sqrt(N)) squarings) and two reverse passes.
    P = I: dL/dH = tau (e^{tau H})^T on the pattern of H, every stored entry against the Kronecker
    closed form.  P seeded diagonal (P_ii ~ U[0,1], seed 4): central differences of the GPU
    forward along two diagonal entries and two symmetric off-diagonal pairs, relative error
    <= 1e-6 with no floor."""
    import torch
    from workloads import diag_weights
    _free_cached()
    c = get_config("lap2d_m1500")
    H = c.build()
    n, m = H.n, 1500
    plan = sx.Plan(torch_csr(H), c.eps)
    tape, res = plan.forward_keep(c.tau)
    st = res.stats()
    res.free()
    ar = lambda k, dt: torch.arange(k, dtype=dt, device="cuda")
    _, _, g_I = tape.adjoint((ar(n + 1, torch.int64), ar(n, torch.int32), torch.ones(n, dtype=torch.float64,
                                                                                     device="cuda"), n))
    P = diag_weights(n, seed=4)
    _, _, g_P = tape.adjoint((ar(n + 1, torch.int64), ar(n, torch.int32), torch.from_numpy(P).cuda(), n))
    live, peak = sx.pool_stats()
    tape.free()
    plan.close()
    g_I, g_P = g_I.cpu().numpy(), g_P.cpu().numpy()
    E1 = _sine_basis_expm(m, c.tau)
    rows = np.repeat(np.arange(n), np.diff(H.row_ptr))
    cols = H.col.astype(np.int64)
    exact = c.tau * E1[rows // m, cols // m] * E1[rows % m, cols % m]   # d trace(e^{tau H})/dH = tau (e^{tau H})^T
    err_I = float(np.abs(g_I - exact).max())
    print(f"adjoint trace: M={st['M']} N={st['N']} |dL/dH - (e^H)^T| max={err_I:.2e} "
          f"peak over forward+reverse={peak / 2**30:.1f} GiB")
    assert err_I <= 1e-11 * float(np.abs(exact).max())

    Pd = torch.from_numpy(P).cuda()

    def loss(vals):
        (erp, eci, ev), _ = sx.expm(torch_csr(CSR(n, H.row_ptr, H.col, vals)), c.tau, c.eps)
        out = float((_diag_of(erp, eci, ev, n) * Pd).sum())
        del erp, eci, ev
        _free_cached()
        return out

    rng = np.random.default_rng(12)
    picks = []
    for i in rng.integers(0, n, size=2):
        p = H.row_ptr[i] + np.searchsorted(H.col[H.row_ptr[i]:H.row_ptr[i + 1]], i)
        picks.append(("diag", [int(p)]))
    for i in rng.integers(m, n - m, size=2):
        p = H.row_ptr[i] + np.searchsorted(H.col[H.row_ptr[i]:H.row_ptr[i + 1]], i + m)
        q = H.row_ptr[i + m] + np.searchsorted(H.col[H.row_ptr[i + m]:H.row_ptr[i + m + 1]], i)
        picks.append(("pair", [int(p), int(q)]))
    for kind, ps in picks:
        d = 1e-4 * abs(H.val[ps[0]])  # the step in H (e^{tau H}: tau H moves by 1e-4 tau |H_p|)
        vp, vm = H.val.copy(), H.val.copy()
        for p in ps:
            vp[p] += d
            vm[p] -= d
        fd = (loss(vp) - loss(vm)) / (2 * d)
        ad = float(sum(g_P[p] for p in ps))
        rel = abs(ad - fd) / abs(fd)
        print(f"  FD {kind} entries {ps}: adjoint {ad:.12e} fd {fd:.12e} rel {rel:.2e}")
        assert rel <= 1e-6
