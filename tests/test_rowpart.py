"""Row-partitioned squaring (paper_2110_04493_gb300.rowpart): the multi-rank logic on CPU ranks
(gloo, 127.0.0.1) against the single-process oracle.

Each rank owns a contiguous row block balanced by product work, exchanges the halo rows its
products read, all-reduces Algorithm 4.1's partial sums (and the partial ||I + T~||_F), and
keeps its filtered block.  On CPU ranks the local arithmetic is plain scipy (test code); the
GPU test runs the same driver on one rank with the library's kernels."""
import math
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import sexpm_oracle as O
from paper_2110_04493_gb300 import rowpart as R
from tests._compare import expm_parity
from workloads import dirichlet_laplacian, diag_scale


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class ScipyOps(R.LocalOps):
    """Local arithmetic in scipy (CPU ranks of the test)."""

    def __init__(self, n):
        self.n = n

    def _m(self, X):
        return sp.csr_matrix((X[2], X[1], X[0]), shape=(self.n, self.n))

    @staticmethod
    def _t(M):
        M = sp.csr_matrix(M)
        M.sum_duplicates()
        M.sort_indices()
        return M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64)

    def product(self, A, B):
        Am, Bm = self._m(A), self._m(B)
        return self._t(Am @ Bm + 2.0 * Am)

    def norm2_I_plus_rows(self, X, r0, r1):
        M = self._m(X)[r0:r1].tocoo()
        d = M.row + r0 == M.col
        return float(np.sum(M.data ** 2) + (r1 - r0) + 2.0 * np.sum(M.data[d]))

    def pass_sum(self, X, t):
        v = X[2]
        return float(np.sum(v[np.abs(v) <= t] ** 2))

    def apply(self, X, t):
        M = self._m(X).copy()
        M.data = np.where(np.abs(M.data) > t, M.data, 0.0)
        M.eliminate_zeros()
        return self._t(M)


def _case(kind):
    if kind == "grid":
        H = dirichlet_laplacian(14, 2)
        tau = 2.253 / 15 ** 2
    else:
        H, _ = diag_scale(dirichlet_laplacian(7, 3), seed=2)
        tau = 2.1125 / 8 ** 2
    Hs = H.to_scipy()
    Hs.data = Hs.data * tau
    normH, M, N, normal, a, r0, eps_g0 = O.plan_scalars(Hs, 1e-12)
    H0 = Hs.copy()
    H0.data = np.ldexp(H0.data, -N)
    T0, _, _ = O.taylor_phase(H0, M, eps_g0, 0.1)
    return T0, N, a, r0


# ------------------------------------------------------------------ host helpers

def test_balanced_row_blocks_split_the_work_evenly():
    work = np.array([5, 1, 1, 1, 8, 0, 0, 2, 2, 4], dtype=np.int64)
    b = R.balanced_row_blocks(work, 3)
    assert b[0] == 0 and b[-1] == len(work) and np.all(np.diff(b) >= 0)
    shares = [work[b[r]:b[r + 1]].sum() for r in range(3)]
    assert sum(shares) == work.sum() and max(shares) <= 11
    assert list(R.balanced_row_blocks(np.zeros(4, dtype=np.int64), 2)) == [0, 0, 4]
    assert list(R.balanced_row_blocks(np.ones(3, dtype=np.int64), 5))[-1] == 3


def test_row_work_counts_the_products_of_each_row():
    A = sp.random(30, 30, density=0.15, random_state=np.random.RandomState(1), format="csr")
    A.sort_indices()
    got = R.row_work(A.indptr, A.indices)
    lens = np.diff(A.indptr)
    want = np.array([lens[A.indices[A.indptr[i]:A.indptr[i + 1]]].sum() for i in range(30)])
    assert np.array_equal(got, want)


def test_halo_rows_and_owners():
    A = sp.csr_matrix(np.array([[1, 0, 0, 1], [0, 1, 1, 0], [1, 1, 1, 0], [0, 0, 1, 1]], dtype=float))
    blk = R.matrix_rows(4, 1, 3, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data)
    assert list(R.halo_rows(blk)) == [0]
    bounds = np.array([0, 1, 3, 4])
    assert list(R.owner_of(np.array([0, 1, 2, 3]), bounds)) == [0, 1, 1, 2]
    req = R.split_requests(np.array([0, 3]), bounds, 3)
    assert [list(r) for r in req] == [[0], [], [3]]


def test_assemble_operand_places_own_and_halo_rows():
    A = sp.random(12, 12, density=0.3, random_state=np.random.RandomState(2), format="csr")
    A.sort_indices()
    rp, ci, v = A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data
    blk = R.matrix_rows(12, 4, 8, rp, ci, v)
    halo = R.halo_rows(blk)
    full = R.matrix_rows(12, 0, 12, rp, ci, v)
    lens, hc, hv = R.rows_of_block(full, halo)
    Brp, Bc, Bv = R.assemble_operand(blk, [(halo, lens, hc, hv)])
    B = sp.csr_matrix((Bv, Bc, Brp), shape=(12, 12)).toarray()
    want = A.toarray()
    keep = np.zeros(12, bool)
    keep[4:8] = True
    keep[halo] = True
    want[~keep] = 0.0
    assert np.array_equal(B, want)
    Arp, Ac, Av = R.block_as_matrix(blk)
    Ab = sp.csr_matrix((Av, Ac, Arp), shape=(12, 12)).toarray()
    want2 = np.zeros((12, 12))
    want2[4:8] = A.toarray()[4:8]
    assert np.array_equal(Ab, want2)


# ------------------------------------------------------------------ gloo ranks

def _rank_main(rank, world, port, kind, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        T0, N, a, r0 = _case(kind)
        T0 = sp.csr_matrix(T0)
        n = T0.shape[0]
        rp, ci, v = T0.indptr.astype(np.int64), T0.indices.astype(np.int32), T0.data.astype(np.float64)
        infos = []
        ops = ScipyOps(n)
        for k in range(1, N + 1):
            bounds = R.balanced_row_blocks(R.row_work(rp, ci), world)
            blk = R.matrix_rows(n, int(bounds[rank]), int(bounds[rank + 1]), rp, ci, v)
            blk, info = R.square_step(blk, bounds, k, a, r0, 0.1, ops)
            infos.append(info)
            rp, ci, v = R.gather_blocks(blk)
        if rank == 0:
            np.savez(os.path.join(out_dir, "out.npz"), rp=rp, ci=ci, v=v,
                     t=np.array([x["t"] for x in infos]), it=np.array([x["iters"] for x in infos]),
                     nnz=np.array([x["nnz"] for x in infos]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,world", [("grid", 2), ("grid", 3), ("dl3d", 2)])
def test_row_partitioned_squarings_match_the_oracle(tmp_path, kind, world):
    """N squarings on `world` gloo ranks (blocks rebalanced every step) give the oracle's
    single-process T^_N: same pass counts and kept counts, thresholds within rounding, values at
    the parity bar."""
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), kind, str(tmp_path)), nprocs=world, join=True)
    d = np.load(tmp_path / "out.npz")
    T0, N, a, r0 = _case(kind)
    T, steps, _ = O.squaring_phase(T0, N, a, r0, 0.1)
    n = T.shape[0]
    G = sp.csr_matrix((d["v"], d["ci"], d["rp"]), shape=(n, n))
    assert list(d["it"]) == [s.iters for s in steps]
    for t, s in zip(d["t"], steps):
        assert t == pytest.approx(s.t, rel=1e-12)
    expm_parity(G + sp.identity(n), sp.csr_matrix(T) + sp.identity(n), max(s.t for s in steps))


@pytest.mark.gpu
def test_row_partitioned_squaring_with_library_kernels_one_rank():
    """The same driver on one rank with the local arithmetic in libsexpm's kernels
    (sexpm_spgemm, sexpm_norm2_I_plus_rows, sexpm_filter_pass, sexpm_filter_apply)."""
    import torch.distributed as dist
    from paper_2110_04493_gb300 import build as B
    B.build()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        T0, N, a, r0 = _case("grid")
        T0 = sp.csr_matrix(T0)
        n = T0.shape[0]
        rp, ci, v = T0.indptr.astype(np.int64), T0.indices.astype(np.int32), T0.data.astype(np.float64)
        ops = R.LibraryOps(n)
        for k in range(1, N + 1):
            bounds = np.array([0, n])
            blk, info = R.square_step(R.matrix_rows(n, 0, n, rp, ci, v), bounds, k, a, r0, 0.1, ops)
            rp, ci, v = R.gather_blocks(blk)
    finally:
        dist.destroy_process_group()
    T, steps, _ = O.squaring_phase(T0, N, a, r0, 0.1)
    G = sp.csr_matrix((v, ci, rp), shape=(n, n))
    expm_parity(G + sp.identity(n), sp.csr_matrix(T) + sp.identity(n), max(s.t for s in steps))
