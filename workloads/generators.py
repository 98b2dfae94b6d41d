"""Seeded generators for the matrices the method is run on.

Every generator returns a :class:`CSR` with int64 row pointers, int32 sorted
unique column indices and float64 values.  Random draws use
``numpy.random.default_rng(seed)`` and nothing else, so both the GPU path and
the CPU oracle see bit-identical inputs.

Workloads (the paper's experiments use heat-conduction, structural and
network matrices, Sec. 5; the datasets themselves are not available, so
grid Laplacians and random geometric graphs of the same sizes stand in):

* ``dirichlet_laplacian(m, dim)`` - the negative-definite 5-/7-point Laplacian
  Delta_h on an m^dim grid with homogeneous Dirichlet boundary, h = 1/(m+1),
  lexicographic numbering x + m*y (+ m^2*z), i.e. L_2D = L_1 (+) L_1 as a
  Kronecker sum.
* ``toeplitz_trid(n, lo, d, up)`` - the paper's Toeplitz examples of Sec. 5.2.
* ``rgg_adjacency(n, ...)`` - symmetric weighted adjacency of a 2-D random
  geometric graph (spatial network stand-in).
* ``paper_table1_matrices()`` - the five small matrices of Sec. 5.1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Tuple

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class CSR:
    """Square sparse matrix in CSR form (int64 row_ptr, int32 col, float64 val)."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    @staticmethod
    def from_scipy(A) -> "CSR":
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        A.sort_indices()
        n = A.shape[0]
        assert A.shape == (n, n)
        return CSR(
            n,
            np.ascontiguousarray(A.indptr, dtype=np.int64),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64),
        )

    @staticmethod
    def from_dense(D) -> "CSR":
        D = np.asarray(D, dtype=np.float64)
        return CSR.from_scipy(sp.csr_matrix(D))


def toeplitz_trid(n: int, lower: float, diag: float, upper: float) -> CSR:
    """Tridiagonal Toeplitz matrix trid_n(lower, diag, upper)."""
    A = sp.diags([np.full(n - 1, lower), np.full(n, diag), np.full(n - 1, upper)], [-1, 0, 1], shape=(n, n), format="csr")
    return CSR.from_scipy(A)


def dirichlet_laplacian(m: int, dim: int) -> CSR:
    """Negative-definite finite-difference Laplacian on an m^dim Dirichlet grid.

    Diagonal -2*dim/h^2, each grid neighbour +1/h^2, h = 1/(m+1); node
    (x, y, z) has index x + m*y + m^2*z.
    """
    h = 1.0 / (m + 1)
    L1 = sp.diags([np.ones(m - 1), -2.0 * np.ones(m), np.ones(m - 1)], [-1, 0, 1], shape=(m, m), format="csr") / (h * h)
    I = sp.identity(m, format="csr")
    if dim == 1:
        L = L1
    elif dim == 2:
        L = sp.kron(I, L1) + sp.kron(L1, I)
    elif dim == 3:
        L = sp.kron(sp.kron(I, I), L1) + sp.kron(sp.kron(I, L1), I) + sp.kron(sp.kron(L1, I), I)
    else:
        raise ValueError("dim must be 1, 2 or 3")
    return CSR.from_scipy(L)


def diag_scale(A: CSR, seed: int, lo: float = 0.5, hi: float = 2.0) -> Tuple[CSR, np.ndarray]:
    """Return (D*A, d) with D = diag(d), d_i ~ U[lo, hi] from ``seed``."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(lo, hi, size=A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val * d[rows]), d


def rgg_adjacency(n: int, seed: int, mean_degree: float = 10.0, wlo: float = 0.5, whi: float = 1.5) -> CSR:
    """Symmetric weighted adjacency of a random geometric graph in the unit square.

    n points uniform in [0,1]^2, an edge between points closer than
    r = sqrt(mean_degree / (pi n)), weight ~ U[wlo, whi] per undirected edge.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    r = math.sqrt(mean_degree / (math.pi * n))
    pairs = np.array(sorted(cKDTree(pts).query_pairs(r)), dtype=np.int64).reshape(-1, 2)
    w = rng.uniform(wlo, whi, size=len(pairs))
    i = np.concatenate([pairs[:, 0], pairs[:, 1]])
    j = np.concatenate([pairs[:, 1], pairs[:, 0]])
    A = sp.csr_matrix((np.concatenate([w, w]), (i, j)), shape=(n, n))
    return CSR.from_scipy(A)


def random_csr(n: int, density: float, seed: int, symmetric: bool = False, scale: float = 1.0) -> CSR:
    """Random sparse matrix with ~density*n*n U[-scale, scale] entries (seeded)."""
    rng = np.random.default_rng(seed)
    nnz = max(1, int(round(density * n * n)))
    i = rng.integers(0, n, size=nnz)
    j = rng.integers(0, n, size=nnz)
    v = rng.uniform(-scale, scale, size=nnz)
    A = sp.csr_matrix((v, (i, j)), shape=(n, n))
    if symmetric:
        A = A + A.T
    return CSR.from_scipy(A)


def sparse_loss_weights(n: int, count: int, seed: int) -> CSR:
    """Loss weights W: ``count`` entries ~U[-1,1] at uniformly random (i, j), duplicates summed."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, size=count)
    j = rng.integers(0, n, size=count)
    v = rng.uniform(-1.0, 1.0, size=count)
    return CSR.from_scipy(sp.csr_matrix((v, (i, j)), shape=(n, n)))


def diag_weights(n: int, seed: int) -> np.ndarray:
    """Diagonal P with P_ii ~ U[0, 1]."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=n)


def batch_instances(count: int, seed: int, side_lo: int = 16, side_hi: int = 128,
                    tau_lo: float = 1e-4, tau_hi: float = 1e-2) -> List[Tuple[int, float]]:
    """(side, tau) pairs: side ~ U{side_lo..side_hi}, tau log-uniform in [tau_lo, tau_hi]."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    taus = np.exp(rng.uniform(math.log(tau_lo), math.log(tau_hi), size=count))
    return [(int(s), float(t)) for s, t in zip(sides, taus)]


def paper_table1_matrices() -> List[np.ndarray]:
    """The five small ill-conditioned test matrices of Sec. 5.1 (Table 1)."""
    H1 = np.array([[6.1, 1e6], [0.0, 6.1]])
    H2 = np.array([[1.0, 1e6, 0.5e12], [0.0, 1.0, 1e6], [0.0, 0.0, 1.0]])
    H3 = np.array([[1.0, math.sqrt(3.0) * 1e6], [0.0, 0.9]])
    H4 = np.array([[-49.0, 24.0], [-64.0, 31.0]])
    H5 = np.array([[1.0 + 1e-5, 1.0], [0.0, 1.0 - 1e-5]])
    return [H1, H2, H3, H4, H5]


def spring_lattice(m: int, dim: int, seed: int, klo: float = 0.5, khi: float = 1.5, mlo: float = 0.5,
                   mhi: float = 2.0) -> Tuple[sp.csr_matrix, np.ndarray]:
    """Stiffness K and lumped masses of an m^dim lattice of point masses joined to their grid
    neighbours by springs, with springs to fixed walls at the boundary (so K is SPD): spring
    stiffness ~ U[klo, khi], masses ~ U[mlo, mhi] (seeded).  Node (x, y, z) has index
    x + m y + m^2 z."""
    rng = np.random.default_rng(seed)
    n = m ** dim
    idx = np.arange(n).reshape((m,) * dim)
    rows, cols, ks = [], [], []
    diag = np.zeros(n)
    for ax in range(dim):
        # springs between neighbours along this axis, and to the walls at both ends
        lo = np.take(idx, range(0, m - 1), axis=ax).ravel()
        hi = np.take(idx, range(1, m), axis=ax).ravel()
        k = rng.uniform(klo, khi, size=lo.size)
        rows += [lo, hi]
        cols += [hi, lo]
        ks += [-k, -k]
        np.add.at(diag, lo, k)
        np.add.at(diag, hi, k)
        for end in (0, m - 1):
            w = np.take(idx, [end], axis=ax).ravel()
            diag[w] += rng.uniform(klo, khi, size=w.size)
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    ks.append(diag)
    K = sp.csr_matrix((np.concatenate(ks), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    K.sum_duplicates()
    K.sort_indices()
    masses = rng.uniform(mlo, mhi, size=n)
    return K, masses


def theta_matrix(K: sp.csr_matrix, masses: np.ndarray, alpha: float = 0.0, beta: float = 0.0) -> CSR:
    """Theta = [[0, I], [-M^-1 K, -M^-1 C]] of U' = Theta U, U = (displacements, velocities), for a
    lumped (diagonal) mass matrix M and Rayleigh damping C = alpha M + beta K (Eq. 2.1)."""
    n = K.shape[0]
    Minv = sp.diags(1.0 / masses)
    I = sp.identity(n, format="csr")
    MK = Minv @ K
    MC = alpha * I + beta * MK
    T = sp.bmat([[None, I], [-MK, -MC]], format="csr")
    return CSR.from_scipy(T)


def theta_lattice(m: int, dim: int, seed: int, dt: float, alpha: float = 0.0, beta: float = 0.0) -> CSR:
    """H = Theta dt (Eq. 2.2) for a seeded spring lattice (see spring_lattice)."""
    K, masses = spring_lattice(m, dim, seed)
    T = theta_matrix(K, masses, alpha, beta)
    return CSR(T.n, T.row_ptr, T.col, T.val * dt)


@dataclasses.dataclass
class Config:
    """A named workload: matrix builder, tau, tolerance and a description."""

    name: str
    build: Callable[[], CSR]
    tau: float
    eps: float
    desc: str


def _lap(m: int, dim: int) -> Callable[[], CSR]:
    return lambda: dirichlet_laplacian(m, dim)


CONFIGS: Dict[str, Config] = {
    "lap2d_m32": Config("lap2d_m32", _lap(32, 2), 1e-3, 1e-14,
                        "2-D 5-point Dirichlet Laplacian, 32x32 grid (n=1024), h=1/33, tau=1e-3, eps=1e-14"),
    "lap3d_m64": Config("lap3d_m64", _lap(64, 3), 5e-4, 1e-12,
                        "3-D 7-point Dirichlet Laplacian, 64^3 grid (n=262144), h=1/65, tau=5e-4, eps=1e-12"),
    "lap3d_m64_DL": Config("lap3d_m64_DL", lambda: diag_scale(dirichlet_laplacian(64, 3), seed=1)[0], 5e-4, 1e-12,
                           "D*L for the 64^3 Laplacian, D_ii ~ U[0.5,2] (seed 1), tau=5e-4, eps=1e-12"),
    "lap2d_m1500": Config("lap2d_m1500", _lap(1500, 2), 1e-6, 1e-12,
                          "2-D 5-point Dirichlet Laplacian, 1500x1500 grid (n=2.25M), h=1/1501, tau=1e-6, eps=1e-12"),
    "rgg_1e5": Config("rgg_1e5", lambda: rgg_adjacency(100_000, seed=3), 0.5, 1e-12,
                      "random geometric graph, n=1e5, mean degree 10, weights U[0.5,1.5], H = 0.5*A, eps=1e-12"),
    "theta_m300": Config("theta_m300", lambda: theta_lattice(300, 2, seed=6, dt=1.0, alpha=1e-3, beta=1e-3), 1.0,
                         1e-12, "structural vibration: Theta of a 300x300 spring lattice (n = 180,000), springs "
                                "U[0.5,1.5], masses U[0.5,2], Rayleigh damping 1e-3 M + 1e-3 K, dt = 1, eps = 1e-12"),
    "toeplitz_trid_n1e4": Config("toeplitz_trid_n1e4", lambda: toeplitz_trid(10_000, 1.0, -2.0, 1.0), 1.0, 1e-16,
                                 "trid(1,-2,1), n=10000, eps=1e-16 (paper Sec. 5.2, Tables 2-3)"),
    "toeplitz_heat_n1e4": Config("toeplitz_heat_n1e4", lambda: toeplitz_trid(10_000, -1.0 / 10_001, 2.0 / 10_001, -1.0 / 10_001),
                                 1.0, 1e-16, "(1/(n+1)) trid(-1,2,-1), n=10000, eps=1e-16 (paper Table 4)"),
}


def laplacian_batch(count: int = 256, seed: int = 2, side_lo: int = 16, side_hi: int = 128,
                    tau_lo: float = 1e-4, tau_hi: float = 1e-2) -> List[Tuple[CSR, float]]:
    """Independent 2-D Dirichlet Laplacians (h = 1/(side+1)) with their own tau: the batched
    workload (256 instances, side ~ U{16..128}, tau log-uniform in [1e-4, 1e-2], seed 2)."""
    return [(dirichlet_laplacian(side, 2), tau)
            for side, tau in batch_instances(count, seed, side_lo, side_hi, tau_lo, tau_hi)]


BATCH_EPS = 1e-12


def get_config(name: str, scale_m: int = 0) -> Config:
    """Named workload; scale_m > 0 gives the same grid family on an m = scale_m grid with the
    same tau/h^2 (so the same per-row kernel width) and tolerance."""
    c = CONFIGS[name]
    if not scale_m:
        return c
    if not (name.startswith("lap2d_m") or name.startswith("lap3d_m")):
        raise ValueError("scale_m applies to the grid-Laplacian workloads only")
    dim = 2 if name.startswith("lap2d") else 3
    m_full = int(name.split("_m")[1].split("_")[0])
    ratio = c.tau * (m_full + 1) ** 2
    tau = ratio / (scale_m + 1) ** 2
    build = (lambda: diag_scale(dirichlet_laplacian(scale_m, dim), seed=1)[0]) if name.endswith("_DL") \
        else _lap(scale_m, dim)
    return Config(f"{name}@m{scale_m}", build, tau, c.eps,
                  f"{c.desc.split(',')[0]} family on a {scale_m}^{dim} grid, same tau/h^2={ratio:.4g}, eps={c.eps}")
