"""Comparison helpers for the GPU-vs-oracle parity tests."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def to_scipy(rp, ci, v, n) -> sp.csr_matrix:
    if hasattr(rp, "cpu"):
        rp, ci, v = rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy()
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def torch_csr(A, device="cuda"):
    import torch
    return (torch.from_numpy(np.asarray(A.row_ptr, dtype=np.int64)).to(device),
            torch.from_numpy(np.asarray(A.col, dtype=np.int32)).to(device),
            torch.from_numpy(np.asarray(A.val, dtype=np.float64)).to(device), A.n)


def norm1(A) -> float:
    return float(np.abs(A).sum(axis=0).max()) if A.nnz else 0.0


def expm_parity(G: sp.csr_matrix, R: sp.csr_matrix, t_drop: float, rtol: float = 1e-12):
    """Parity bar for e^H: max |G - R| <= rtol ||R||_1 over the union of both patterns, and
    entries stored in only one of them have magnitude <= 2 t_drop (the allowed filter flips).

    Returns a dict of the measured quantities; raises AssertionError on failure."""
    G = sp.csr_matrix(G); R = sp.csr_matrix(R)
    G.sort_indices(); R.sort_indices()
    D = (G - R).tocsr()
    maxabs = float(np.abs(D.data).max()) if D.nnz else 0.0
    n1 = norm1(R)
    gp = sp.csr_matrix((np.ones(G.nnz), G.indices, G.indptr), shape=G.shape)
    rp = sp.csr_matrix((np.ones(R.nnz), R.indices, R.indptr), shape=R.shape)
    only_g = (gp - gp.multiply(rp)).tocoo()
    only_r = (rp - rp.multiply(gp)).tocoo()
    vg = np.abs(np.asarray(G[only_g.row, only_g.col]).ravel()) if only_g.nnz else np.zeros(0)
    vr = np.abs(np.asarray(R[only_r.row, only_r.col]).ravel()) if only_r.nnz else np.zeros(0)
    worst_flip = float(max(vg.max() if vg.size else 0.0, vr.max() if vr.size else 0.0))
    out = {"maxabs": maxabs, "norm1": n1, "only_gpu": int(only_g.nnz), "only_oracle": int(only_r.nnz),
           "worst_flip": worst_flip, "nnz_gpu": int(G.nnz), "nnz_oracle": int(R.nnz), "t_drop": t_drop}
    DROP_FLIPS.append(out)
    assert maxabs <= rtol * max(n1, 1e-300), out
    assert worst_flip <= 2.0 * t_drop, out
    return out


# Every expm_parity call of the session, for the drop-decision summary printed at the end of the
# run (entries stored by one side only, i.e. filter decisions that differ, and their size against
# the drop threshold).
DROP_FLIPS: list = []


def taylor_time_stepper(Ht, R, substeps: int, rel_stop: float = 1e-20):
    """e^H R by `substeps` steps of a truncated Taylor series of e^{H/substeps} applied to the block
    of vectors R (torch sparse CSR H on the GPU, cuSPARSE products): each step sums terms until one
    falls below rel_stop of the running sum.  Independent of the library's method."""
    import torch
    Y = R.clone()
    for _ in range(substeps):
        term, acc = Y.clone(), Y.clone()
        for k in range(1, 80):
            term = torch.sparse.mm(Ht, term) / (substeps * k)
            acc = acc + term
            if term.abs().max() <= rel_stop * acc.abs().max():
                break
        Y = acc
    return Y
