"""sexpm_filter_noalloc: the Algorithm 4.1 filter for callers that cannot allocate device
memory when they filter (another allocator owns the GPU's memory, or a fixed memory
budget is in force).  The entry point keeps its scratch in a static device array and
writes into caller-provided outputs; this test checks, through the C ABI, that two calls
in a row reproduce the allocating entry point sexpm_filter, and that the second call
allocates nothing: the device's free memory, torch's allocated bytes and the library's own
pool counters are the same before and after it.

Kept in a file of its own, named to be collected last."""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


def _matrix(n, seed):
    """About 25 entries per row, values spread over 45 orders of magnitude (seeded)."""
    rng = np.random.default_rng(seed)
    k = 25 * n
    A = sp.csr_matrix((rng.standard_normal(k) * np.exp(rng.uniform(-45, 0, k)),
                       (rng.integers(0, n, k), rng.integers(0, n, k))), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A, float(np.exp(rng.uniform(-33, -18)))


def _dev(A):
    import torch
    return (torch.from_numpy(A.indptr.astype(np.int64)).cuda(), torch.from_numpy(A.indices.astype(np.int32)).cuda(),
            torch.from_numpy(A.data.astype(np.float64)).cuda(), A.shape[0])


def test_noalloc_filter_matches_allocating_filter_twice():
    import torch
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm

    for seed, n in [(11, 5000), (12, 70000)]:
        A, eps_g = _matrix(n, seed)
        dA = _dev(A)
        (rp0, ci0, v0), t0, it0, b0 = sexpm.filter_csr(dA, eps_g, 0.1)
        cap = A.nnz
        out = (torch.empty(n + 1, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int32, device="cuda"),
               torch.empty(cap, dtype=torch.float64, device="cuda"))
        for call in range(2):
            # poison the outputs so a stale result cannot pass
            out[0].fill_(-7); out[1].fill_(-7); out[2].fill_(float("nan"))
            torch.cuda.synchronize()
            before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), sexpm.pool_stats())
            (rp, ci, v), t, it, b = sexpm.filter_noalloc(dA, eps_g, 0.1, out=out)
            torch.cuda.synchronize()
            after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), sexpm.pool_stats())
            if call == 1:
                # the first call on a device may load kernels; from the second on nothing is allocated
                assert after == before, (before, after)
            assert it == it0
            assert t == pytest.approx(t0, rel=1e-12)
            assert b == pytest.approx(b0, rel=1e-12)
            G = sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))
            R = sp.csr_matrix((v0.cpu().numpy(), ci0.cpu().numpy(), rp0.cpu().numpy()), shape=(n, n))
            assert G.nnz == R.nnz
            assert np.array_equal(G.indptr, R.indptr) and np.array_equal(G.indices, R.indices)
            assert np.array_equal(G.data, R.data)


def test_noalloc_filter_rejects_too_many_rows():
    import torch
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm

    n = sexpm.NOALLOC_MAX_ROWS + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sexpm.SexpmError) as ei:
        sexpm.filter_noalloc((rp, ci[:0], v[:0], n), 1e-12, 0.1, out=(rp, ci, v))
    assert ei.value.code == -7
    assert "at most" in str(ei.value)


def test_noalloc_filter_leaves_outputs_untouched_on_overflow():
    """An output too small for the kept part returns SEXPM_EOVERFLOW before any output is written."""
    import torch
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm

    A, eps_g = _matrix(3000, 13)
    dA = _dev(A)
    (_, ci0, _), _, _, _ = sexpm.filter_csr(dA, eps_g, 0.1)
    cap = int(ci0.numel()) - 1
    assert cap >= 0
    out = (torch.full((A.shape[0] + 1,), -7, dtype=torch.int64, device="cuda"),
           torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda"),
           torch.full((max(cap, 1),), -7.0, dtype=torch.float64, device="cuda"))
    with pytest.raises(sexpm.SexpmError) as ei:
        sexpm.filter_noalloc(dA, eps_g, 0.1, out=(out[0], out[1][:cap], out[2][:cap]))
    assert ei.value.code == -7
    assert bool((out[0] == -7).all()) and bool((out[1] == -7).all()) and bool((out[2] == -7.0).all())
