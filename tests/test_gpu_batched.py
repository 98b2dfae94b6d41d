"""Batched form: many independent e^{tau_b H_b} in one block-diagonal run (sexpm_plan_batched /
sexpm_compute_batched), each instance held to the same parity bar against the oracle as the
plain path."""
import numpy as np
import pytest

from oracle import sexpm_oracle as O
from tests._compare import expm_parity, to_scipy, torch_csr
from workloads import CSR, diag_scale, dirichlet_laplacian, laplacian_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sx():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    sexpm.load()
    return sexpm


def _check_batch(sx, items, eps, **opts):
    outs = sx.expm_batched([torch_csr(H) for H, _ in items], [t for _, t in items], eps, **opts)
    assert len(outs) == len(items)
    for (H, tau), ((rp, ci, v), st) in zip(items, outs):
        G = to_scipy(rp, ci, v, H.n)
        E, so = O.expm(H.to_scipy(), tau, eps)
        assert (st["M"], st["N"]) == (so.M, so.N)
        assert bool(st["normal"]) == bool(so.normal)
        ts = [r["t"] for r in st["steps"]] + [s.t for s in so.steps] + [t.t for t in so.taylor]
        expm_parity(G, E, max(ts) if ts else 0.0)
    return outs


@pytest.mark.parametrize("symmetric", [1, 0])
def test_batched_laplacians_match_oracle(sx, symmetric):
    """Twelve 2-D Laplacians of different sizes and tau (different M_b, N_b)."""
    items = laplacian_batch(count=12, seed=5, side_lo=4, side_hi=24, tau_lo=1e-4, tau_hi=1e-2)
    outs = _check_batch(sx, items, 1e-12, symmetric=symmetric)
    assert len({st["N"] for _, st in outs}) > 1  # the instances really need different step counts


def test_batched_mixed_instances(sx):
    """Non-symmetric, scalar, zero and ragged instances in one batch."""
    L = dirichlet_laplacian(6, 3)
    DL, _ = diag_scale(L, seed=4)
    Z = CSR(4, np.array([0, 1, 1, 1, 1], dtype=np.int64), np.array([2], dtype=np.int32), np.zeros(1))
    items = [(DL, 2.0 / 49.0), (CSR.from_dense([[-2.0]]), 0.3), (Z, 1.0), (dirichlet_laplacian(9, 2), 1e-3),
             (CSR.from_dense([[1.0, 1e3], [0.0, 0.5]]), 1.0)]
    _check_batch(sx, items, 1e-12)


def test_batched_single_instance_equals_plain(sx):
    H = dirichlet_laplacian(20, 2)
    tau = 2e-3
    [((rp, ci, v), st)] = sx.expm_batched([torch_csr(H)], [tau], 1e-12)
    (rp2, ci2, v2), st2 = sx.expm(torch_csr(H), tau, 1e-12)
    A, B = to_scipy(rp, ci, v, H.n), to_scipy(rp2, ci2, v2, H.n)
    assert (st["M"], st["N"]) == (st2["M"], st2["N"])
    assert abs(A - B).max() <= 1e-14


def _sine_basis_expm(m, tau):
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam = -(4.0 / h ** 2) * np.sin(j * np.pi * h / 2) ** 2
    V = np.sqrt(2 * h) * np.sin(np.outer(j, j) * np.pi * h)
    return (V * np.exp(tau * lam)) @ V.T


def test_batched_full_workload_against_closed_form(sx):
    """The 256-instance workload (sides 16..128, tau log-uniform in [1e-4, 1e-2], eps = 1e-12),
    run as one batch exactly as bench.py times it; every instance is checked on sampled entries
    against e^{tau L_1} (x) e^{tau L_1} built from the 1-D sine eigenbasis, max-abs <= 1e-12 ||e^H||_1."""
    from workloads import BATCH_EPS
    items = laplacian_batch()
    outs = sx.expm_batched([torch_csr(H) for H, _ in items], [t for _, t in items], BATCH_EPS)
    rng = np.random.default_rng(0)
    worst = 0.0
    for (H, tau), ((rp, ci, v), st) in zip(items, outs):
        m = int(round(np.sqrt(H.n)))
        E1 = _sine_basis_expm(m, tau)
        norm1 = float(np.abs(E1).sum(axis=0).max()) ** 2   # ||E_1 (x) E_1||_1 = ||E_1||_1^2
        G = to_scipy(rp, ci, v, H.n)
        rows = rng.integers(0, H.n, size=8)
        for i in rows:
            row = G.getrow(int(i)).toarray().ravel()
            xi, yi = i % m, i // m
            exact = np.outer(E1[yi], E1[xi]).ravel()  # node j = x + m y
            err = float(np.abs(row - exact).max())
            worst = max(worst, err / norm1)
            assert err <= 1e-12 * norm1, (H.n, tau, i, err, norm1)
    print(f"batched workload: worst max-abs error / ||e^H||_1 over 256 instances x 8 rows = {worst:.2e}")


# ------------------------------------------------------------------ the captured squaring step

def _batch_results(sx, items, eps, **opts):
    plan = sx.BatchedPlan([torch_csr(H) for H, _ in items], eps, **opts)
    try:
        res = plan.compute([t for _, t in items])
        out = []
        for r in res:
            rp, ci, v = r.to_torch("cpu")
            out.append((rp.numpy().copy(), ci.numpy().copy(), v.numpy().copy(), r.stats()))
            r.free()
        info = plan.graph_info()
    finally:
        plan.close()
    return out, info


def _same_bits(A, B):
    for (rp, ci, v, st), (rp2, ci2, v2, st2) in zip(A, B):
        assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
        assert np.array_equal(v.view(np.uint64), v2.view(np.uint64))
        assert (st["M"], st["N"]) == (st2["M"], st2["N"])
        sq = [r for r in st["steps"] if r["phase"] == 1]
        sq2 = [r for r in st2["steps"] if r["phase"] == 1]
        assert [(r["nnz_raw"], r["nnz"], r["iters"], r["products"]) for r in sq] == \
            [(r["nnz_raw"], r["nnz"], r["iters"], r["products"]) for r in sq2]
        assert [r["t"] for r in sq] == [r["t"] for r in sq2]


@pytest.mark.parametrize("symmetric", [1, 0])
def test_graph_step_equals_host_driven_launches_bit_for_bit(sx, symmetric):
    """The captured step (sizes on the device, Algorithm 4.1 in a WHILE node) runs the same
    kernels and reductions as the host-driven batched launches: results, thresholds, pass counts
    and sizes agree bit for bit; and it matches the oracle."""
    items = laplacian_batch(count=10, seed=7, side_lo=4, side_hi=20, tau_lo=1e-4, tau_hi=1e-2)
    g, info = _batch_results(sx, items, 1e-12, symmetric=symmetric, batched_graph=1)
    h, info_h = _batch_results(sx, items, 1e-12, symmetric=symmetric, batched_graph=0)
    _same_bits(g, h)
    assert info["captures"] >= 1 and info["host_steps"] == 0
    assert info["kernels_per_step"] > 0 and info["kernels_per_pass"] == 3
    assert info_h["captures"] == 0
    _check_batch(sx, items, 1e-12, symmetric=symmetric, batched_graph=1)


def test_graph_arena_overflow_grows_and_resumes(sx):
    """A first arena far too small for the products (Taylor terms and squarings): the device flags
    the overflow, the host grows the arena to the recorded size and resumes at that step; the
    result is the same bit for bit as the host-driven launches."""
    items = laplacian_batch(count=6, seed=9, side_lo=6, side_hi=16, tau_lo=1e-3, tau_hi=1e-2)
    g, info = _batch_results(sx, items, 1e-12, batched_graph=1, batch_arena_bytes=4096)
    h, _ = _batch_results(sx, items, 1e-12, batched_graph=0)
    _same_bits(g, h)
    assert info["reruns"] >= 1 and info["captures"] == info["reruns"] + 1 and info["host_steps"] == 0


def test_graph_is_reused_across_computes_and_mixed_instances(sx):
    """A second compute of the same plan replays the captured graph (no new capture); a batch
    with non-normal, 1x1, all-zero and non-symmetric instances matches the oracle."""
    L = dirichlet_laplacian(6, 3)
    DL, _ = diag_scale(L, seed=4)
    Z = CSR(4, np.array([0, 1, 1, 1, 1], dtype=np.int64), np.array([2], dtype=np.int32), np.zeros(1))
    items = [(DL, 2.0 / 49.0), (CSR.from_dense([[-2.0]]), 0.3), (Z, 1.0), (dirichlet_laplacian(9, 2), 1e-3),
             (CSR.from_dense([[1.0, 1e3], [0.0, 0.5]]), 1.0)]
    plan = sx.BatchedPlan([torch_csr(H) for H, _ in items], 1e-12, batched_graph=1)
    try:
        taus = [t for _, t in items]
        first = []
        for r in plan.compute(taus):
            first.append(r.to_torch("cpu"))
            r.free()
        captures = plan.graph_info()["captures"]
        for r, (rp, ci, v) in zip(plan.compute(taus), first):
            rp2, ci2, v2 = r.to_torch("cpu")
            r.free()
            assert np.array_equal(v.numpy().view(np.uint64), v2.numpy().view(np.uint64))
        assert plan.graph_info()["captures"] == captures
    finally:
        plan.close()
    _check_batch(sx, items, 1e-12, batched_graph=1)


def test_layout_tuner_picks_a_candidate_and_results_stay_at_the_bar(sx):
    """sexpm_tune_batched times the built-in layouts (k-split budgets, wide blocks) and keeps the
    fastest; the tuned plan's results match the oracle."""
    items = laplacian_batch(count=8, seed=11, side_lo=8, side_hi=24, tau_lo=1e-3, tau_hi=1e-2)
    plan = sx.BatchedPlan([torch_csr(H) for H, _ in items], 1e-12)
    try:
        ms, best = plan.tune([t for _, t in items])
        assert len(ms) == 4 and 0 <= best < 4 and all(m > 0 for m in ms)
        assert ms[best] == min(ms)
        res = plan.compute([t for _, t in items])
        for (H, tau), r in zip(items, res):
            rp, ci, v = r.to_torch("cpu")
            st = r.stats()
            r.free()
            E, so = O.expm(H.to_scipy(), tau, 1e-12)
            ts = [x["t"] for x in st["steps"]] + [s.t for s in so.steps] + [t.t for t in so.taylor]
            expm_parity(to_scipy(rp, ci, v, H.n), E, max(ts) if ts else 0.0)
        assert plan.graph_info()["captures"] >= 4
    finally:
        plan.close()
