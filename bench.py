#!/usr/bin/env python
"""Benchmark: time to e^{tau H} on a GB300 through the library's C ABI.

One step = one sexpm_compute(plan, tau): the whole hot path of Algorithm 4.2
((M, N) choice, filtered Taylor phase, N filtered squarings with Algorithm 4.1,
I + T^_N) on a synthetic workload whose input H is resident in HBM.

Default workload: the 2-D 5-point Dirichlet Laplacian on a 1500x1500 grid
(n = 2.25M, 11.2M nnz), h = 1/1501, tau = 1e-6, eps = 1e-12.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead,
on a bounded sample of the same workload, in the same unit.
Multi-GPU runs (torchrun, N ranks) are independent replicas: the method has no
data-path exchange on one matrix in this build, so each rank computes its own e^{tau H}.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07e9 / 1e9   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
# DRAM bytes (read + write) of the numeric pass per formed product, from one ncu capture of every
# k_numeric launch of the 2-D Laplacian family on a 300^2 grid (same row widths as the 1500^2
# workload; 26.07 GB for 5.372e10 formed products); the full-size traffic is this times the
# products formed (the full-size run holds too much device memory for a multi-pass capture).
NUMERIC_DRAM_BYTES_PER_PRODUCT = 26.071323392e9 / 53716599900
METRIC = "time-to-e^{tau H} (reported as e^{tau H} computations per second, whole job)"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """Max of x over the ranks of the process group (x itself for one rank).  The reduction runs
    on the group's device: CUDA tensors for NCCL, host tensors for gloo."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ms_max: float, ws: int) -> float:
    """e^{tau H} per second over all replicas: each rank computes one per step, and the job's
    step takes as long as its slowest rank's (ms_max)."""
    return ws * 1000.0 / ms_max


def _oracle_sample(cfg_name: str, m_sample: int):
    """Runs the CPU oracle on the same workload family at a smaller grid; returns (seconds, products, desc)."""
    from oracle import sexpm_oracle as O
    from workloads import dirichlet_laplacian, get_config
    c = get_config(cfg_name)
    if cfg_name.startswith("lap2d") or cfg_name.startswith("lap3d"):
        dim = 2 if cfg_name.startswith("lap2d") else 3
        m_full = int(cfg_name.split("_m")[1].split("_")[0])
        ratio = c.tau * (m_full + 1) ** 2           # tau / h^2 of the full workload
        H = dirichlet_laplacian(m_sample, dim).to_scipy()
        tau = ratio / (m_sample + 1) ** 2
        desc = (f"oracle (numpy/scipy, 1 thread) on the {dim}-D Laplacian with m={m_sample} "
                f"(n={m_sample ** dim}), same tau/h^2={ratio:.4g} and eps={c.eps}")
    else:
        H = c.build().to_scipy()
        tau = c.tau
        desc = f"oracle on {cfg_name}"
    t0 = time.perf_counter()
    E, st = O.expm(H, tau, c.eps)
    dt = time.perf_counter() - t0
    return dt, H.shape[0], desc


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    from workloads import get_config
    c = get_config(args.workload)
    n_full = c.build().n
    times = []
    n_s = None
    desc = ""
    for k in range(args.warmup + args.steps):
        dt, n_s, desc = _oracle_sample(args.workload, args.sample_m)
        if k >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = (n_s / t) / n_full                            # rows of e^{tau H} per second, scaled to the full n
    ncores = 1                                            # scipy's sparse product runs on one thread
    est = {"kind": "estimate: the timed sample's rate per row times the workload's rows",
           "timed_n": n_s, "timed_ms_per_step": 1000.0 * t, "workload_n": n_full}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "expm/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t,
        "ms_per_step_is": "the timed sample's (n = %d), not the workload's" % n_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": c.desc, "timed_sample": desc},
        "value_estimate": est,
        "cpu_baseline": {"value": value, "unit": "expm/s", "cores": ncores, "host_cores": _host_cores(),
                         "kind": "oracle", "estimate": est,
                         "sample": f"{desc}; {t:.2f} s per step; scaled by the row count to n={n_full} "
                                   f"(same per-row work for interior rows)"},
        "e2e": {"value": value, "unit": "expm/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_batched(sexpm, torch, steps: int = 2):
    """Batched form (256 independent 2-D Laplacians, one block-diagonal run): the captured squaring
    step (one CUDA graph launch per squaring, sizes decided on the device), the same run with
    host-driven launches, and the plain per-matrix loop, on the same GPU with inputs resident on
    the device."""
    from workloads import BATCH_EPS, laplacian_batch
    items = laplacian_batch()
    devs = [(torch.from_numpy(H.row_ptr).cuda(), torch.from_numpy(H.col).cuda(), torch.from_numpy(H.val).cuda(), H.n)
            for H, _ in items]
    taus = [t for _, t in items]

    def run_batched(graph: int):
        bplan = sexpm.BatchedPlan(devs, BATCH_EPS, batched_graph=graph)
        for r in bplan.compute(taus):      # warm-up (captures the step graph, sizes the arena)
            r.free()
        torch.cuda.synchronize()
        l0 = sexpm.kernel_launches()
        t0 = time.perf_counter()
        st = None
        mmax = 0
        for _ in range(steps):
            res = bplan.compute(taus)
            st = res[0].stats()
            mmax = max(r.stats()["M"] for r in res)
            for r in res:
                r.free()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        launches = (sexpm.kernel_launches() - l0) // steps
        info = bplan.graph_info()
        bplan.close()
        sexpm.release_memory()
        sq = [x for x in st["steps"] if x["phase"] == 1]
        return (dt, launches, info, sum(x["products_done"] for x in sq), st["ms_squaring"], len(sq), st["peak_bytes"],
                max(mmax - 1, 0))

    t_graph, l_graph, info, formed, sq_ms, nsq, peak_g, nterms = run_batched(1)
    t_host, l_host, _, _, sq_ms_host, _, peak_h, _ = run_batched(0)
    plans = [sexpm.Plan(d, BATCH_EPS) for d in devs]
    for p, t in zip(plans, taus):      # warm-up
        p.compute(t).free()
    torch.cuda.synchronize()
    l0 = sexpm.kernel_launches()
    t0 = time.perf_counter()
    for p, t in zip(plans, taus):
        p.compute(t).free()
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    l_loop = sexpm.kernel_launches() - l0
    for p in plans:
        p.close()
    peak = 152 * 2 * 2 * 2.07  # GFLOP/s of the FP64 pipe (derived, as in the headline roofline)
    gflops = 2.0 * formed / (sq_ms * 1e6) if sq_ms > 0 else 0.0
    return {"workload": "256 2-D Dirichlet Laplacians, side ~ U{16..128}, tau log-uniform [1e-4, 1e-2], eps 1e-12",
            "n_total": int(sum(H.n for H, _ in items)), "batched_ms": 1000.0 * t_graph,
            "batched_host_driven_ms": 1000.0 * t_host, "per_matrix_loop_ms": 1000.0 * t_loop,
            "speedup_vs_loop": t_loop / t_graph, "launches_batched": int(l_graph),
            "launches_batched_host_driven": int(l_host), "launches_loop": int(l_loop),
            "graph": {"squaring_steps": nsq, "taylor_terms": nterms,
                      "graph_launches_per_batch": nterms + nsq - info["host_steps"],
                      "kernels_per_step": info["kernels_per_step"], "kernels_per_alg41_pass": info["kernels_per_pass"],
                      "arena_bytes": info["arena_bytes"], "resumed_steps": info["reruns"],
                      "host_driven_steps": info["host_steps"]},
            "peak_bytes_graph": int(peak_g), "peak_bytes_host_driven": int(peak_h),
            "squaring_products_formed": int(formed), "squaring_ms": sq_ms, "squaring_ms_host_driven": sq_ms_host,
            "squaring_fp64_gflops": gflops, "squaring_fp64_frac": gflops / peak, "steps": steps}


def measure_complex(sexpm, torch, m: int = 600):
    """Complex H: the Schroedinger propagator e^{i tau L} of the 2-D Dirichlet Laplacian on an m x m
    grid (tau / h^2 = 2.253 as in the bench workload, eps = 1e-12) against the real e^{tau L} on
    the same grid; inputs resident on the device."""
    import numpy as np
    from workloads import dirichlet_laplacian
    L = dirichlet_laplacian(m, 2)
    tau = 2.253 / (m + 1) ** 2
    rp = torch.from_numpy(L.row_ptr).cuda()
    ci = torch.from_numpy(L.col).cuda()
    vr = torch.from_numpy(L.val).cuda()
    vz = torch.from_numpy((1j * L.val).astype(np.complex128)).cuda()
    out = {"workload": f"e^(i tau L), 2-D Dirichlet Laplacian {m}x{m} (n={L.n}), tau/h^2 = 2.253, eps 1e-12"}
    for key, plan in (("complex", sexpm.ComplexPlan((rp, ci, vz, L.n), 1e-12)), ("real", sexpm.Plan((rp, ci, vr, L.n), 1e-12))):
        plan.compute(tau).free()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = plan.compute(tau)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = r.stats()
        r.free()
        plan.close()
        formed = sum(x["products_done"] for x in st["steps"])
        num_ms = sum(x["ms_numeric"] for x in st["steps"])
        out[key] = {"ms": 1000.0 * dt, "M": st["M"], "N": st["N"], "nnz_out": st["nnz_out"],
                    "real_products_formed": int(formed), "numeric_ms": num_ms,
                    "numeric_gflops": 2.0 * formed / (num_ms * 1e6) if num_ms > 0 else 0.0}
    out["complex_over_real"] = out["complex"]["ms"] / out["real"]["ms"]
    return out


def measure_adjoint(sexpm, torch, fd_edges: int = 0):
    """Adjoint form on the random-geometric-graph workload: H = beta A (n = 1e5, mean degree 10,
    weights U[0.5, 1.5], beta = 0.5, eps = 1e-12), L = sum_ij W_ij [e^H]_ij with 1e5 seeded
    entries of W; dL/dA_e = beta (dL/dH_uv + dL/dH_vu) on every edge.  Times the plain forward
    and the adjoint (its own forward plus the reverse pass) and, optionally, checks fd_edges
    random edges against central differences of the GPU forward."""
    import numpy as np
    import scipy.sparse as sp
    from workloads import rgg_adjacency, sparse_loss_weights
    beta, eps, n = 0.5, 1e-12, 100_000
    A = rgg_adjacency(n, seed=3)
    W = sparse_loss_weights(n, 100_000, seed=3)
    dev = lambda M, vals=None: (torch.from_numpy(M.row_ptr).cuda(), torch.from_numpy(M.col).cuda(),
                                torch.from_numpy(M.val if vals is None else vals).cuda(), M.n)
    Hv = beta * A.val
    plan = sexpm.Plan(dev(A, Hv), eps)
    plan.compute(1.0).free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = plan.compute(1.0)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    st = res.stats()
    res.free()
    t0 = time.perf_counter()
    rp, ci, g = sexpm.adjoint(plan, 1.0, eps, dev(W))
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    plan.close()
    G = sp.csr_matrix((g.cpu().numpy(), A.col, A.row_ptr), shape=(n, n))
    out = {"workload": "RGG n=1e5, mean degree 10, H = 0.5 A, eps 1e-12, W with 1e5 entries",
           "M": st["M"], "N": st["N"], "nnz_expm": st["nnz_out"], "forward_ms": 1000.0 * t_fwd,
           "adjoint_ms": 1000.0 * t_adj, "adjoint_over_forward": t_adj / t_fwd}
    if fd_edges:
        Ws = W.to_scipy()
        Au = sp.triu(A.to_scipy(), 1).tocoo()
        rng = np.random.default_rng(3)
        pick = rng.choice(Au.nnz, size=fd_edges, replace=False)
        Acsr = A.to_scipy()

        def loss(vals):
            (erp, eci, ev), _ = sexpm.expm(dev(A, beta * vals), 1.0, eps, symmetric=0)
            E = sp.csr_matrix((ev.cpu().numpy(), eci.cpu().numpy(), erp.cpu().numpy()), shape=(n, n))
            return float(E.multiply(Ws).sum())

        worst = 0.0
        gmax = float(np.abs(G).max()) if G.nnz else 0.0
        for e in pick:
            u, v = int(Au.row[e]), int(Au.col[e])
            puv = A.row_ptr[u] + np.searchsorted(A.col[A.row_ptr[u]:A.row_ptr[u + 1]], v)
            pvu = A.row_ptr[v] + np.searchsorted(A.col[A.row_ptr[v]:A.row_ptr[v + 1]], u)
            d = 1e-4 * A.val[puv]
            vp, vm = A.val.copy(), A.val.copy()
            vp[[puv, pvu]] += d
            vm[[puv, pvu]] -= d
            fd = (loss(vp) - loss(vm)) / (2 * d)
            ad = beta * (G[u, v] + G[v, u])
            worst = max(worst, abs(ad - fd) / max(abs(fd), abs(ad), 1e-3 * beta * gmax, 1e-300))
        out.update({"fd_edges": int(fd_edges), "fd_max_rel_err": worst,
                    "fd_rel_err_floor": "max(|fd|, |adjoint|, 1e-3 max|dL/dA|)"})
    return out


def measure_adjoint_trace(sexpm, torch, Hdev, c, n: int):
    """Adjoint form on the bench workload: L = trace(P e^{tau H}) with a seeded diagonal P
    (P_ii ~ U[0, 1], seed 4), i.e. dL/dE = P.  Times the kept forward (every product formed,
    checkpoints every ceil(sqrt(N)) squarings) and the reverse pass (recomputing the iterates between
    checkpoints), and the peak device memory the library held over both."""
    import numpy as np
    from workloads import diag_weights
    P = diag_weights(n, seed=4)
    W = (torch.arange(n + 1, dtype=torch.int64, device="cuda"), torch.arange(n, dtype=torch.int32, device="cuda"),
         torch.from_numpy(P).cuda(), n)
    plan = sexpm.Plan(Hdev, c.eps)
    sexpm.release_memory()
    live0, _ = sexpm.pool_stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tape, res = plan.forward_keep(c.tau)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st = res.stats()
    res.free()
    rp, ci, g = tape.adjoint(W)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    live1, peak1 = sexpm.pool_stats()
    tape.free()
    plan.close()
    gmax = float(g.abs().max()) if g.numel() else 0.0
    del rp, ci, g
    sexpm.release_memory()
    return {"workload": "L = trace(P e^{tau H}), P_ii ~ U[0,1] (seed 4), on the bench workload",
            "M": st["M"], "N": st["N"], "forward_keep_ms": 1000.0 * (t1 - t0), "reverse_ms": 1000.0 * (t2 - t1),
            "adjoint_total_ms": 1000.0 * (t2 - t0), "peak_hbm_bytes": int(peak1 - live0), "max_abs_dL_dH": gmax}


def error_vs_exact(sexpm, torch, res, c, H, rows: int = 16):
    """Max-abs error of sampled full rows of e^{tau H} against the closed form of the grid
    Laplacian: e^{tau L_1} (x) e^{tau L_1} (x ...) with the 1-D sine eigenbasis.  None for other
    workloads."""
    import numpy as np
    name = c.name.split("@")[0]
    if not (name.startswith("lap2d_m") or name.startswith("lap3d_m")) or name.endswith("_DL"):
        return None
    dim = 2 if name.startswith("lap2d") else 3
    m = int(round(H.n ** (1.0 / dim)))
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    lam = -(4.0 / h ** 2) * np.sin(j * np.pi * h / 2) ** 2
    V = np.sqrt(2 * h) * np.sin(np.outer(j, j) * np.pi * h)
    E1 = (V * np.exp(c.tau * lam)) @ V.T
    try:
        n_, nnz = res.info()
        rp = np.empty(n_ + 1, dtype=np.int64)
        import ctypes
        sexpm._check(sexpm.load().sexpm_result_copy(res._h, rp.ctypes.data, None, None, 0))
        rng = np.random.default_rng(11)
        pick = sorted(set(int(x) for x in rng.integers(0, H.n, size=rows)) | {0, H.n - 1, H.n // 2})
        ci_all, v_all = res.to_torch("cuda")[1:]
        worst = 0.0
        for i in pick:
            a, b = int(rp[i]), int(rp[i + 1])
            cols = ci_all[a:b].cpu().numpy()
            vals = v_all[a:b].cpu().numpy()
            if dim == 2:
                exact = np.outer(E1[i // m], E1[i % m]).ravel()
            else:
                exact = np.einsum("a,b,c->abc", E1[i // (m * m)], E1[(i // m) % m], E1[i % m]).ravel()
            got = np.zeros(H.n)
            got[cols] = vals
            worst = max(worst, float(np.abs(got - exact).max()))
        del ci_all, v_all
    finally:
        res.free()
    sexpm.release_memory()
    return {"max_abs": worst, "rows_sampled": len(pick), "norm1_of_expm_at_most": 1.0,
            "reference": "e^{tau L_1} Kronecker products from the 1-D sine eigenbasis (exact up to rounding)"}


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    from workloads import get_config

    c = get_config(args.workload, args.scale_m)
    H = c.build()
    dev = (torch.from_numpy(H.row_ptr).cuda(), torch.from_numpy(H.col).cuda(), torch.from_numpy(H.val).cuda(), H.n)
    plan = sexpm.Plan(dev, c.eps)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (also establishes the output size for the e2e buffers)
    last = None
    for _ in range(args.warmup):
        res = plan.compute(c.tau)
        last = res.stats()
        res.free()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sexpm.kernel_launches()
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    last = None
    for k in range(args.steps):
        res = plan.compute(c.tau)
        stats.append(res.stats())
        if k == args.steps - 1:
            last = res          # kept for the error check after the timed region
        else:
            res.free()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = sexpm.kernel_launches() - l0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
    value = whole_job_rate(ms, ws)

    # roofline: dominant kernel = numeric pass of the sparse products (FP64 ALU bound)
    st = stats[-1]
    num_flops = sum(r["flops"] for r in st["steps"])
    num_ms = sum(r["ms_numeric"] for r in st["steps"])
    sq_flops = sum(r["flops"] for r in st["steps"] if r["phase"] == 1)
    sq_ms = sum(r["ms_numeric"] for r in st["steps"] if r["phase"] == 1)
    sq_step_ms = sum(r["ms"] for r in st["steps"] if r["phase"] == 1)
    achieved = num_flops / (num_ms * 1e-3) / 1e9 if num_ms else 0.0
    hbm_peak, hbm_kind = _peaks()
    f_bytes = sum(r["bytes_filter"] for r in st["steps"])
    f_ms = sum(r["ms_filter"] for r in st["steps"])
    f_gbs = f_bytes / (f_ms * 1e-3) / 1e9 if f_ms else 0.0
    products = sum(r["products"] for r in st["steps"])

    err = None
    if rank == 0 and ws == 1:
        err = error_vs_exact(sexpm, torch, last, c, H)
    last = None
    sexpm.release_memory()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hp = [torch.from_numpy(H.row_ptr).pin_memory(), torch.from_numpy(H.col).pin_memory(),
              torch.from_numpy(H.val).pin_memory()]
        nnz_out = st["nnz_out"]
        out_rp = torch.empty(H.n + 1, dtype=torch.int64).pin_memory()
        out_ci = torch.empty(nnz_out, dtype=torch.int32).pin_memory()
        out_v = torch.empty(nnz_out, dtype=torch.float64).pin_memory()
        h2d = sum(x.numel() * x.element_size() for x in hp)
        d2h_list = []
        times = []
        parts = []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            p2 = sexpm.Plan((hp[0], hp[1], hp[2], H.n), c.eps)
            t1 = time.perf_counter()
            res = p2.compute(c.tau)
            t2 = time.perf_counter()
            n_, nnz_ = res.info()
            if nnz_ > out_v.numel():
                out_ci = torch.empty(nnz_, dtype=torch.int32).pin_memory()
                out_v = torch.empty(nnz_, dtype=torch.float64).pin_memory()
            sexpm._check(sexpm.load().sexpm_result_copy(res._h, out_rp.data_ptr(), out_ci.data_ptr(),
                                                        out_v.data_ptr(), 0))
            t3 = time.perf_counter()
            res.free()
            p2.close()
            dt = time.perf_counter() - t0
            if k > 0:
                times.append(dt)
                parts.append((t1 - t0, t2 - t1, t3 - t2))
                d2h_list.append((H.n + 1) * 8 + nnz_ * 12)
        e2e_s = max_over_ranks(statistics.mean(times), ws)
        e2e = {"value": whole_job_rate(1000.0 * e2e_s, ws), "unit": "expm/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(statistics.mean(d2h_list)), "ms_per_step": 1000.0 * e2e_s,
               "plan_ms": 1000.0 * statistics.mean(x[0] for x in parts),
               "compute_ms": 1000.0 * statistics.mean(x[1] for x in parts),
               "copy_ms": 1000.0 * statistics.mean(x[2] for x in parts)}

    forms = None
    if rank == 0 and ws == 1:
        if not args.no_forms:
            forms = {"adjoint_trace": measure_adjoint_trace(sexpm, torch, dev, c, H.n),
                     "adjoint_rgg": measure_adjoint(sexpm, torch, args.fd_edges)}
        if args.forms:
            forms = forms or {}
            forms["complex"] = measure_complex(sexpm, torch)
            forms["batched"] = measure_batched(sexpm, torch)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        dt, n_s, desc = _oracle_sample(args.workload, args.sample_m)
        cpu_val = (n_s / dt) / H.n
        cpu = {"value": cpu_val, "unit": "expm/s", "cores": 1, "host_cores": _host_cores(), "kind": "oracle",
               "estimate": {"kind": "estimate: the timed sample's rate per row times the workload's rows",
                            "timed_n": n_s, "timed_ms_per_step": 1000.0 * dt, "workload_n": H.n},
               "sample": f"{desc}; {dt:.2f} s; scaled by the row count to n={H.n} "
                         f"(same per-row work for interior rows)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "expm/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": c.name, "desc": c.desc, "n": H.n, "nnz_H": H.nnz,
                       "M": st["M"], "N": st["N"], "nnz_expm": st["nnz_out"],
                       "l2": "inputs larger than L2 (every squaring streams T^_i of > 129 MB)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "alu", "kernel": "k_numeric (sparse product numeric pass, FP64)",
                         "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_PEAK_GFLOPS,
                         "traffic": NUMERIC_DRAM_BYTES_PER_PRODUCT * sum(r["products_done"] for r in st["steps"]),
                         "traffic_note": "bytes per e^{tau H} (all k_numeric launches): ncu DRAM bytes per formed "
                                         "product on the 300^2 case times the products formed here",
                         "peak_kind": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (derived)"},
            "roofline_hbm": {"bound": "hbm", "kernel": "Algorithm 4.1 passes + scan + compaction",
                             "achieved": f_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": f_gbs / hbm_peak, "peak_kind": hbm_kind},
            "phases_ms": {"total": st["ms_total"], "taylor": st["ms_taylor"], "squaring": st["ms_squaring"],
                          "final": st["ms_final"], "numeric": num_ms,
                          "symbolic": sum(r["ms_symbolic"] for r in st["steps"]), "filter": f_ms},
            "squaring_gflops_useful": (2.0 * sum(r["products"] for r in st["steps"] if r["phase"] == 1)) /
                                      (sq_step_ms * 1e-3) / 1e9 if sq_step_ms else None,
            "squaring_numeric_gflops": sq_flops / (sq_ms * 1e-3) / 1e9 if sq_ms else None,
            "products": products, "products_done": sum(r["products_done"] for r in st["steps"]),
            "symmetric_products": bool(st["symmetric"]), "peak_hbm_bytes": st["peak_bytes"],
            "per_step": [{"phase": "taylor" if r["phase"] == 0 else "square", "i": r["i"], "products": r["products"],
                          "chunks": r["chunks"], "rows_class": r["rows_class"], "nnz_stream": r["nnz_stream"],
                          "products_done": r["products_done"],
                          "nnz_raw": r["nnz_raw"], "nnz": r["nnz"], "t": r["t"], "iters": r["iters"],
                          "ms": round(r["ms"], 3), "ms_numeric": round(r["ms_numeric"], 3),
                          "ms_symbolic": round(r["ms_symbolic"], 3), "ms_filter": round(r["ms_filter"], 3),
                          "numeric_gflops": round(r["flops"] / (r["ms_numeric"] * 1e6), 1) if r["ms_numeric"] else None}
                         for r in st["steps"]] if args.per_step else None,
            "gpu_launches": launches, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "forms": forms,
            "error_vs_exact": err,
            "chunked_steps": sum(1 for r in st["steps"] if r["chunks"] > 1),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _relaunch_with_ranks(n: int, argv) -> int:
    """`bench.py --gpus N` started as one process: launch N ranks on this node (one per GPU) through
    torch.distributed.run, as the multi-GPU launch does, and return its exit code."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", os.environ.get("SEXPM_BENCH_PORT", "29517"),
           os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lap2d_m1500")
    ap.add_argument("--scale-m", type=int, default=0,
                    help="run the grid workload on an m-sided grid with the same tau/h^2 (profiling sizes)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--per-step", action="store_true", help="add the per-step records to the JSON line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fd-edges", type=int, default=0,
                    help="with --forms: check the adjoint on this many random edges by finite differences")
    ap.add_argument("--forms", action="store_true",
                    help="also time the batched form against the per-matrix loop and check the adjoint by "
                         "finite differences (several minutes)")
    ap.add_argument("--sample-m", type=int, default=80,
                    help="grid side of the oracle's sample of the workload (same tau/h^2 and eps)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the adjoint timings that the default line carries")
    args = ap.parse_args(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return _relaunch_with_ranks(args.gpus, argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
