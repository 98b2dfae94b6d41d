"""Python binding of libsexpm (the C ABI declared in include/sexpm.h).

Argument marshalling only: every step of the method runs inside the library's
CUDA kernels.  PyTorch supplies device buffers and the current CUDA stream.
The library must have been built (``python -m paper_2110_04493_gb300.build``);
without it the first call into the library raises ImportError: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Any, Dict, List, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsexpm.so")

SEXPM_OK = 0
ERROR_NAMES = {
    -1: "SEXPM_EINVAL", -2: "SEXPM_ENOMEM", -3: "SEXPM_ECUDA", -4: "SEXPM_ENOCONV",
    -5: "SEXPM_ENOPARAM", -6: "SEXPM_ETIMEOUT", -7: "SEXPM_EOVERFLOW",
}


class SexpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class CsrView(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class Options(ctypes.Structure):
    _fields_ = [("e_r", ctypes.c_double), ("square_scale", ctypes.c_int32), ("normal_override", ctypes.c_int32),
                ("max_filter_iters", ctypes.c_int32), ("n_extra", ctypes.c_int32), ("max_taylor", ctypes.c_int32),
                ("symmetric", ctypes.c_int32), ("row_order", ctypes.c_int32), ("chunk_bytes", ctypes.c_int64),
                ("scaling", ctypes.c_int32), ("refine_kmax", ctypes.c_int32), ("batched_graph", ctypes.c_int32),
                ("batch_arena_bytes", ctypes.c_int64)]


class StepStats(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int32), ("i", ctypes.c_int32), ("iters", ctypes.c_int32), ("chunks", ctypes.c_int32),
                ("eps_g", ctypes.c_double), ("t", ctypes.c_double), ("b", ctypes.c_double),
                ("norm_F", ctypes.c_double), ("nnz_raw", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("products", ctypes.c_int64), ("products_done", ctypes.c_int64), ("ms", ctypes.c_double), ("ms_symbolic", ctypes.c_double),
                ("ms_numeric", ctypes.c_double), ("ms_filter", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes_filter", ctypes.c_double), ("nnz_stream", ctypes.c_int64), ("rows_class", ctypes.c_int64 * 6)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("norm_H", ctypes.c_double), ("M", ctypes.c_int32), ("N", ctypes.c_int32),
                ("normal", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("symmetric", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("a", ctypes.c_double),
                ("r0", ctypes.c_double), ("eps_g0", ctypes.c_double), ("nnz_out", ctypes.c_int64),
                ("ms_total", ctypes.c_double), ("ms_taylor", ctypes.c_double), ("ms_squaring", ctypes.c_double),
                ("ms_final", ctypes.c_double), ("peak_bytes", ctypes.c_int64), ("launches", ctypes.c_int64)]


_lib: Optional[ctypes.CDLL] = None


def load() -> ctypes.CDLL:
    """Load libsexpm.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built; run python -m paper_2110_04493_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.sexpm_last_error.restype = ctypes.c_char_p
    L.sexpm_options_default.argtypes = [P(Options)]
    L.sexpm_plan.argtypes = [P(CsrView), ctypes.c_int64, ctypes.c_double, P(Options), vp, P(vp)]
    L.sexpm_compute.argtypes = [vp, ctypes.c_double, P(vp)]
    L.sexpm_result_info.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64)]
    L.sexpm_result_copy.argtypes = [vp, vp, vp, vp, ctypes.c_int32]
    L.sexpm_stats.argtypes = [vp, P(Stats), P(StepStats), ctypes.c_int32]
    L.sexpm_result_free.argtypes = [vp]
    L.sexpm_result_free.restype = None
    L.sexpm_plan_destroy.argtypes = [vp]
    L.sexpm_plan_destroy.restype = None
    L.sexpm_kernel_launches.restype = ctypes.c_int64
    L.sexpm_kernel_launches.argtypes = []
    L.sexpm_release_memory.argtypes = []
    L.sexpm_pool_stats.argtypes = [P(ctypes.c_int64), P(ctypes.c_int64)]
    L.sexpm_rho.argtypes = [ctypes.c_int32, ctypes.c_double]
    L.sexpm_rho.restype = ctypes.c_double
    L.sexpm_choose_MN.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                  P(ctypes.c_int32), P(ctypes.c_int32)]
    L.sexpm_spgemm.argtypes = [P(CsrView), P(CsrView), P(CsrView), ctypes.c_double, ctypes.c_double, vp, P(vp),
                               P(ctypes.c_int64)]
    L.sexpm_filter.argtypes = [P(CsrView), ctypes.c_double, ctypes.c_double, ctypes.c_int32, vp, P(vp),
                               P(ctypes.c_double), P(ctypes.c_int32), P(ctypes.c_double)]
    L.sexpm_plan_batched.argtypes = [P(CsrView), ctypes.c_int32, ctypes.c_double, P(Options), vp, P(vp)]
    L.sexpm_compute_batched.argtypes = [vp, P(ctypes.c_double), P(vp)]
    L.sexpm_plan_z.argtypes = [P(CsrView), ctypes.c_int64, ctypes.c_double, P(Options), vp, P(vp)]
    L.sexpm_result_is_complex.argtypes = [vp, P(ctypes.c_int32)]
    L.sexpm_result_copy_z.argtypes = [vp, vp, vp, vp, ctypes.c_int32]
    L.sexpm_batched_graph_info.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_int32),
                                           P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_int64)]
    L.sexpm_tune_batched.argtypes = [vp, P(ctypes.c_double), ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                     P(ctypes.c_double), P(ctypes.c_int32)]
    L.sexpm_adjoint.argtypes = [vp, ctypes.c_double, P(CsrView), ctypes.c_int32, P(vp), P(vp)]
    L.sexpm_forward_keep.argtypes = [vp, ctypes.c_double, ctypes.c_int32, P(vp), P(vp)]
    L.sexpm_transpose.argtypes = [P(CsrView), vp, P(vp)]
    L.sexpm_power_norms.argtypes = [P(CsrView), ctypes.c_int32, vp, P(ctypes.c_double)]
    L.sexpm_alpha_hat.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  P(ctypes.c_double), ctypes.c_int32, P(ctypes.c_int32)]
    L.sexpm_choose_MN_refined.argtypes = [ctypes.c_double, P(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32)]
    L.sexpm_result_spmm.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    L.sexpm_propagate.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    L.sexpm_spmm.argtypes = [P(CsrView), vp, ctypes.c_int64, vp, vp]
    L.sexpm_filter_pass.argtypes = [P(CsrView), ctypes.c_double, vp, P(ctypes.c_double), P(ctypes.c_int64)]
    L.sexpm_filter_apply.argtypes = [P(CsrView), ctypes.c_double, vp, P(vp)]
    L.sexpm_norm2_I_plus_rows.argtypes = [P(CsrView), ctypes.c_int64, ctypes.c_int64, vp, P(ctypes.c_double)]
    L.sexpm_adjoint_tape.argtypes = [vp, P(CsrView), P(vp)]
    L.sexpm_tape_free.argtypes = [vp]
    L.sexpm_tape_free.restype = None
    L.sexpm_filter_noalloc.argtypes = [P(CsrView), ctypes.c_double, ctypes.c_double, ctypes.c_int32, vp, vp, vp, vp,
                                       ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_int32),
                                       P(ctypes.c_double)]
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != SEXPM_OK:
        raise SexpmError(rc, load().sexpm_last_error().decode())


def _stream_ptr(stream=None) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ------------------------------------------------------------------ views

def _is_sparse_csr(H) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(H, torch.Tensor) and H.layout == torch.sparse_csr


def _arrays(H) -> Tuple[Any, Any, Any, int]:
    """Accepts a square 2-D torch.sparse_csr tensor, (row_ptr, col, val[, n]) tuples, or objects
    with row_ptr/col/val/n attributes."""
    if _is_sparse_csr(H):
        if H.dim() != 2 or H.shape[0] != H.shape[1]:
            raise ValueError("a square 2-D sparse CSR tensor is required")
        return H.crow_indices(), H.col_indices(), H.values(), int(H.shape[0])
    if isinstance(H, (tuple, list)):
        rp, ci, v = H[0], H[1], H[2]
        n = H[3] if len(H) > 3 else len(rp) - 1
    else:
        rp, ci, v, n = H.row_ptr, H.col, H.val, H.n
    return rp, ci, v, int(n)


def _make_view(H, keep: List[Any]) -> CsrView:
    rp, ci, v, n = _arrays(H)
    try:
        import torch
        is_t = isinstance(rp, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        on_dev = rp.is_cuda
        rp = rp.to(dtype=torch.int64).contiguous()
        ci = ci.to(dtype=torch.int32).contiguous()
        v = v.to(dtype=torch.float64).contiguous()
        if not (rp.is_cuda == ci.is_cuda == v.is_cuda):
            raise ValueError("row_ptr, col and val must live on the same device")
        keep += [rp, ci, v]
        ptrs = (rp.data_ptr(), ci.data_ptr() if ci.numel() else None, v.data_ptr() if v.numel() else None)
        nnz = int(ci.numel())
    else:
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.float64)
        keep += [rp, ci, v]
        on_dev = False
        ptrs = (rp.ctypes.data, ci.ctypes.data if ci.size else None, v.ctypes.data if v.size else None)
        nnz = int(ci.size)
    return CsrView(n, nnz, ptrs[0], ptrs[1], ptrs[2], 1 if on_dev else 0)


def options(**kw) -> Options:
    o = Options()
    _check(load().sexpm_options_default(ctypes.byref(o)))
    for k, val in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, val)
    return o


# ------------------------------------------------------------------ results

class Result:
    """A library-owned device CSR result."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def info(self) -> Tuple[int, int]:
        n, nnz = ctypes.c_int64(), ctypes.c_int64()
        _check(load().sexpm_result_info(self._h, ctypes.byref(n), ctypes.byref(nnz)))
        return n.value, nnz.value

    def to_torch(self, device="cuda"):
        import torch
        n, nnz = self.info()
        rp = torch.empty(n + 1, dtype=torch.int64, device=device)
        ci = torch.empty(nnz, dtype=torch.int32, device=device)
        v = torch.empty(nnz, dtype=torch.float64, device=device)
        on_dev = 1 if rp.is_cuda else 0
        if on_dev:
            torch.cuda.current_stream().synchronize()
        _check(load().sexpm_result_copy(self._h, rp.data_ptr(), ci.data_ptr() if nnz else None,
                                        v.data_ptr() if nnz else None, on_dev))
        return rp, ci, v

    def to_numpy(self):
        n, nnz = self.info()
        rp = np.empty(n + 1, dtype=np.int64)
        ci = np.empty(nnz, dtype=np.int32)
        v = np.empty(nnz, dtype=np.float64)
        _check(load().sexpm_result_copy(self._h, rp.ctypes.data, ci.ctypes.data if nnz else None,
                                        v.ctypes.data if nnz else None, 0))
        return rp, ci, v

    def spmm(self, X):
        """E X for a device block X (n x r float64 torch tensor, or a length-n vector):
        sexpm_result_spmm."""
        import torch
        vec = X.dim() == 1
        X2 = X.reshape(X.shape[0], -1).to(torch.float64).contiguous()
        Y = torch.empty_like(X2)
        _check(load().sexpm_result_spmm(self._h, X2.data_ptr(), X2.shape[1], Y.data_ptr(), _stream_ptr()))
        return Y.reshape(-1) if vec else Y

    def propagate(self, U0, steps: int):
        """E^steps U0 by time stepping U_k = E U_{k-1} (sexpm_propagate)."""
        import torch
        vec = U0.dim() == 1
        U2 = U0.reshape(U0.shape[0], -1).to(torch.float64).contiguous()
        out = torch.empty_like(U2)
        _check(load().sexpm_propagate(self._h, U2.data_ptr(), U2.shape[1], int(steps), out.data_ptr(),
                                      _stream_ptr()))
        return out.reshape(-1) if vec else out

    def stats(self) -> Dict[str, Any]:
        st = Stats()
        steps = (StepStats * 512)()
        _check(load().sexpm_stats(self._h, ctypes.byref(st), steps, 512))
        d = {f: getattr(st, f) for f, _ in Stats._fields_}
        d["steps"] = [{f: (list(getattr(steps[k], f)) if f == "rows_class" else getattr(steps[k], f))
                       for f, _ in StepStats._fields_} for k in range(min(st.n_steps, 512))]
        return d

    def free(self) -> None:
        if self._h:
            load().sexpm_result_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Plan:
    """sexpm_plan: H copied to the device, ||H||_F and normality computed on the GPU."""

    def __init__(self, H, eps: float, stream=None, **opts):
        keep: List[Any] = []
        view = _make_view(H, keep)
        self._stream = _stream_ptr(stream)
        h = ctypes.c_void_p()
        o = options(**opts)
        _check(load().sexpm_plan(ctypes.byref(view), view.n, float(eps), ctypes.byref(o), self._stream,
                                 ctypes.byref(h)))
        self._h = h
        self.n = view.n

    def compute(self, tau: float = 1.0) -> Result:
        r = ctypes.c_void_p()
        _check(load().sexpm_compute(self._h, float(tau), ctypes.byref(r)))
        return Result(r.value)

    def forward_keep(self, tau: float = 1.0, ckpt_stride: int = 0) -> Tuple["Tape", Result]:
        """sexpm_forward_keep: e^{tau H} (every product formed) and a Tape holding the checkpoints
        its reverse pass needs."""
        t, r = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().sexpm_forward_keep(self._h, float(tau), int(ckpt_stride), ctypes.byref(r), ctypes.byref(t)))
        return Tape(t.value, self), Result(r.value)

    def close(self) -> None:
        if self._h:
            load().sexpm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tape:
    """A kept forward run (sexpm_forward_keep); adjoint(W) runs the reverse pass (sexpm_adjoint_tape).
    Holds a reference to its plan, which must stay open while the tape is alive."""

    def __init__(self, handle: int, plan: Plan):
        self._h = ctypes.c_void_p(handle)
        self.plan = plan

    def adjoint(self, W, device="cuda"):
        """dL/dH on the stored pattern of H for dL/dE = W: (row_ptr, col, val) torch tensors."""
        keep: List[Any] = []
        w = _make_view(W, keep)
        r = ctypes.c_void_p()
        _check(load().sexpm_adjoint_tape(self._h, ctypes.byref(w), ctypes.byref(r)))
        res = Result(r.value)
        try:
            return res.to_torch(device)
        finally:
            res.free()

    def free(self) -> None:
        if self._h:
            load().sexpm_tape_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def expm(H, tau: float = 1.0, eps: float = 1e-12, device="cuda", **opts):
    """e^{tau H} as (row_ptr, col, val) torch tensors on `device`, plus the stats dict.  When H is
    a torch.sparse_csr tensor, e^{tau H} is returned as one too (float64, int64 indices)."""
    plan = Plan(H, eps, **opts)
    try:
        res = plan.compute(tau)
        try:
            release_memory()  # the pool's cached working memory goes back before the copy is allocated
            out = res.to_torch(device)
            st = res.stats()
        finally:
            res.free()
    finally:
        plan.close()
    if _is_sparse_csr(H):
        import torch
        rp, ci, v = out
        n = rp.numel() - 1
        out = torch.sparse_csr_tensor(rp, ci.to(torch.int64), v, size=(n, n))
    return out, st


def _make_view_z(H, keep: List[Any]) -> CsrView:
    """A complex CSR view: val holds complex128 entries ((re, im) pairs of doubles)."""
    rp, ci, v, n = _arrays(H)
    try:
        import torch
        is_t = isinstance(rp, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        on_dev = rp.is_cuda
        rp = rp.to(dtype=torch.int64).contiguous()
        ci = ci.to(dtype=torch.int32).contiguous()
        v = v.to(dtype=torch.complex128).contiguous()
        if not (rp.is_cuda == ci.is_cuda == v.is_cuda):
            raise ValueError("row_ptr, col and val must live on the same device")
        keep += [rp, ci, v]
        ptrs = (rp.data_ptr(), ci.data_ptr() if ci.numel() else None, v.data_ptr() if v.numel() else None)
        nnz = int(ci.numel())
    else:
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.complex128)
        keep += [rp, ci, v]
        on_dev = False
        ptrs = (rp.ctypes.data, ci.ctypes.data if ci.size else None, v.ctypes.data if v.size else None)
        nnz = int(ci.size)
    return CsrView(n, nnz, ptrs[0], ptrs[1], ptrs[2], 1 if on_dev else 0)


class ComplexPlan(Plan):
    """sexpm_plan_z: complex H ((row_ptr, col, val complex128[, n]) as torch tensors or numpy
    arrays); compute() gives results whose to_torch() returns complex128 values."""

    def __init__(self, H, eps: float, stream=None, **opts):  # noqa: D107 (Plan.__init__ not reused)
        keep: List[Any] = []
        view = _make_view_z(H, keep)
        self._stream = _stream_ptr(stream)
        h = ctypes.c_void_p()
        o = options(**opts)
        _check(load().sexpm_plan_z(ctypes.byref(view), view.n, float(eps), ctypes.byref(o), self._stream,
                                   ctypes.byref(h)))
        self._h = h
        self.n = view.n

    def compute(self, tau: float = 1.0) -> "ComplexResult":
        r = ctypes.c_void_p()
        _check(load().sexpm_compute(self._h, float(tau), ctypes.byref(r)))
        return ComplexResult(r.value)


class ComplexResult(Result):
    """A library-owned complex result (sexpm_result_copy_z)."""

    def to_torch(self, device="cuda"):
        import torch
        n, nnz = self.info()
        rp = torch.empty(n + 1, dtype=torch.int64, device=device)
        ci = torch.empty(nnz, dtype=torch.int32, device=device)
        v = torch.empty(nnz, dtype=torch.complex128, device=device)
        on_dev = 1 if rp.is_cuda else 0
        if on_dev:
            torch.cuda.current_stream().synchronize()
        _check(load().sexpm_result_copy_z(self._h, rp.data_ptr(), ci.data_ptr() if nnz else None,
                                          v.data_ptr() if nnz else None, on_dev))
        return rp, ci, v


def expm_complex(H, tau: float = 1.0, eps: float = 1e-12, device="cuda", **opts):
    """e^{tau H} for complex H as (row_ptr, col, val complex128) torch tensors on `device`, plus
    the stats dict."""
    plan = ComplexPlan(H, eps, **opts)
    try:
        res = plan.compute(tau)
        try:
            out = res.to_torch(device)
            st = res.stats()
        finally:
            res.free()
    finally:
        plan.close()
    return out, st


class BatchedPlan:
    """sexpm_plan_batched: many matrices planned as one block-diagonal problem."""

    def __init__(self, Hs, eps: float, stream=None, **opts):
        keep: List[Any] = []
        views = (CsrView * len(Hs))(*[_make_view(H, keep) for H in Hs])
        self.count = len(Hs)
        self._stream = _stream_ptr(stream)
        h = ctypes.c_void_p()
        o = options(**opts)
        _check(load().sexpm_plan_batched(views, self.count, float(eps), ctypes.byref(o), self._stream,
                                         ctypes.byref(h)))
        self._h = h

    def compute(self, taus) -> List[Result]:
        taus = (ctypes.c_double * self.count)(*[float(t) for t in taus])
        outs = (ctypes.c_void_p * self.count)()
        _check(load().sexpm_compute_batched(self._h, taus, outs))
        return [Result(outs[k]) for k in range(self.count)]

    def graph_info(self) -> dict:
        """sexpm_batched_graph_info: the captured squaring step's arena and counters."""
        ab, kps, kpp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        cap, rer, hst = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().sexpm_batched_graph_info(self._h, ctypes.byref(ab), ctypes.byref(cap), ctypes.byref(rer),
                                               ctypes.byref(hst), ctypes.byref(kps), ctypes.byref(kpp)))
        return {"arena_bytes": ab.value, "captures": cap.value, "reruns": rer.value, "host_steps": hst.value,
                "kernels_per_step": kps.value, "kernels_per_pass": kpp.value}

    def tune(self, taus, candidates=None):
        """sexpm_tune_batched over [(ks_bytes, wide), ...] (None: the library's list); returns
        (squaring ms per candidate, index chosen)."""
        taus_c = (ctypes.c_double * self.count)(*[float(t) for t in taus])
        nc = len(candidates) if candidates else 0
        ks = (ctypes.c_int32 * max(nc, 1))(*[int(c[0]) for c in candidates or []])
        wd = (ctypes.c_int32 * max(nc, 1))(*[int(c[1]) for c in candidates or []])
        ms = (ctypes.c_double * (nc if nc else 4))()
        best = ctypes.c_int32()
        _check(load().sexpm_tune_batched(self._h, taus_c, nc, ks, wd, ms, ctypes.byref(best)))
        return list(ms), best.value

    def close(self) -> None:
        if self._h:
            load().sexpm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def expm_batched(Hs, taus, eps: float = 1e-12, device="cuda", **opts):
    """[e^{tau_b H_b}] as a list of ((row_ptr, col, val), stats) through the batched entry points."""
    plan = BatchedPlan(Hs, eps, **opts)
    try:
        out = []
        for r in plan.compute(taus):
            try:
                out.append((r.to_torch(device), r.stats()))
            finally:
                r.free()
    finally:
        plan.close()
    return out


def adjoint(H, tau: float, eps: float, W, ckpt_stride: int = 0, device="cuda", want_expm: bool = False, **opts):
    """dL/dH on the pattern of H for dL/dE = W (E = e^{tau H}) through sexpm_adjoint.
    Returns (row_ptr, col, val) of dH (and ((row_ptr, col, val), stats) of E if want_expm)."""
    plan = H if isinstance(H, Plan) else Plan(H, eps, **opts)
    keep: List[Any] = []
    w = _make_view(W, keep)
    r, e = ctypes.c_void_p(), ctypes.c_void_p()
    try:
        _check(load().sexpm_adjoint(plan._h, float(tau), ctypes.byref(w), int(ckpt_stride), ctypes.byref(r),
                                    ctypes.byref(e) if want_expm else None))
        res = Result(r.value)
        try:
            g = res.to_torch(device)
            st = res.stats()
        finally:
            res.free()
        if want_expm:
            er = Result(e.value)
            try:
                return g, (er.to_torch(device), er.stats())
            finally:
                er.free()
        return g
    finally:
        if plan is not H:
            plan.close()


def spgemm(A, B, D=None, div: float = 1.0, beta: float = 0.0, device="cuda"):
    """C = (A B)/div + beta D through sexpm_spgemm; returns ((row_ptr, col, val), products)."""
    keep: List[Any] = []
    a, b = _make_view(A, keep), _make_view(B, keep)
    d = _make_view(D, keep) if D is not None else None
    r = ctypes.c_void_p()
    prod = ctypes.c_int64()
    _check(load().sexpm_spgemm(ctypes.byref(a), ctypes.byref(b), ctypes.byref(d) if d is not None else None,
                               float(div), float(beta), _stream_ptr(), ctypes.byref(r), ctypes.byref(prod)))
    res = Result(r.value)
    try:
        return res.to_torch(device), prod.value
    finally:
        res.free()


def spgemm_rows_per_class(A, B, D=None, div: float = 1.0, beta: float = 0.0) -> List[int]:
    """Rows of the numeric pass of sexpm_spgemm per size class (shared memory 8, 24, 56, 112 and
    220 KB, then global memory), from the step record of its result."""
    keep: List[Any] = []
    a, b = _make_view(A, keep), _make_view(B, keep)
    d = _make_view(D, keep) if D is not None else None
    r = ctypes.c_void_p()
    prod = ctypes.c_int64()
    _check(load().sexpm_spgemm(ctypes.byref(a), ctypes.byref(b), ctypes.byref(d) if d is not None else None,
                               float(div), float(beta), _stream_ptr(), ctypes.byref(r), ctypes.byref(prod)))
    res = Result(r.value)
    try:
        return list(res.stats()["steps"][0]["rows_class"])
    finally:
        res.free()


def filter_csr(A, eps_g: float, e_r: float = 0.1, max_iters: int = 100, device="cuda"):
    """Algorithm 4.1 through sexpm_filter; returns ((row_ptr, col, val), t, iters, b)."""
    keep: List[Any] = []
    a = _make_view(A, keep)
    r = ctypes.c_void_p()
    t, it, b = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
    _check(load().sexpm_filter(ctypes.byref(a), float(eps_g), float(e_r), int(max_iters), _stream_ptr(),
                               ctypes.byref(r), ctypes.byref(t), ctypes.byref(it), ctypes.byref(b)))
    res = Result(r.value)
    try:
        return res.to_torch(device), t.value, it.value, b.value
    finally:
        res.free()


def spmm(A, X):
    """A X for a CSR A (copied to the device) and a device block X (n x r float64): sexpm_spmm."""
    import torch
    keep: List[Any] = []
    a = _make_view(A, keep)
    vec = X.dim() == 1
    X2 = X.reshape(X.shape[0], -1).to(torch.float64).contiguous()
    Y = torch.empty_like(X2)
    _check(load().sexpm_spmm(ctypes.byref(a), X2.data_ptr(), X2.shape[1], Y.data_ptr(), _stream_ptr()))
    return Y.reshape(-1) if vec else Y


def transpose(A, device="cuda"):
    """A^T (sexpm_transpose) as (row_ptr, col, val) torch tensors."""
    keep: List[Any] = []
    a = _make_view(A, keep)
    r = ctypes.c_void_p()
    _check(load().sexpm_transpose(ctypes.byref(a), _stream_ptr(), ctypes.byref(r)))
    res = Result(r.value)
    try:
        return res.to_torch(device)
    finally:
        res.free()


def filter_pass(A, t: float) -> Tuple[float, int]:
    """One Algorithm 4.1 pass (sexpm_filter_pass): (sum of v^2 over |v| <= t, entries with |v| > t)."""
    keep: List[Any] = []
    a = _make_view(A, keep)
    sd, kept = ctypes.c_double(), ctypes.c_int64()
    _check(load().sexpm_filter_pass(ctypes.byref(a), float(t), _stream_ptr(), ctypes.byref(sd), ctypes.byref(kept)))
    return sd.value, kept.value


def filter_apply(A, t: float, device="cuda"):
    """The entries of A with |v| > t (sexpm_filter_apply) as (row_ptr, col, val) torch tensors."""
    keep: List[Any] = []
    a = _make_view(A, keep)
    r = ctypes.c_void_p()
    _check(load().sexpm_filter_apply(ctypes.byref(a), float(t), _stream_ptr(), ctypes.byref(r)))
    res = Result(r.value)
    try:
        return res.to_torch(device)
    finally:
        res.free()


def norm2_I_plus_rows(A, r0: int, r1: int) -> float:
    """sum over rows r0..r1-1 of sum_j (delta_ij + a_ij)^2 (sexpm_norm2_I_plus_rows)."""
    keep: List[Any] = []
    a = _make_view(A, keep)
    out = ctypes.c_double()
    _check(load().sexpm_norm2_I_plus_rows(ctypes.byref(a), int(r0), int(r1), _stream_ptr(), ctypes.byref(out)))
    return out.value


NOALLOC_MAX_ROWS = 1048576


def filter_noalloc(A, eps_g: float, e_r: float = 0.1, max_iters: int = 100, out=None):
    """Algorithm 4.1 through sexpm_filter_noalloc, which allocates nothing itself.

    A holds device tensors; `out` = (row_ptr[n+1], col[cap], val[cap]) device tensors (allocated
    here with torch when omitted).  Returns ((row_ptr, col[:nnz], val[:nnz]), t, iters, b)."""
    import torch
    keep: List[Any] = []
    a = _make_view(A, keep)
    if out is None:
        cap = max(1, a.nnz)
        out = (torch.empty(a.n + 1, dtype=torch.int64, device="cuda"),
               torch.empty(cap, dtype=torch.int32, device="cuda"),
               torch.empty(cap, dtype=torch.float64, device="cuda"))
    rp, ci, v = out
    nnz, t, it, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
    _check(load().sexpm_filter_noalloc(ctypes.byref(a), float(eps_g), float(e_r), int(max_iters), _stream_ptr(),
                                       rp.data_ptr(), ci.data_ptr(), v.data_ptr(), int(ci.numel()),
                                       ctypes.byref(nnz), ctypes.byref(t), ctypes.byref(it), ctypes.byref(b)))
    return (rp, ci[:nnz.value], v[:nnz.value]), t.value, it.value, b.value


def kernel_launches() -> int:
    """Kernels enqueued by the library since it was loaded."""
    return int(load().sexpm_kernel_launches())


def release_memory() -> None:
    """Return the library's cached device memory to the driver."""
    _check(load().sexpm_release_memory())


def pool_stats() -> Tuple[int, int]:
    """(live, peak) bytes the library holds from its device pool (sexpm_pool_stats)."""
    live, peak = ctypes.c_int64(), ctypes.c_int64()
    _check(load().sexpm_pool_stats(ctypes.byref(live), ctypes.byref(peak)))
    return live.value, peak.value


def rho(M: int, x: float) -> float:
    """Eq. (4.5), evaluated by the library's host code."""
    return load().sexpm_rho(int(M), float(x))


def power_norms(H, kmax: int) -> List[float]:
    """||H^k||_F for k = 1..kmax from exact sparse powers on the GPU (sexpm_power_norms)."""
    keep: List[Any] = []
    a = _make_view(H, keep)
    out = (ctypes.c_double * int(kmax))()
    _check(load().sexpm_power_norms(ctypes.byref(a), int(kmax), _stream_ptr(), out))
    return list(out)


def alpha_hat(norm_H: float, M: int, N: int, i: int, pnorms=None) -> int:
    """alpha^_i of Eq. (4.8) (pnorms None) or Eq. (4.9) (sexpm_alpha_hat, host)."""
    a = ctypes.c_int32()
    arr = (ctypes.c_double * len(pnorms))(*pnorms) if pnorms is not None else None
    _check(load().sexpm_alpha_hat(float(norm_H), int(M), int(N), int(i), arr, len(pnorms) if pnorms else 0,
                                  ctypes.byref(a)))
    return a.value


def choose_MN_refined(norm_H: float, pnorms, eps: float, n_extra: int = 50) -> Tuple[int, int]:
    """Eq. (4.20)'s rule on the refined norm h_{M,N} (sexpm_choose_MN_refined, host)."""
    M, N = ctypes.c_int32(), ctypes.c_int32()
    arr = (ctypes.c_double * len(pnorms))(*pnorms)
    _check(load().sexpm_choose_MN_refined(float(norm_H), arr, len(pnorms), float(eps), int(n_extra),
                                          ctypes.byref(M), ctypes.byref(N)))
    return M.value, N.value


def choose_MN(norm_H: float, eps: float, n_extra: int = 50, max_M: int = 1000) -> Tuple[int, int]:
    """Eq. (4.20), evaluated by the library's host code."""
    M, N = ctypes.c_int32(), ctypes.c_int32()
    _check(load().sexpm_choose_MN(float(norm_H), float(eps), int(n_extra), int(max_M), ctypes.byref(M),
                                  ctypes.byref(N)))
    return M.value, N.value


def _autograd_class():
    import torch

    class SexpmFn(torch.autograd.Function):
        """e^{tau H} with a gradient, for H = beta A where A has the values `values_of_A` on a fixed
        sparse pattern = (row_ptr, col, n).  forward returns the values of E = e^{tau H} and its
        pattern (row_ptr, col; not differentiable); it keeps the forward's checkpoints
        (sexpm_forward_keep), and backward maps dL/d(E values) to dL/dA = beta dL/dH through
        sexpm_adjoint_tape (the filter decisions of the forward held fixed)."""

        @staticmethod
        def forward(ctx, values_of_A, pattern, beta, tau, eps, ckpt_stride=0):
            row_ptr, col, n = pattern
            H = (row_ptr, col, float(beta) * values_of_A.detach(), int(n))
            plan = Plan(H, eps, symmetric=0)
            tape, res = plan.forward_keep(tau, ckpt_stride)
            try:
                erp, eci, ev = res.to_torch(values_of_A.device)
            finally:
                res.free()
            ctx.tape, ctx.beta, ctx.n = tape, float(beta), int(n)
            ctx.save_for_backward(erp, eci)
            ctx.mark_non_differentiable(erp, eci)
            return ev, erp, eci

        @staticmethod
        def backward(ctx, g_ev, g_erp=None, g_eci=None):
            erp, eci = ctx.saved_tensors
            tape = ctx.tape
            try:
                _, _, g = tape.adjoint((erp, eci, g_ev.contiguous(), ctx.n), device=g_ev.device)
            finally:
                plan = tape.plan
                tape.free()
                plan.close()
                ctx.tape = None
            return ctx.beta * g, None, None, None, None, None

    return SexpmFn


_sexpm_fn = None


def sexpm_fn():
    """The torch.autograd.Function SexpmFn: SexpmFn.apply(values_of_A, (row_ptr, col, n), beta, tau, eps
    [, ckpt_stride]) -> (E values, E row_ptr, E col)."""
    global _sexpm_fn
    if _sexpm_fn is None:
        _sexpm_fn = _autograd_class()
    return _sexpm_fn


def expm_autograd(h_val, row_ptr, col, n, tau, eps, ckpt_stride=0):
    """Differentiable e^{tau H} for H given by its values h_val on (row_ptr, col): returns
    (E values, E row_ptr, E col); gradients flow to h_val."""
    return sexpm_fn().apply(h_val, (row_ptr, col, int(n)), 1.0, tau, eps, ckpt_stride)


def edge_pattern(edge_index, n: int):
    """Symmetric CSR pattern of an undirected graph given by its edges (2 x m, u != v, each edge
    once): returns (row_ptr int64, col int32, entry_edge int64), entry_edge[p] the edge of stored
    entry p (both (u, v) and (v, u) map to the same edge)."""
    ei = np.asarray(edge_index, dtype=np.int64)
    m = ei.shape[1]
    rows = np.concatenate([ei[0], ei[1]])
    cols = np.concatenate([ei[1], ei[0]])
    eid = np.concatenate([np.arange(m), np.arange(m)])
    order = np.lexsort((cols, rows))
    rows, cols, eid = rows[order], cols[order], eid[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), eid


def expm_edges(w, edge_index, n: int, beta: float, tau: float, eps: float, ckpt_stride: int = 0):
    """e^{tau beta A} for the symmetric weighted adjacency A of an undirected graph with edge
    weights w (torch tensor, one per edge of edge_index, 2 x m): returns (E values, E row_ptr,
    E col); dL/dw_e = beta (dL/dH_uv + dL/dH_vu) flows back to w."""
    import torch
    rp, ci, eid = edge_pattern(edge_index, n)
    dev = w.device
    vals = w[torch.from_numpy(eid).to(dev)]
    return sexpm_fn().apply(vals, (torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), int(n)), beta, tau, eps,
                            ckpt_stride)
