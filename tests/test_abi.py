"""CPU-only checks of the C ABI: the library loads, exports every declared symbol,
and its host-side scalar code (Eq. 4.5, Eq. 4.20) matches the mathematics.
No GPU call is made here."""
import ctypes
import decimal
import math
import os
import re

import numpy as np
import pytest

from oracle import sexpm_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sexpm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2110_04493_gb300 import build as B
    B.build()
    from paper_2110_04493_gb300 import sexpm
    return sexpm.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sexpm_[a-z_A-Z0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["sexpm_plan", "sexpm_compute", "sexpm_result_info", "sexpm_result_copy", "sexpm_stats",
                     "sexpm_result_free", "sexpm_plan_destroy", "sexpm_last_error", "sexpm_spgemm", "sexpm_filter"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in _declared_functions() if not hasattr(lib, f)]
    assert missing == []


def test_options_default(lib):
    from paper_2110_04493_gb300 import sexpm
    o = sexpm.options()
    assert (o.e_r, o.square_scale, o.normal_override, o.max_filter_iters, o.n_extra, o.symmetric, o.row_order) == \
        (0.1, 1, -1, 100, 50, 1, 1)
    assert (o.batched_graph, o.batch_arena_bytes, o.scaling, o.refine_kmax) == (1, 0, 0, 41)


def _rho_closed(M, x):
    with decimal.localcontext() as ctx:
        ctx.prec = 250
        X = decimal.Decimal(repr(x))
        s, term = decimal.Decimal(0), decimal.Decimal(1)
        for k in range(M + 1):
            if k:
                term = term * (-X) / k
            s += term
        return float((X.exp() * s - 1) * (-1 if M % 2 else 1))


@pytest.mark.parametrize("M,x", [(1, 0.5), (7, 0.0245), (15, 0.6), (20, 0.95664), (30, 1.0), (12, 2.5)])
def test_host_rho_is_eq_4_5(lib, M, x):
    from paper_2110_04493_gb300 import sexpm
    assert sexpm.rho(M, x) == pytest.approx(_rho_closed(M, x), rel=1e-13)


def test_host_choose_MN_reproduces_sec_5_2(lib):
    from paper_2110_04493_gb300 import sexpm
    assert sexpm.choose_MN(244.94489, 1e-16) == (20, 8)
    assert sexpm.choose_MN(0.0, 1e-12) == (0, 0)


def test_host_choose_MN_agrees_with_oracle_over_a_sweep(lib):
    """Two independent codings of Eq. (4.20); the oracle's is pinned to the paper."""
    from paper_2110_04493_gb300 import sexpm
    for k in range(60):
        normH = 10 ** (-3 + 9 * k / 59)
        for eps in (1e-6, 1e-12, 1e-16):
            assert sexpm.choose_MN(normH, eps) == O.choose_MN(normH, eps), (normH, eps)


def test_host_choose_MN_rejects_bad_input(lib):
    from paper_2110_04493_gb300 import sexpm
    for bad in [(1.0, 0.0), (1.0, -1.0), (float("nan"), 1e-12), (1.0, float("inf"))]:
        with pytest.raises(sexpm.SexpmError) as ei:
            sexpm.choose_MN(*bad)
        assert ei.value.code == -1


def test_binding_marshals_a_torch_sparse_csr_tensor():
    """A square torch.sparse_csr tensor is accepted as H: its crow/col/values become the CSR view
    (int64 row pointers, int32 columns, float64 values); other layouts and shapes are rejected."""
    torch = pytest.importorskip("torch")
    import warnings
    from paper_2110_04493_gb300 import sexpm
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        A = torch.tensor([[2.0, 0.0, 1.0], [0.0, 3.0, 0.0], [1.0, 0.0, 4.0]]).to_sparse_csr()
        keep = []
        view = sexpm._make_view(A, keep)
        assert (view.n, view.nnz, view.on_device) == (3, 5, 0)
        rp, ci, v = keep
        assert rp.dtype == torch.int64 and ci.dtype == torch.int32 and v.dtype == torch.float64
        assert rp.tolist() == [0, 2, 3, 5] and ci.tolist() == [0, 2, 1, 0, 2]
        assert v.tolist() == [2.0, 1.0, 3.0, 1.0, 4.0]
        with pytest.raises(ValueError):
            sexpm._arrays(torch.ones(2, 3).to_sparse_csr())


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with libsexpm.so absent, every entry into the method raises ImportError."""
    from paper_2110_04493_gb300 import sexpm
    monkeypatch.setattr(sexpm, "_lib", None)
    monkeypatch.setattr(sexpm, "LIB_PATH", str(tmp_path / "libsexpm.so"))
    with pytest.raises(ImportError):
        sexpm.load()
    with pytest.raises(ImportError):
        sexpm.rho(10, 0.5)
    # the method itself: ImportError for the library, or the CUDA runtime's own error first on a
    # machine without a GPU; never a result
    with pytest.raises((ImportError, RuntimeError)):
        sexpm.expm((np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), np.array([1.0]), 1), 1.0, 1e-12)


def test_host_choose_MN_returns_enoparam_for_an_unreachable_tolerance(lib):
    """No (M, N) in [N0, N0 + n_extra] with M <= max_M meets a tolerance far below what M terms
    reach: SEXPM_ENOPARAM (-5), no output written."""
    import ctypes
    M, N = ctypes.c_int32(-9), ctypes.c_int32(-9)
    rc = lib.sexpm_choose_MN(1e3, 1e-300, 0, 3, ctypes.byref(M), ctypes.byref(N))
    assert rc == -5 and (M.value, N.value) == (-9, -9)


def test_host_alpha_hat_and_refined_choice_match_the_oracle(lib):
    """sexpm_alpha_hat (Eqs. 4.8, 4.9) and sexpm_choose_MN_refined give the oracle's values from the
    same power norms (the Sec. 5.2 Toeplitz matrix, and a 2-D grid Laplacian)."""
    from paper_2110_04493_gb300 import sexpm
    from workloads import dirichlet_laplacian, toeplitz_trid
    H = toeplitz_trid(10_000, 1.0, -2.0, 1.0).to_scipy()
    nH = O.fro_norm(H)
    pn = O.power_norms(H, 81)
    for i in range(0, 9):
        assert sexpm.alpha_hat(nH, 20, 8, i) == O.alpha_hat(nH, 20, 8, i)
        assert sexpm.alpha_hat(nH, 20, 8, i, pn) == O.alpha_hat(nH, 20, 8, i, pn)
    for eps in (1e-16, 1e-12, 1e-8):
        assert sexpm.choose_MN_refined(nH, pn[:41], eps) == O.choose_MN_refined(nH, pn[:41], eps)
    L = dirichlet_laplacian(30, 2).to_scipy() * (2.253 / 31 ** 2)
    nL = O.fro_norm(L)
    pl = O.power_norms(L, 41)
    MN = sexpm.choose_MN_refined(nL, pl, 1e-12)
    assert MN == O.choose_MN_refined(nL, pl, 1e-12)
    assert MN[1] < O.choose_MN(nL, 1e-12)[1]   # the refined norm needs fewer squarings


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/sexpm.h, from a C program compiled with gcc."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"sexpm.h\"\nint main(void) {\n"
    src += f'  printf("%zu\\n", sizeof({struct}));\n'
    for f in fields:
        src += f'  printf("%zu\\n", offsetof({struct}, {f}));\n'
    src += "  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run([gcc, "-std=c99", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("cname,pyname", [("sexpm_options", "Options"), ("sexpm_step_stats", "StepStats"),
                                          ("sexpm_stats_t", "Stats"), ("sexpm_csr_view", "CsrView")])
def test_binding_structs_match_the_header_layout(cname, pyname):
    """The ctypes mirrors of the C structs have the header's size and field offsets (a field added
    on one side only would shift every later field)."""
    from paper_2110_04493_gb300 import sexpm
    py = getattr(sexpm, pyname)
    fields = [f for f, _ in py._fields_ if not f.endswith("_")]
    size, offs = _c_layout(cname, fields)
    assert ctypes.sizeof(py) == size
    assert [getattr(py, f).offset for f in fields] == offs
