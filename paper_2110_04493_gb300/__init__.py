"""GB300 (sm_103a) implementation of the filtered incremental scaling-and-squaring
method for a large sparse matrix exponential (arXiv 2110.04493).

The compute path lives in libsexpm.so (CUDA kernels behind the C ABI of
include/sexpm.h); :mod:`paper_2110_04493_gb300.sexpm` is its Python binding.
"""
from .sexpm import (  # noqa: F401
    BatchedPlan,
    ComplexPlan,
    ComplexResult,
    Plan,
    Result,
    adjoint,
    SexpmError,
    choose_MN,
    expm,
    expm_autograd,
    expm_batched,
    expm_complex,
    filter_csr,
    load,
    rho,
    spgemm,
)
