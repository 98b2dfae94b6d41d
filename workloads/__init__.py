"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This package only builds input matrices and seeds; it performs none of the
matrix-exponential method's arithmetic, so the CUDA path and the CPU oracle
can both draw their inputs from it without sharing any computation.
"""
from .generators import (  # noqa: F401
    BATCH_EPS,
    CSR,
    CONFIGS,
    Config,
    batch_instances,
    diag_scale,
    diag_weights,
    dirichlet_laplacian,
    get_config,
    laplacian_batch,
    paper_table1_matrices,
    random_csr,
    rgg_adjacency,
    sparse_loss_weights,
    spring_lattice,
    theta_lattice,
    theta_matrix,
    toeplitz_trid,
)
