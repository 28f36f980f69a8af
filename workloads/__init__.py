"""Seeded synthetic inputs for the truncated Neumann series S_k(A).

This package only draws random matrices with the shapes and spectra of the
paper's workloads (Sec. 6 "Setup": A = alpha * Omega D Omega^T with D in
[-1, 1]); it holds none of the series arithmetic. Both the CPU oracle and the
CUDA path take their inputs from here.
"""

from .generators import (  # noqa: F401
    GEN_VERSION,
    gaussian_scaled,
    planted_symmetric,
    planted_perturbed,
    jacobi_batch,
    nonnormal_triangular,
    rational_small,
    config_inputs,
)
