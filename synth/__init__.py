"""Seeded synthetic inputs for the norm-1 ADMM imaging problem g = Hu + w.

This module is shared by the FP64 CPU oracle (``oracle/``), the CUDA library's
tests and ``bench.py``.  It only *creates* problem instances (sensing matrix H,
sparse scene u, noise w, the regularisation weight and the augmented
parameter); it performs none of the ADMM method's arithmetic.
"""

from .workloads import (  # noqa: F401
    Problem,
    gaussian_problem,
    chunked_gaussian_rows,
    chunked_gaussian_problem,
    ROWS_PER_DRAW,
    cra_matrix,
    plate_scene,
    noisy_measurements,
    cra_problem,
    lambda_from_fraction,
    spectral_norm_sq,
    sectioning_rho,
    round_to_c64,
    CONFIG1,
    CONFIG2,
    CONFIG3,
    TALL,
    gaussian_problem_device,
    shared_h_scenes,
    uneven_problem_sizes,
)
