"""Seeded synthetic inputs for supernodal selected inversion.

This package only builds test and benchmark matrices (values, sparsity
pattern and a fill-reducing symmetric ordering).  It holds none of the
selected-inversion arithmetic: no elimination tree, no factorization, no
inverse.  Both the CPU oracle (``oracle/``) and the GPU library consume what
it produces.
"""
from .problems import (  # noqa: F401
    Problem,
    laplacian_2d,
    laplacian_3d,
    dft_sheet,
    diffusion_3d,
    pole_shifts,
    batch_laplacians,
    random_sparse_spd,
    random_sparse_hpd,
    magnetic_laplacian_3d,
    random_sparse_nonsym,
    symmetric_scaling,
    tridiagonal,
    make_config,
    lower_pattern_weights,
)
