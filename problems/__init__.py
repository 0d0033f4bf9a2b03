"""Seeded synthetic linear systems Ax = b used by the tests and the benchmark.

This package only *builds problem instances* (sparse matrices in CSR form and
right-hand sides).  It contains none of the solver's arithmetic, so both the
CPU oracle and the CUDA path can be fed from it without sharing method code.

The paper evaluates on SuiteSparse / HPCG / HPGMP matrices (Sec. 5, Table 2);
those are not available here, so seeded stencil generators with the shapes and
coefficient laws of the target workloads stand in for them.
"""
from .generators import (  # noqa: F401
    Problem,
    poisson2d_5pt,
    diffusion3d_7pt,
    convdiff3d_27pt,
    diffusion27_nodal,
    hpcg_27pt,
    batched_diffusion_systems,
    random_dd_sparse,
    rhs_uniform01,
    by_name,
)
from .rng import uniform01, normal, stream_seed  # noqa: F401
