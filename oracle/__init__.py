"""FP64 CPU oracle for chain TV and 2D TV-l2 (ROF) denoising.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers. It shares no code with the CUDA library
and never imports it.
"""
from .oracle import (  # noqa: F401
    build,
    chain_solve,
    chain_solve_batch,
    chain_solve_general,
    chain_solve_nonconvex,
    chain_solve_pq,
    chain_vjp,
    rof_primal,
    tv2d_l1,
    tv2d_lagrangian,
    tv2d_pd,
)
