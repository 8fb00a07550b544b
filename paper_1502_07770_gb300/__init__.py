"""GB300-native total variation on chains and 2D TV-l2 denoising.

Implements the O(n) chain dynamic program of "Total variation on a tree"
(Algorithm 2 with the quadratic-unary specialisation of Sec. 4.1) as batched
sm_103a CUDA kernels behind a C ABI (``include/tv.h``), and the paper's 2D
Lagrangian-decomposition primal-dual ROF solver (Sec. 6.1) built on it, with
general and piecewise-quadratic chains (Sec. 4.2) and 2D TV-l1 denoising (Sec. 6).

The CUDA binding is imported lazily so that ``synth`` (input generators) can
be used without a GPU.
"""
_LIB_NAMES = ("chain_prox", "chain_prox_columns", "chain_prox_backward", "chain_prox_diff",
              "chain_prox_general", "chain_prox_pq", "chain_prox_nonconvex", "ChainProxFn",
              "tv2d_denoise", "tv2d_denoise_batched", "tv2d_denoise_lagrangian", "tv2d_denoise_l1",
              "workspace_status")
__all__ = list(_LIB_NAMES) + ["synth", "autotune"]


def __getattr__(name):
    if name in _LIB_NAMES or name in ("load", "TVError"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
