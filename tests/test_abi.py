"""The C-ABI library builds, loads and exports what include/*.h declares (no GPU).

Only calls that return before touching the GPU are made here: size queries and
argument validation.
"""
import ctypes
import glob
import os
import re

import pytest

from paper_1502_07770_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(tv\w*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"tv_chain_solve", "tv2d_denoise", "tv_chain_solve_columns"} <= names
    for name in names:
        assert hasattr(lib, name), name
    # the Python binding mirrors exactly the declared C ABI
    assert set(_lib.SIGNATURES) == names


def test_version_and_sizes(lib):
    assert lib.tv_version() >= 100
    n = lib.tv_chain_workspace_size(512, 256)
    # 8 bytes of records per node plus a reserve of 2n+2 breakpoints per chain
    assert n >= 512 * 256 * 8 + (2 * 512 * 256 + 2 * 512) * 8
    assert lib.tv_chain_workspace_size(-1, 3) == 0
    assert lib.tv2d_workspace_size(1024, 1024, 100) > 4 * 1024 * 1024 * 4
    assert lib.tv2d_workspace_size(0, 5, 1) == 0
    assert lib.tv_columns_workspace_size(256, 300) > 0


def test_argument_errors_before_launch(lib):
    dummy = ctypes.c_void_p(0x1000)
    st = lib.tv_chain_solve(dummy, None, 0.1, None, -1, 10, dummy, dummy, 1 << 20, None)
    assert st == _lib.TV_ERR_INVALID and b"num_chains" in lib.tv_last_error()
    st = lib.tv_chain_solve(dummy, None, float("nan"), None, 4, 10, ctypes.c_void_p(0x9000),
                            dummy, 1 << 20, None)
    assert st == _lib.TV_ERR_INVALID and b"lambda" in lib.tv_last_error()
    # x aliasing y
    st = lib.tv_chain_solve(dummy, None, 0.1, None, 4, 10, dummy, ctypes.c_void_p(0x100000),
                            1 << 20, None)
    assert st == _lib.TV_ERR_INVALID
    # workspace too small
    st = lib.tv_chain_solve(dummy, None, 0.1, None, 4, 10, ctypes.c_void_p(0x9000),
                            ctypes.c_void_p(0x100000), 16, None)
    assert st == _lib.TV_ERR_NOMEM
    st = lib.tv_chain_solve_columns(dummy, None, 0.1, 8, 8, 4, ctypes.c_void_p(0x9000), dummy,
                                    1 << 20, None)
    assert st == _lib.TV_ERR_INVALID
    it = ctypes.c_int(0)
    gap = ctypes.c_double(0)
    st = lib.tv2d_denoise(dummy, 0, 8, None, None, 0.1, None, 10, 1e-4, ctypes.c_void_p(0x9000),
                          ctypes.byref(it), ctypes.byref(gap), dummy, 1 << 20, None)
    assert st == _lib.TV_ERR_INVALID
    st = lib.tv2d_denoise(dummy, 8, 8, None, None, 0.1, None, 10, -1.0, ctypes.c_void_p(0x9000),
                          ctypes.byref(it), ctypes.byref(gap), dummy, 1 << 20, None)
    assert st == _lib.TV_ERR_INVALID and b"gap_tol" in lib.tv_last_error()
    # empty batches are a no-op that needs no device
    assert lib.tv_chain_solve(None, None, 0.1, None, 0, 10, None, None, 0, None) == _lib.TV_OK


def test_product_path_has_no_cpu_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    y = torch.from_numpy(np.zeros((2, 4), np.float32))
    with pytest.raises((RuntimeError, ValueError)):
        _lib.chain_prox(y, lam=0.1)
