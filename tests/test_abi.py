"""The C-ABI library builds, loads and exports every symbol that
include/bse.h declares; host-only entry points behave (CPU only)."""
import ctypes

import pytest

from paper_2008_08825_gb300 import bse


@pytest.fixture(scope="module")
def lib():
    return bse.lib()


def test_header_declares_the_boundary():
    names = set(bse.header_functions())
    for required in ("bse_solve_chol", "bse_solve_svd", "bse_grad", "bse_create", "bse_destroy",
                     "bse_workspace_size", "bse_solve_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in bse.header_functions():
        assert hasattr(lib, name), name


def test_workspace_size_host_only(lib):
    b = ctypes.c_size_t(0)
    assert lib.bse_workspace_size(0, 0, 0, ctypes.byref(b)) == 0
    small = ctypes.c_size_t(0)
    assert lib.bse_workspace_size(64, 0, 0, ctypes.byref(small)) == 0
    big = ctypes.c_size_t(0)
    assert lib.bse_workspace_size(2048, 1, 0, ctypes.byref(big)) == 0
    assert big.value > small.value > 0
    # n x n complex buffers dominate: CHOL needs >= 5 of them
    assert lib.bse_workspace_size(2048, 0, 0, ctypes.byref(b)) == 0 and b.value >= 5 * 2048 * 2048 * 16
    assert lib.bse_workspace_size(-1, 0, 0, ctypes.byref(b)) == 1
    assert lib.bse_workspace_size(8, 7, 0, ctypes.byref(b)) == 1


def test_null_handle_is_an_argument_error(lib):
    assert lib.bse_solve_chol(None, 4, None, 4, None, 4, 1, 4, 0, None, None, 4, None, 4, None, None) == 1
    assert lib.bse_grad(None, 4, 1, None, 4, None, 4, None, None, 4, None, 4, None) == 1
    assert b"handle" in lib.bse_last_error()
