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


def test_workspace_sizes_per_method(lib):
    """TDA needs least, CHOL less than SVD and SQRT (eight n x n complex
    buffers plus the full tridiagonal work); sizes grow with n; the mixed form
    adds the slice workspace of the tensor-core products."""
    def ws(n, method, prec=0):
        b = ctypes.c_size_t(0)
        assert lib.bse_workspace_size(n, method, prec, ctypes.byref(b)) == 0
        return b.value

    n = 1024
    chol, svd, sqrt, tda = ws(n, 0), ws(n, 1), ws(n, 2), ws(n, 3)
    assert tda < chol < min(svd, sqrt)
    assert sqrt >= 8 * n * n * 16
    for m in range(4):
        assert ws(n, m) <= ws(2 * n, m)
    assert ws(n, 0, 1) > chol + 8 * 2 * (2 * n) * (n + 2 * n)  # 8 BF16 slices of both operands


def test_noalloc_host_checks_need_no_gpu(lib):
    """Argument checks of the allocation-free entry point run before any CUDA
    call: n above the limit gives BSE_ERR_TOO_LARGE, bad k an argument error,
    k = 0 success; none of them touches a device.  n = 0 is the set-up call,
    which needs a device: without one it reports BSE_ERR_CUDA."""
    lib.bse_solve_chol_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 7
    lib.bse_solve_chol_noalloc.restype = ctypes.c_int
    assert lib.bse_solve_chol_noalloc(bse.NOALLOC_MAX_N + 1, 1, None, None, None, None, None, None, None) == 10
    assert lib.bse_solve_chol_noalloc(8, 9, None, None, None, None, None, None, None) == 1
    assert lib.bse_solve_chol_noalloc(8, -1, None, None, None, None, None, None, None) == 1
    assert lib.bse_solve_chol_noalloc(8, 0, None, None, None, None, None, None, None) == 0
    assert lib.bse_solve_chol_noalloc(0, 0, None, None, None, None, None, None, None) == 7
    assert lib.bse_solve_chol_noalloc(8, 2, None, None, None, None, None, None, None) == 1  # NULL pointers


def test_out_of_core_plan_checks_need_no_gpu(lib):
    """bse_ooc_run checks a plan on the host before any CUDA call: residency,
    the tile budget, indices and the TRSM/POTRF pairing are refused with an
    argument error naming the op; a consistent plan then meets the handle
    check (NULL here) and nothing runs."""
    from paper_2008_08825_gb300 import ooc

    Op, Task = bse.OocOp, bse.OocTask
    tiles = (ctypes.c_void_p * 3)(1, 2, 3)  # never dereferenced: every call below is refused first
    gemm = Task(ooc.TASK_KINDS["GEMM"], 2, 0, 1, 0)
    trsm = Task(ooc.TASK_KINDS["TRSM"], 1, 0, -1, 0)

    def run(ops, tasks, budget, nb=16):
        o = (Op * max(len(ops), 1))(*[Op(k, a) for k, a in ops])
        t = (Task * max(len(tasks), 1))(*tasks)
        return lib.bse_ooc_run(None, nb, 3, tiles, len(ops), o, len(tasks), t, budget, None, None)

    cases = [
        ([(2, 0)], [gemm], 3, "not resident"),
        ([(0, 0), (0, 1), (0, 2)], [gemm], 2, "budget"),
        ([(0, 0), (0, 0)], [gemm], 3, "already resident"),
        ([(3, 1)], [gemm], 3, "not resident"),
        ([(0, 0), (0, 1), (0, 2), (2, 5)], [gemm], 3, "task index"),
        ([(0, 7)], [gemm], 3, "out of range"),
        ([(0, 0), (0, 1), (2, 0)], [trsm], 3, "POTRF"),
        ([(0, 0), (4, 0), (4, 0)], [gemm], 3, "not resident"),
    ]
    for ops, tasks, budget, what in cases:
        assert run(ops, tasks, budget) == 1, ops
        assert what.encode() in lib.bse_last_error(), (ops, lib.bse_last_error())
    assert run([(0, 0)], [gemm], 3, nb=0) == 1 and b"nb" in lib.bse_last_error()
    assert run([(0, 0), (0, 1), (0, 2), (2, 0), (3, 2), (4, 0), (4, 1), (4, 2)], [gemm], 3) == 1
    assert b"handle" in lib.bse_last_error()
