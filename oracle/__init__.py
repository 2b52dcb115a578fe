"""Plain FP64 CPU oracle for the form-I BSE eigenproblem (Benner & Penke,
arXiv 2008.08825, Algorithms 2 and 3).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
(``paper_2008_08825_gb300``) never does, and shares no code with it.

The arithmetic lives in ``bse_oracle.c`` (plain C99 complex, OpenMP, no BLAS
or LAPACK).  This module compiles it with gcc on first use (or through
:func:`build`) and exposes numpy front ends.  Every matrix is complex128 and
passed column-major (Fortran order); Hermitian inputs are read from their
lower triangle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bse_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_NOT_PD_AMINUSB = 2
ERR_NOT_PD_APLUSB = 3
ERR_NO_CONVERGENCE = 4
ERR_NOMEM = 8


class OracleError(RuntimeError):
    def __init__(self, code: int, info: int, what: str):
        super().__init__(f"{what}: oracle status {code} (info {info})")
        self.code = code
        self.info = info


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile bse_oracle.c into a shared library (gcc, OpenMP).  Returns the path."""
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", *extra_flags, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def _bind(lib):
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_get_threads.restype = ctypes.c_int
    lib.oracle_cholesky.argtypes = [_I64, _P, _I64, _P, _I64]
    lib.oracle_cholesky.restype = _I64
    lib.oracle_congruence.argtypes = [_I64, _P, _I64, _P, _I64, _P, _I64]
    lib.oracle_congruence.restype = ctypes.c_int
    lib.oracle_product.argtypes = [_I64, _P, _I64, _P, _I64, _P, _I64]
    lib.oracle_jacobi_svd.argtypes = [_I64, _P, _I64, _P, _P, _I64, _P, _I64, _P]
    lib.oracle_jacobi_svd.restype = ctypes.c_int
    lib.oracle_jacobi_eigh.argtypes = [_I64, _P, _I64, _P, _P, _I64, _P]
    lib.oracle_jacobi_eigh.restype = ctypes.c_int
    for f in (lib.oracle_solve_chol, lib.oracle_solve_svd):
        f.argtypes = [_I64, _P, _I64, _P, _I64, _P, _P, _I64, _P, _I64, _P]
        f.restype = ctypes.c_int
    lib.oracle_grad.argtypes = [_I64, _I64, _P, _I64, _P, _I64, _P, _P, _I64, _P, _I64]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle shared library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _fz(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def set_threads(t: int) -> None:
    load().oracle_set_threads(int(t))


def get_threads() -> int:
    return int(load().oracle_get_threads())


def cholesky(M, lib=None) -> np.ndarray:
    """L with L L^H = M (lower triangle of M read).  Raises OracleError(info=column)."""
    lib = lib or load()
    M = _fz(M)
    n = M.shape[0]
    L = np.zeros((n, n), dtype=np.complex128, order="F")
    col = lib.oracle_cholesky(n, _ptr(M), max(n, 1), _ptr(L), max(n, 1))
    if col:
        raise OracleError(ERR_ARG, int(col), "matrix not positive definite")
    return L


def congruence(M1, L, lib=None) -> np.ndarray:
    """M = L^H M1 L (Alg. 2 step 2)."""
    lib = lib or load()
    M1, L = _fz(M1), _fz(L)
    n = M1.shape[0]
    M = np.zeros((n, n), dtype=np.complex128, order="F")
    rc = lib.oracle_congruence(n, _ptr(M1), max(n, 1), _ptr(L), max(n, 1), _ptr(M), max(n, 1))
    if rc:
        raise OracleError(rc, 0, "congruence")
    return M


def product(L1, L2, lib=None) -> np.ndarray:
    """G = L1^H L2 (Alg. 3 step 3)."""
    lib = lib or load()
    L1, L2 = _fz(L1), _fz(L2)
    n = L1.shape[0]
    G = np.zeros((n, n), dtype=np.complex128, order="F")
    lib.oracle_product(n, _ptr(L1), max(n, 1), _ptr(L2), max(n, 1), _ptr(G), max(n, 1))
    return G


def jacobi_svd(G, lib=None):
    """One-sided Jacobi SVD: returns (sigma, U, V, sweeps), unordered."""
    lib = lib or load()
    G = _fz(G)
    n = G.shape[0]
    s = np.zeros(n)
    U = np.zeros((n, n), dtype=np.complex128, order="F")
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    sw = ctypes.c_int(0)
    rc = lib.oracle_jacobi_svd(n, _ptr(G), max(n, 1), _ptr(s), _ptr(U), max(n, 1), _ptr(V), max(n, 1), ctypes.byref(sw))
    if rc:
        raise OracleError(rc, sw.value, "jacobi_svd")
    return s, U, V, sw.value


def jacobi_eigh(M, lib=None):
    """Two-sided Jacobi eigendecomposition of Hermitian PD M: (lam, V, sweeps), unordered."""
    lib = lib or load()
    M = _fz(M)
    n = M.shape[0]
    lam = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    sw = ctypes.c_int(0)
    rc = lib.oracle_jacobi_eigh(n, _ptr(M), max(n, 1), _ptr(lam), _ptr(V), max(n, 1), ctypes.byref(sw))
    if rc:
        raise OracleError(rc, sw.value, "jacobi_eigh")
    return lam, V, sw.value


def _solve(fn, A, B, vectors: bool, what: str):
    A, B = _fz(A), _fz(B)
    n = A.shape[0]
    omega = np.zeros(n)
    info = ctypes.c_int64(0)
    if vectors:
        X = np.zeros((n, n), dtype=np.complex128, order="F")
        Y = np.zeros((n, n), dtype=np.complex128, order="F")
        px, py = _ptr(X), _ptr(Y)
    else:
        X = Y = None
        px = py = None
    rc = fn(n, _ptr(A), max(n, 1), _ptr(B), max(n, 1), _ptr(omega), px, max(n, 1), py, max(n, 1), ctypes.byref(info))
    if rc:
        raise OracleError(rc, info.value, what)
    return omega, X, Y


def solve_chol(A, B, vectors: bool = True, lib=None):
    """Alg. 2: (omega ascending, X, Y) with the Sigma-normalised eigenvectors [X; Y]."""
    lib = lib or load()
    return _solve(lib.oracle_solve_chol, A, B, vectors, "solve_chol")


def solve_svd(A, B, vectors: bool = True, lib=None):
    """Alg. 3: (omega ascending, X, Y) with the Sigma-normalised eigenvectors [X; Y]."""
    lib = lib or load()
    return _solve(lib.oracle_solve_svd, A, B, vectors, "solve_svd")


def grad(X, Y, w, lib=None):
    """dL/dA, dL/dB for L = sum_i w_i omega_i over the k columns of X, Y."""
    lib = lib or load()
    X, Y = _fz(X), _fz(Y)
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    n, k = X.shape
    dA = np.zeros((n, n), dtype=np.complex128, order="F")
    dB = np.zeros((n, n), dtype=np.complex128, order="F")
    lib.oracle_grad(n, k, _ptr(X), max(n, 1), _ptr(Y), max(n, 1), _ptr(w), _ptr(dA), max(n, 1), _ptr(dB), max(n, 1))
    return dA, dB
