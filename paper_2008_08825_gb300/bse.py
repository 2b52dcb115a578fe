"""Thin Python binding of the C ABI in include/bse.h (argument marshalling only).

Every step of the solve runs in the CUDA library libbse_gb300.so; this module
only converts PyTorch CUDA tensors to the ABI's column-major device pointers
and back.  There is no CPU fallback: if the library cannot be built or
loaded, or no CUDA device is present, the calls raise.

Layout: the ABI is column-major.  A PyTorch (row-major) n x n tensor is
passed as ``A.mT.contiguous()`` (the column-major storage of A); outputs are
allocated as (k, n) row-major tensors and returned as their ``.mT`` views.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
STATUS_NAMES = {
    0: "BSE_OK",
    1: "BSE_ERR_ARG",
    2: "BSE_ERR_NOT_PD_AMINUSB",
    3: "BSE_ERR_NOT_PD_APLUSB",
    4: "BSE_ERR_NO_CONVERGENCE",
    5: "BSE_ERR_REFINE",
    6: "BSE_ERR_TIMEOUT",
    7: "BSE_ERR_CUDA",
    8: "BSE_ERR_NOMEM",
    9: "BSE_ERR_NOT_IMPLEMENTED",
    10: "BSE_ERR_TOO_LARGE",
}
NOALLOC_MAX_N = 256
METHODS = {"chol": 0, "svd": 1, "sqrt": 2, "tda": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}


class BseError(RuntimeError):
    def __init__(self, code: int, msg: str, info: int = 0):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg} (info={info})")
        self.code = code
        self.info = info


class _Info(ctypes.Structure):
    _fields_ = [("info", ctypes.c_int64), ("err_est", ctypes.c_double), ("refine_iters", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.POINTER(ctypes.c_double)


def header_functions() -> list[str]:
    """Names of the functions declared in include/bse.h."""
    hdr = os.path.join(_build.ROOT, "include", "bse.h")
    txt = open(hdr).read()
    return re.findall(r"^\s*(?:bse_status|const char\*|int64_t)\s+(bse_\w+)\s*\(", txt, flags=re.M)


def _bind(lib):
    lib.bse_create.argtypes = [ctypes.POINTER(_P)]
    lib.bse_destroy.argtypes = [_P]
    lib.bse_last_error.restype = ctypes.c_char_p
    lib.bse_workspace_size.argtypes = [_I64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    lib.bse_set_workspace.argtypes = [_P, _P, ctypes.c_size_t]
    for f in (lib.bse_solve_chol, lib.bse_solve_svd, lib.bse_solve_sqrt):
        f.argtypes = [_P, _I64, _P, _I64, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P, _I64, _P, _I64,
                      ctypes.POINTER(_Info), _P]
    lib.bse_solve_tda.argtypes = [_P, _I64, _P, _I64, _I64, _I64, _P, _P, _I64, ctypes.POINTER(_Info), _P]
    lib.bse_grad.argtypes = [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _P, _I64, _P, _I64, _P]
    lib.bse_solve_host.argtypes = [_P, ctypes.c_int, _I64, _P, _I64, _P, _I64, _I64, _I64, ctypes.c_int, _P, _P,
                                   _I64, _P, _I64, ctypes.POINTER(_Info), _P]
    lib.bse_launch_count.argtypes = [_P]
    lib.bse_launch_count.restype = ctypes.c_int64
    for f in (lib.bse_solve_batched, lib.bse_solve_batched_async):
        f.argtypes = [_P, _I64, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]
        f.restype = ctypes.c_int
    lib.bse_solve_chol_noalloc.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _P]
    lib.bse_solve_chol_noalloc.restype = ctypes.c_int
    lib.bse_ooc_run.argtypes = [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, ctypes.POINTER(_Info), _P]
    lib.bse_ooc_run.restype = ctypes.c_int
    lib.bse_set_option.argtypes = [_P, ctypes.c_int, _I64]
    lib.bse_set_option.restype = ctypes.c_int
    lib.bse_profile_enable.argtypes = [_P, ctypes.c_int]
    lib.bse_profile_enable.restype = ctypes.c_int
    lib.bse_profile_read.restype = ctypes.c_int
    lib.bse_profile_kernels.argtypes = [_P, ctypes.c_char_p, ctypes.c_size_t]
    lib.bse_profile_kernels.restype = ctypes.c_int64
    for name in ("bse_create", "bse_destroy", "bse_workspace_size", "bse_set_workspace", "bse_solve_chol",
                 "bse_solve_svd", "bse_grad", "bse_solve_host"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def lib():
    """The loaded CUDA library (built in-tree on first use if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.lib_path()
            if not os.path.exists(path):
                path = _build.build()
            _lib = _bind(ctypes.CDLL(path))
        return _lib


def _check(code: int, info: int = 0):
    if code != OK:
        raise BseError(code, lib().bse_last_error().decode(errors="replace"), info)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Handle:
    """Owns a bse_handle bound to the current CUDA device (workspace from torch)."""

    def __init__(self):
        if not torch.cuda.is_available():
            raise RuntimeError("bse: a CUDA device is required (no CPU fallback)")
        h = _P()
        _check(lib().bse_create(ctypes.byref(h)))
        self._h = h
        self._ws = None

    @property
    def ptr(self):
        return self._h

    def reserve(self, n: int, method: str, device, precision: str = "fp64") -> None:
        need = ctypes.c_size_t(0)
        _check(lib().bse_workspace_size(int(n), METHODS[method], PRECISIONS[precision], ctypes.byref(need)))
        if self._ws is None or self._ws.numel() < need.value or self._ws.device != device:
            self._ws = torch.empty(need.value, dtype=torch.uint8, device=device)
            _check(lib().bse_set_workspace(self._h, _P(self._ws.data_ptr()), self._ws.numel()))

    def set_tc_min_mnk(self, value: int) -> None:
        """Mixed form: products with m*n*k >= value use the tensor-core engine."""
        _check(lib().bse_set_option(self._h, 1, int(value)))

    def set_tc_engine(self, engine: str) -> None:
        """Mixed form: 'tcgen05' (default; TMEM accumulators, TMA) or 'mma_sync'."""
        _check(lib().bse_set_option(self._h, 3, {"tcgen05": 0, "mma_sync": 1}[engine]))

    def set_tc_wait_cycles(self, value: int) -> None:
        """Mixed form, tcgen05 engine: limit of its pipeline waits in clock
        cycles (0 restores the default, about 1 s)."""
        _check(lib().bse_set_option(self._h, 4, int(value)))

    def set_launch_shapes(self, hemv_item_tiles: int = 0, splitk_max: int = 0) -> None:
        """Matvec row tiles per work item (1..16) and split-K cap (1..8); 0 = library default."""
        _check(lib().bse_set_option(self._h, 7, int(hemv_item_tiles)))
        _check(lib().bse_set_option(self._h, 8, int(splitk_max)))

    def set_batch_team(self, team: int, min_n: int | None = None) -> None:
        """Batched Alg. 2: CTAs per team (1, 2, 4, 8) for instances with n >= min_n."""
        _check(lib().bse_set_option(self._h, 5, int(team)))
        if min_n is not None:
            _check(lib().bse_set_option(self._h, 6, int(min_n)))

    def set_batch_ctas_per_sm(self, value: int) -> None:
        """Batched solves: 1 or 2 resident CTAs per SM for the persistent kernel."""
        _check(lib().bse_set_option(self._h, 2, int(value)))

    def kernel_profile(self) -> dict:
        """Per-kernel (launches, total ms) recorded at profiling level 2."""
        buf = ctypes.create_string_buffer(1 << 16)
        lib().bse_profile_kernels(self._h, buf, len(buf))
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms = line.rsplit(" ", 2)
            out[name] = (int(cnt), float(ms))
        return out

    def launches(self) -> int:
        return int(lib().bse_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().bse_set_workspace(self._h, None, 0)
            lib().bse_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default = threading.local()


def default_handle() -> Handle:
    h = getattr(_default, "h", None)
    if h is None:
        h = Handle()
        _default.h = h
    return h


def _default_tuned(n: int, precision: str) -> Handle:
    """The default handle with the tuned launch shapes for this size and
    precision applied (the autotuner's cache, else the table shipped for
    GB300; the library defaults when neither has an entry)."""
    from . import autotune

    h = default_handle()
    key = (autotune.size_bucket(n), precision)
    if getattr(h, "_tuned_key", None) != key:
        h.set_launch_shapes(0, 0)
        h.tuning = autotune.apply_tuned(h, n, precision)
        h._tuned_key = key
    return h


def _colmajor(A: torch.Tensor) -> torch.Tensor:
    if A.dtype != torch.complex128:
        raise TypeError("bse: A and B must be complex128")
    if not A.is_cuda:
        raise TypeError("bse: device tensors required (use solve_host for host arrays)")
    return A.mT.contiguous()


def solve(A: torch.Tensor, B: torch.Tensor, method: str = "chol", precision: str = "fp64", il: int | None = None,
          iu: int | None = None, vectors: bool = True, handle: Handle | None = None, stream=None):
    """Positive eigenvalues omega (ascending) and Sigma-normalised eigenvectors
    [X; Y] of H1 = [A B; -B -A] (Alg. 2 for method='chol', Alg. 3 for 'svd',
    Alg. 1, the square-root method, for 'sqrt').

    Returns (omega, X, Y) with omega of shape (k,), X, Y of shape (n, k)
    (None when vectors=False), k = iu - il + 1 (1-based, inclusive; default all).
    """
    n = A.shape[0]
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    k = max(iu - il + 1, 0)
    h = handle or _default_tuned(n, precision)
    h.reserve(n, method, A.device, precision)
    Ac, Bc = _colmajor(A), _colmajor(B)
    omega = torch.empty(k, dtype=torch.float64, device=A.device)
    if vectors:
        Xt = torch.empty((k, n), dtype=torch.complex128, device=A.device)
        Yt = torch.empty((k, n), dtype=torch.complex128, device=A.device)
        px, py = _P(Xt.data_ptr()), _P(Yt.data_ptr())
    else:
        Xt = Yt = None
        px = py = None
    info = _Info()
    fn = {"chol": lib().bse_solve_chol, "svd": lib().bse_solve_svd, "sqrt": lib().bse_solve_sqrt}[method]
    code = fn(h.ptr, n, _P(Ac.data_ptr()), max(n, 1), _P(Bc.data_ptr()), max(n, 1), il, iu, PRECISIONS[precision],
              _P(omega.data_ptr()), px, max(n, 1), py, max(n, 1), ctypes.byref(info), _P(_stream_ptr(stream)))
    _check(code, info.info)
    if not vectors:
        return omega, None, None
    return omega, Xt.mT, Yt.mT



def solve_noalloc(A: torch.Tensor, B: torch.Tensor, k: int, omega: torch.Tensor, Xt: torch.Tensor, Yt: torch.Tensor,
                  stream=None):
    '''The k lowest pairs of one small problem (n <= NOALLOC_MAX_N) through
    bse_solve_chol_noalloc, which allocates nothing (for callers that cannot
    allocate: memory held by another allocator's pool, latency-critical loops).
    Every buffer is the caller's and is used in place: A, B complex128
    column-major (A.mT contiguous, n x n), omega (k,) float64, Xt, Yt (k, n)
    complex128 contiguous (Xt.mT is X).  This wrapper allocates nothing on the
    device either.  Raises BseError on a nonzero status.
    '''
    if A.dim() != 2 or A.shape[0] != A.shape[1] or tuple(B.shape) != tuple(A.shape):
        raise TypeError("bse: A and B must both be n x n")
    n = int(A.shape[0])
    for T in (A, B):
        if T.dtype != torch.complex128 or not T.is_cuda or not _is_colmajor(T):
            raise TypeError("bse: A and B must be column-major complex128 device tensors")
    if omega.dtype != torch.float64 or omega.numel() < k or not omega.is_contiguous():
        raise TypeError("bse: omega must be a contiguous float64 tensor of k elements")
    for T in (Xt, Yt):
        if T.dtype != torch.complex128 or tuple(T.shape) != (k, n) or not T.is_contiguous():
            raise TypeError("bse: Xt, Yt must be contiguous complex128 tensors of shape (k, n)")
    if any(T.device != A.device for T in (B, omega, Xt, Yt)):
        raise TypeError("bse: A, B, omega, Xt and Yt must be on one device")
    info = _Info()
    with torch.cuda.device(A.device):
        code = lib().bse_solve_chol_noalloc(n, int(k), _P(A.data_ptr()), _P(B.data_ptr()), _P(omega.data_ptr()),
                                            _P(Xt.data_ptr()), _P(Yt.data_ptr()), ctypes.byref(info),
                                            _P(_stream_ptr(stream)))
    if code != OK:
        msg = (f"n = {n} above the allocation-free limit {NOALLOC_MAX_N}" if code == 10
               else "allocation-free solve failed")
        raise BseError(code, msg, info.info)
    return omega, Xt.mT, Yt.mT


def solve_tda(A: torch.Tensor, il: int | None = None, iu: int | None = None, vectors: bool = True,
              handle: Handle | None = None, stream=None):
    """Tamm-Dancoff approximation (B = 0): omega = eigenvalues of the Hermitian
    positive definite A (ascending, 1-based inclusive range [il, iu]) and the
    unit eigenvectors X (n x k); the Y half of [X; Y] is zero."""
    n = A.shape[0]
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    k = max(iu - il + 1, 0)
    h = handle or default_handle()
    h.reserve(n, "tda", A.device)
    Ac = _colmajor(A)
    omega = torch.empty(k, dtype=torch.float64, device=A.device)
    Xt = torch.empty((k, n), dtype=torch.complex128, device=A.device) if vectors else None
    info = _Info()
    code = lib().bse_solve_tda(h.ptr, n, _P(Ac.data_ptr()), max(n, 1), il, iu, _P(omega.data_ptr()),
                               _P(Xt.data_ptr()) if vectors else None, max(n, 1), ctypes.byref(info),
                               _P(_stream_ptr(stream)))
    _check(code, info.info)
    return omega, (Xt.mT if vectors else None)

def solve_host(A, B, method: str = "chol", il: int | None = None, iu: int | None = None, handle: Handle | None = None,
               stream=None):
    """End-to-end solve from host arrays (numpy complex128 or CPU tensors; pinned
    CPU tensors give full copy bandwidth) through bse_solve_host; returns host
    (omega, X, Y) as CPU tensors."""
    At = torch.as_tensor(A)
    Bt = torch.as_tensor(B)
    n = At.shape[0]
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    k = iu - il + 1
    h = handle or default_handle()
    h.reserve(n, method, torch.device("cuda", torch.cuda.current_device()))
    Ac = At.mT.contiguous() if not _is_colmajor(At) else At
    Bc = Bt.mT.contiguous() if not _is_colmajor(Bt) else Bt
    omega = torch.empty(k, dtype=torch.float64)
    Xt = torch.empty((k, n), dtype=torch.complex128)
    Yt = torch.empty((k, n), dtype=torch.complex128)
    info = _Info()
    code = lib().bse_solve_host(h.ptr, METHODS[method], n, _P(Ac.data_ptr()), max(n, 1), _P(Bc.data_ptr()), max(n, 1),
                                il, iu, 0, _P(omega.data_ptr()), _P(Xt.data_ptr()), max(n, 1), _P(Yt.data_ptr()),
                                max(n, 1), ctypes.byref(info), _P(_stream_ptr(stream)))
    _check(code, info.info)
    return omega, Xt.mT, Yt.mT


class OocOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("arg", ctypes.c_int32)]


class OocTask(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("out", ctypes.c_int32), ("in0", ctypes.c_int32), ("in1", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


def ooc_run(nb: int, host_tiles, ops, tasks, budget: int, handle: Handle | None = None, stream=None) -> None:
    """bse_ooc_run: execute an out-of-core tile plan.
    host_tiles: list of CPU tensors (nb x nb complex128 tiles stored column-major, e.g. a
    tile's transpose made contiguous; pinned memory lets copies overlap) or None;
    ops: list of (kind, arg); tasks: list of (kind, out, in0, in1, flags)."""
    h = handle or default_handle()
    ptrs = (ctypes.c_void_p * max(len(host_tiles), 1))(*[t.data_ptr() if t is not None else None
                                                          for t in host_tiles])
    op_arr = (OocOp * max(len(ops), 1))(*[OocOp(int(k), int(a)) for k, a in ops])
    task_arr = (OocTask * max(len(tasks), 1))(*[OocTask(*[int(v) for v in t]) for t in tasks])
    info = _Info()
    code = lib().bse_ooc_run(h.ptr, int(nb), len(host_tiles), ptrs, len(ops), op_arr, len(tasks), task_arr,
                             int(budget), ctypes.byref(info), _P(_stream_ptr(stream)))
    _check(code, info.info)


def _is_colmajor(T: torch.Tensor) -> bool:
    return T.dim() == 2 and T.stride(0) == 1 and T.stride(1) == T.shape[0]


def grad(X: torch.Tensor, Y: torch.Tensor, w: torch.Tensor, handle: Handle | None = None, stream=None):
    """dL/dA, dL/dB (full Hermitian, n x n) for L = sum_i w_i omega_i, given the k
    eigenvector columns X, Y (n x k) of the selected omega_i."""
    n, k = X.shape
    h = handle or default_handle()
    X = X if _is_colmajor(X) else X.mT.contiguous().mT
    Y = Y if _is_colmajor(Y) else Y.mT.contiguous().mT
    w = w.to(dtype=torch.float64, device=X.device).contiguous()
    dAt = torch.empty((n, n), dtype=torch.complex128, device=X.device)
    dBt = torch.empty((n, n), dtype=torch.complex128, device=X.device)
    code = lib().bse_grad(h.ptr, n, k, _P(_cm_ptr(X)), max(n, 1), _P(_cm_ptr(Y)), max(n, 1), _P(w.data_ptr()),
                          _P(dAt.data_ptr()), max(n, 1), _P(dBt.data_ptr()), max(n, 1), _P(_stream_ptr(stream)))
    _check(code)
    return dAt.mT, dBt.mT


def _cm_ptr(T: torch.Tensor) -> int:
    if not _is_colmajor(T):
        raise ValueError("expected a column-major (n, k) view, e.g. the X returned by solve()")
    return T.data_ptr()


class Omega(torch.autograd.Function):
    """omega[idx] of H1 = [A B; -B -A] with a backward through bse_grad.

    The gradient is the Hermitian Frobenius gradient (the convention of
    torch.linalg.eigh): d omega_i = <x x^H + y y^H, dA> + <x y^H + y x^H, dB>.
    """

    @staticmethod
    def forward(ctx, A, B, idx, method="chol"):
        idx = torch.as_tensor(idx, device=A.device, dtype=torch.long)
        omega, X, Y = solve(A.detach(), B.detach(), method=method)
        ctx.save_for_backward(X[:, idx], Y[:, idx])
        return omega[idx]

    @staticmethod
    def backward(ctx, g):
        Xs, Ys = ctx.saved_tensors
        Xs = Xs.mT.contiguous().mT
        Ys = Ys.mT.contiguous().mT
        dA, dB = grad(Xs, Ys, g)
        return dA, dB, None, None


class Batch:
    """Device buffers and pointer tables of a batched solve (the k lowest pairs
    of many instances, Alg. 2 or Alg. 3 each, one persistent launch).

    instances: list of (A, B) complex128 CUDA tensors (n_i x n_i, n_i <= 1024);
    method: "chol" (Alg. 2) or "svd" (Alg. 3).
    """

    def __init__(self, instances, k: int = 32, method: str = "chol"):
        self.count = len(instances)
        self.k = int(k)
        self.method = method
        dev = instances[0][0].device if instances else torch.device("cuda")
        self.n = [int(A.shape[0]) for A, _ in instances]
        self.A = [_colmajor(A) for A, _ in instances]
        self.B = [_colmajor(B) for _, B in instances]
        self.ks = [min(self.k, n) for n in self.n]
        self.omega = [torch.empty(k_i, dtype=torch.float64, device=dev) for k_i in self.ks]
        self.Xt = [torch.empty((k_i, n), dtype=torch.complex128, device=dev) for n, k_i in zip(self.n, self.ks)]
        self.Yt = [torch.empty((k_i, n), dtype=torch.complex128, device=dev) for n, k_i in zip(self.n, self.ks)]
        self.dstatus = torch.zeros(2 * max(self.count, 1), dtype=torch.int64, device=dev)

        def arr(ctype, vals):
            return (ctype * max(len(vals), 1))(*vals)

        self._n = arr(ctypes.c_int64, self.n)
        self._A = arr(ctypes.c_void_p, [t.data_ptr() for t in self.A])
        self._B = arr(ctypes.c_void_p, [t.data_ptr() for t in self.B])
        self._om = arr(ctypes.c_void_p, [t.data_ptr() for t in self.omega])
        self._X = arr(ctypes.c_void_p, [t.data_ptr() for t in self.Xt])
        self._Y = arr(ctypes.c_void_p, [t.data_ptr() for t in self.Yt])

    def _args(self):
        return (self.count, self._n, self._A, self._B, self.k, METHODS[self.method], 0, self._om, self._X, self._Y)

    def run(self, handle: Handle | None = None, stream=None):
        """Synchronous solve; raises on the first failing instance."""
        h = handle or default_handle()
        st = (ctypes.c_int64 * max(self.count, 1))()
        code = lib().bse_solve_batched(h.ptr, *self._args(), st, _P(_stream_ptr(stream)))
        self.status = list(st)[: self.count]
        _check(code)
        return self

    def enqueue(self, handle: Handle | None = None, stream=None):
        """Enqueue only (capturable in a CUDA graph); statuses land in self.dstatus."""
        h = handle or default_handle()
        code = lib().bse_solve_batched_async(h.ptr, *self._args(), _P(self.dstatus.data_ptr()),
                                             _P(_stream_ptr(stream)))
        _check(code)
        return self

    def results(self):
        return [(o, X.mT, Y.mT) for o, X, Y in zip(self.omega, self.Xt, self.Yt)]
