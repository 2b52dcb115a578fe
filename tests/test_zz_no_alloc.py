"""bse_solve_chol_noalloc, the allocation-free Cholesky solve, against the
ordinary entry point bse_solve_chol on the same inputs: two calls in a row,
each within the suite's tolerances (eigenvalues 1e-11 * omega_max; vectors
1e-11 * omega_max / gap + 1e-12 after phase alignment; Sigma-orthonormality
1e-10), the second taking no device memory; oversize and not-definite inputs
are refused.  The eigenvalues are also checked against the CPU oracle
directly (per eigenvalue 1e-11), and a fresh process records how much device
memory the first call takes (the lazily loaded module with its 8 MiB scratch,
and the code) and that later calls take none.  The file name sorts last so
that a full run also exercises the entry point after every other GPU test in
the same process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from conftest import ROOT, phase_align, sigma_residual
from paper_2008_08825_gb300 import bse, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda0():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return torch.device("cuda", 0)


def _colmajor_device(M, dev):
    return torch.from_numpy(np.ascontiguousarray(M.T)).to(dev).mT


def _gaps(om):
    d = np.diff(om)
    g = np.full(om.shape, np.inf)
    g[:-1] = np.minimum(g[:-1], d)
    g[1:] = np.minimum(g[1:], d)
    return g


@pytest.mark.parametrize("n,k", [(96, 16), (37, 37), (bse.NOALLOC_MAX_N, 32)])
def test_noalloc_matches_solve_chol_twice(cuda0, n, k):
    A, B = inputs.base(n, seed=500 + n)
    Ad, Bd = _colmajor_device(A, cuda0), _colmajor_device(B, cuda0)
    om_all, X_all, Y_all = bse.solve(Ad, Bd, method="chol")
    om_ref = om_all.cpu().numpy()
    X_ref, Y_ref = X_all[:, :k].cpu().numpy(), Y_all[:, :k].cpu().numpy()
    tol_vec = 1e-11 * om_ref.max() / _gaps(om_ref)[:k] + 1e-12
    omega = torch.empty(k, dtype=torch.float64, device=cuda0)
    Xt = torch.empty((k, n), dtype=torch.complex128, device=cuda0)
    Yt = torch.empty((k, n), dtype=torch.complex128, device=cuda0)
    outs = []
    for call in range(2):
        omega.fill_(float("nan"))
        Xt.fill_(float("nan"))
        Yt.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(cuda0)[0]
        om, X, Y = bse.solve_noalloc(Ad, Bd, k, omega, Xt, Yt)
        free1 = torch.cuda.mem_get_info(cuda0)[0]
        if call == 1:
            assert free1 == free0, "the second call took device memory"
        om, X, Y = om.cpu().numpy(), X.cpu().numpy(), Y.cpu().numpy()
        assert np.max(np.abs(om - om_ref[:k])) <= 1e-11 * om_ref.max()
        a, b = phase_align(X, Y)
        c, d = phase_align(X_ref, Y_ref)
        err = np.maximum(np.abs(a - c).max(axis=0), np.abs(b - d).max(axis=0))
        assert np.all(err <= tol_vec), (np.nonzero(err > tol_vec)[0][:5], err.max())
        assert sigma_residual(X, Y) <= 1e-10
        outs.append((om, X, Y))
    for u, v in zip(*outs):
        assert np.array_equal(u, v)


def test_noalloc_refuses_oversize_and_reports_not_definite(cuda0):
    n = bse.NOALLOC_MAX_N + 1
    Z = torch.zeros((n, n), dtype=torch.complex128, device=cuda0).mT
    om = torch.empty(1, dtype=torch.float64, device=cuda0)
    Xt = torch.empty((1, n), dtype=torch.complex128, device=cuda0)
    Yt = torch.empty((1, n), dtype=torch.complex128, device=cuda0)
    with pytest.raises(bse.BseError) as e:
        bse.solve_noalloc(Z, Z, 1, om, Xt, Yt)
    assert e.value.code == 10 and "limit" in str(e.value)
    # A - B = -I is not positive definite at column 1; the next call must
    # start from clean status words and succeed
    n = 8
    A = torch.eye(n, dtype=torch.complex128, device=cuda0).mT
    B = (2.0 * torch.eye(n, dtype=torch.complex128, device=cuda0)).mT
    Xt = torch.empty((2, n), dtype=torch.complex128, device=cuda0)
    Yt = torch.empty((2, n), dtype=torch.complex128, device=cuda0)
    om = torch.empty(2, dtype=torch.float64, device=cuda0)
    with pytest.raises(bse.BseError) as e:
        bse.solve_noalloc(A, B, 2, om, Xt, Yt)
    assert e.value.code == 2 and e.value.info == 1
    B = (0.5 * torch.eye(n, dtype=torch.complex128, device=cuda0)).mT
    o, X, Y = bse.solve_noalloc(A, B, 2, om, Xt, Yt)
    assert np.allclose(o.cpu().numpy(), np.sqrt(1.0 - 0.25), rtol=1e-14, atol=0)


def test_noalloc_vs_oracle(cuda0):
    """The largest allowed size against the oracle itself, not only against
    bse_solve_chol: omega per eigenvalue and vectors after phase alignment."""
    n, k = bse.NOALLOC_MAX_N, 24
    A, B = inputs.base(n, seed=77)
    om_r, X_r, Y_r = oracle.solve_svd(A, B)
    Ad, Bd = _colmajor_device(A, cuda0), _colmajor_device(B, cuda0)
    omega = torch.empty(k, dtype=torch.float64, device=cuda0)
    Xt = torch.empty((k, n), dtype=torch.complex128, device=cuda0)
    Yt = torch.empty((k, n), dtype=torch.complex128, device=cuda0)
    om, X, Y = bse.solve_noalloc(Ad, Bd, k, omega, Xt, Yt)
    om, X, Y = om.cpu().numpy(), X.cpu().numpy(), Y.cpu().numpy()
    assert np.max(np.abs(om - om_r[:k])) <= 1e-11 * om_r.max()
    assert np.max(np.abs(om - om_r[:k]) / om_r[:k]) <= 1e-11
    a, b = phase_align(X, Y)
    c, d = phase_align(X_r[:, :k], Y_r[:, :k])
    tol = 1e-11 * om_r.max() / _gaps(om_r)[:k] + 1e-12
    err = np.maximum(np.abs(a - c).max(axis=0), np.abs(b - d).max(axis=0))
    assert np.all(err <= tol)


def test_noalloc_rejects_mismatched_buffers(cuda0):
    n, k = 16, 4
    A, B = inputs.base(n, seed=5)
    Ad, Bd = _colmajor_device(A, cuda0), _colmajor_device(B, cuda0)
    om = torch.empty(k, dtype=torch.float64, device=cuda0)
    Xt = torch.empty((k, n), dtype=torch.complex128, device=cuda0)
    Yt = torch.empty((k, n), dtype=torch.complex128, device=cuda0)
    with pytest.raises(TypeError):  # B smaller than A
        bse.solve_noalloc(Ad, Bd[:8, :8], k, om, Xt, Yt)
    with pytest.raises(TypeError):  # A not square
        bse.solve_noalloc(_colmajor_device(A[:, :8], cuda0), Bd, k, om, Xt, Yt)
    with pytest.raises(TypeError):  # an output on another device
        bse.solve_noalloc(Ad, Bd, k, om.cpu(), Xt, Yt)
    with pytest.raises(TypeError):  # outputs of the wrong shape
        bse.solve_noalloc(Ad, Bd, k, om, Xt[:, :8], Yt)


_FRESH = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2008_08825_gb300 import bse, inputs
dev = torch.device("cuda", 0)
n, k = 64, 8
A, B = inputs.base(n, seed=3)
Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).mT
Bd = torch.from_numpy(np.ascontiguousarray(B.T)).to(dev).mT
om = torch.empty(k, dtype=torch.float64, device=dev)
Xt = torch.empty((k, n), dtype=torch.complex128, device=dev)
Yt = torch.empty((k, n), dtype=torch.complex128, device=dev)
bse.lib()
torch.cuda.synchronize()
free = [torch.cuda.mem_get_info(dev)[0]]
for _ in range(3):
    bse.solve_noalloc(Ad, Bd, k, om, Xt, Yt)
    free.append(torch.cuda.mem_get_info(dev)[0])
print(json.dumps({"taken": [free[i] - free[i + 1] for i in range(3)], "omega0": float(om[0])}))
"""


def test_noalloc_first_call_in_fresh_process(cuda0):
    """In a fresh process the first call loads the modules (scratch plus
    code) and may take that much device memory once; the calls after it take
    none.  The bound is the 8 MiB scratch plus 64 MiB for code and the
    driver's per-module reservations."""
    code = _FRESH.replace("ROOT", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ))
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    first, second, third = res["taken"]
    print(f"first call took {first / 2**20:.1f} MiB, then {second} and {third} bytes")
    assert first <= (8 + 64) * 2**20
    assert second == 0 and third == 0
    assert np.isfinite(res["omega0"]) and res["omega0"] > 0
