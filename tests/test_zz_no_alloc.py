"""bse_solve_chol_noalloc, the allocation-free Cholesky solve, against the
ordinary entry point bse_solve_chol on the same inputs: two calls in a row,
each within the suite's tolerances (eigenvalues 1e-11 * omega_max; vectors
1e-11 * omega_max / gap + 1e-12 after phase alignment; Sigma-orthonormality
1e-10), the second taking no device memory; oversize and not-definite inputs
are refused.  The file name sorts last so that a full run also exercises the
entry point after every other GPU test in the same process.
"""
import numpy as np
import pytest
import torch

from conftest import phase_align, sigma_residual
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
