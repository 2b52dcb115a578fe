"""Seeded synthetic inputs for the form-I BSE eigenproblem.

This module holds input construction only -- none of the solver's arithmetic
-- and is the one piece of code that both the CUDA path's callers (tests,
benchmark) and the CPU oracle's callers use.  Every generator returns
complex128 matrices in Fortran (column-major) order, the layout of the C ABI.

Generators
----------
``base(n, seed)``
    A = diag(d) + 0.1 G_A, B = 0.05 G_B with d ~ U[1, 10] and G Hermitian
    Gaussian: Z has iid entries (N(0,1) + i N(0,1))/sqrt(2) and
    G = (Z + Z^H)/sqrt(2)/sqrt(n) (off-diagonal CN(0, 1/n), diagonal N(0, 1/n),
    spectrum on [-2, 2]).  A +- B is positive definite by Weyl's inequality
    (smallest eigenvalue >= 1 - 0.3 - o(1)).  Draw order from
    ``numpy.random.default_rng(seed)``: d, Re Z_A, Im Z_A, Re Z_B, Im Z_B, all
    row-major.  This is the "random A, B with A's diagonal scaled up" workload
    of the paper's runtime experiment (Section 4, Fig. 1).
``commuting(n, seed)``
    A = Q diag(a) Q^H, B = Q diag(b) Q^H with a ~ U[2, 10], b ~ U[-1, 1] and Q
    Haar-unitary; the exact answer is omega_i = sqrt(a_i^2 - b_i^2).
``paper_e1(n, kappa, seed)``
    The accuracy experiment of Section 4 (Table 1): d equally spaced in
    [1, kappa/3], A = Q^H diag(d) Q, B = Q^H diag(d/2) Q; omega = (sqrt(3)/2) d
    and cond(H) = kappa.
``kappa_sweep(n, kappa, seed)``
    The base generator with the smallest d set to 0.5 and a rank-one shift
    along the lowest eigenvector u of A - B: A -= (c/2) u u^H,
    B += (c/2) u u^H with c = mu_min - mu_max / kappa, so that A - B has
    condition number kappa while A + B is unchanged.
``batched_sizes(count, seed)``
    n_i = round(exp(U[ln 32, ln 1024])).
``hermitian_direction(n, rng)``
    A Hermitian Gaussian direction with unit Frobenius norm.
"""
from __future__ import annotations

import numpy as np


def _hermitian_gaussian(rng: np.random.Generator, n: int) -> np.ndarray:
    re = rng.standard_normal((n, n))
    im = rng.standard_normal((n, n))
    z = (re + 1j * im) * np.sqrt(0.5)
    del re, im
    g = z + z.conj().T
    del z
    g *= 1.0 / np.sqrt(2.0 * n)
    return g


def haar_unitary(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed unitary: QR of a complex Gaussian, R's diagonal phases removed."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * np.sqrt(0.5)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.asfortranarray(q * ph[None, :])


def base(n: int, seed: int = 0):
    """The base workload: (A, B), complex128, Fortran order."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(1.0, 10.0, n)
    A = np.asfortranarray(_hermitian_gaussian(rng, n) * 0.1)
    A[np.diag_indices(n)] += d
    B = np.asfortranarray(_hermitian_gaussian(rng, n) * 0.05)
    return A, B


def commuting(n: int, seed: int = 1):
    """Commuting closed-form instance: (A, B, a, b, Q)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(2.0, 10.0, n)
    b = rng.uniform(-1.0, 1.0, n)
    Q = haar_unitary(rng, n)
    A = np.asfortranarray((Q * a[None, :]) @ Q.conj().T)
    B = np.asfortranarray((Q * b[None, :]) @ Q.conj().T)
    return A, B, a, b, Q


def commuting_omega(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact omega of the commuting instance, ascending."""
    return np.sort(np.sqrt(a * a - b * b))


def paper_e1(n: int, kappa: float, seed: int = 0):
    """Section 4 accuracy workload: (A, B, d); exact omega = sqrt(3)/2 d."""
    rng = np.random.default_rng(seed)
    d = np.linspace(1.0, kappa / 3.0, n)
    Q = haar_unitary(rng, n)
    A = np.asfortranarray((Q.conj().T * d[None, :]) @ Q)
    B = np.asfortranarray((Q.conj().T * (0.5 * d)[None, :]) @ Q)
    return A, B, d


def _hermitian_full(M: np.ndarray) -> np.ndarray:
    L = np.tril(M, -1)
    return L + L.conj().T + np.diag(np.real(np.diag(M)))


def _rank_one(u: np.ndarray, s: float) -> np.ndarray:
    """s u u^H built from real element-wise products and sums, one rounding
    each, so that the same u and s give the same bits on every platform (a
    complex multiply may be fused differently by different numpy builds)."""
    ur, ui = np.ascontiguousarray(u.real), np.ascontiguousarray(u.imag)
    P = np.empty((u.size, u.size), dtype=np.complex128, order="F")
    P.real = (np.multiply.outer(ur, ur) + np.multiply.outer(ui, ui)) * s
    P.imag = (np.multiply.outer(ui, ur) - np.multiply.outer(ur, ui)) * s
    return P


def _kappa_base(n: int, seed: int):
    rng = np.random.default_rng(seed)
    d = rng.uniform(1.0, 10.0, n)
    d[np.argmin(d)] = 0.5
    A = np.asfortranarray(_hermitian_gaussian(rng, n) * 0.1)
    A[np.diag_indices(n)] += d
    B = np.asfortranarray(_hermitian_gaussian(rng, n) * 0.05)
    return A, B, rng


def kappa_shift(n: int, kappa: float, seed: int = 0, iters: int = 60, power_iters: int = 200):
    """The rank-one shift of ``kappa_sweep``: (u, c, achieved_kappa_estimate).

    The lowest eigenpair (mu, u) of A - B comes from inverse iteration with a
    library (LAPACK, through scipy) Cholesky solve, and mu_max from power
    iteration; both are input construction, not part of the solver.  Their
    last bits depend on the platform's LAPACK and BLAS, so a result that must
    be reproduced elsewhere stores (u, c) and passes them back as ``shift``.
    """
    import scipy.linalg as sla

    A, B, rng = _kappa_base(n, seed)
    M2 = A - B
    cf = sla.cho_factor(M2, lower=True, check_finite=False)
    u = np.ones(n, dtype=np.complex128) / np.sqrt(n)
    for _ in range(iters):
        u = sla.cho_solve(cf, u, check_finite=False)
        u /= np.linalg.norm(u)
    mu = float(np.real(np.vdot(u, M2 @ u)))
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v /= np.linalg.norm(v)
    for _ in range(power_iters):
        v = M2 @ v
        v /= np.linalg.norm(v)
    mu_max = float(np.real(np.vdot(v, M2 @ v)))
    c = mu - mu_max / kappa
    return u, c, mu_max / (mu - c)


def kappa_sweep(n: int, kappa: float, seed: int = 0, iters: int = 60, power_iters: int = 200, shift=None):
    """Base workload with kappa(A - B) set to `kappa`; returns (A, B, achieved_kappa_estimate).

    ``shift`` = (u, c) from an earlier ``kappa_shift`` call reproduces that
    call's matrices bit for bit on any platform (the estimate is then None).
    """
    if shift is None:
        u, c, est = kappa_shift(n, kappa, seed, iters, power_iters)
    else:
        (u, c), est = shift, None
    A, B, _ = _kappa_base(n, seed)
    P = _rank_one(np.asarray(u, dtype=np.complex128), 0.5 * float(c))
    A -= P
    B += P
    return A, B, est


def batched_sizes(count: int = 512, seed: int = 10_000, lo: int = 32, hi: int = 1024) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def hermitian_direction(n: int, rng: np.random.Generator) -> np.ndarray:
    E = _hermitian_gaussian(rng, n)
    E /= np.linalg.norm(E)
    return np.asfortranarray(E)


def grad_weights(k: int = 16, seed: int = 1) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(k)


def assemble_h1(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """H1 = [A B; -B -A] from the lower triangles of A and B (for checks only)."""
    Af, Bf = _hermitian_full(A), _hermitian_full(B)
    return np.block([[Af, Bf], [-Bf, -Af]])


def hermitian_full(M: np.ndarray) -> np.ndarray:
    """Full Hermitian matrix from the lower triangle of M."""
    return _hermitian_full(M)
