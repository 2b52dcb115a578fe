"""Pins of the CPU oracle to facts fixed by the paper and by mathematics,
independent of the oracle's own code (CPU only).

Each test names the fact it checks.  Together they are chosen so that a
plausible slip anywhere in the oracle (a dropped 1/2, a wrong sign in Y, a
transposed triangular product, a missing conjugate, a wrong Lambda power)
breaks at least one of them; ``test_oracle_mutants.py`` checks exactly that.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2008_08825_gb300 import inputs
from conftest import eig_residual, phase_align, sigma_residual

SOLVERS = [oracle.solve_chol, oracle.solve_svd]
HERE = os.path.dirname(os.path.abspath(__file__))


def _positive_eigs_bruteforce(A, B):
    H = inputs.assemble_h1(A, B)
    ev, V = np.linalg.eig(H)
    pos = ev.real > 0
    order = np.argsort(ev.real[pos])
    return ev.real[pos][order], V[:, pos][:, order], ev


# --- omega against independent solvers ---------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17, 32])
@pytest.mark.parametrize("solve", SOLVERS)
def test_omega_vs_bruteforce_nonsymmetric_eig(n, solve):
    """Thm. 5 / Lemma ComputeNegEvecs: H1 has n positive eigenvalues, +-paired; the
    oracle's omega equal the positive eigenvalues of numpy.linalg.eig(H1)."""
    A, B = inputs.base(n, seed=n)
    ref, Vref, ev = _positive_eigs_bruteforce(A, B)
    assert len(ref) == n
    assert np.allclose(np.sort(ev.real), np.sort(np.concatenate([-ref, ref])), rtol=0, atol=1e-12 * ref.max())
    omega, X, Y = solve(A, B)
    assert np.max(np.abs(omega - ref)) <= 1e-13 * ref.max()
    # eigenvectors: Sigma-normalise eig's vectors and compare after phase alignment
    if n <= 8:
        Xr, Yr = Vref[:n], Vref[n:]
        s = np.sqrt(np.real(np.sum(np.abs(Xr) ** 2 - np.abs(Yr) ** 2, axis=0)))
        Xr, Yr = phase_align(Xr / s, Yr / s)
        Xo, Yo = phase_align(X, Y)
        assert np.max(np.abs(Xo - Xr)) < 1e-11 and np.max(np.abs(Yo - Yr)) < 1e-11


@pytest.mark.parametrize("n", [64, 160])
@pytest.mark.parametrize("solve", SOLVERS)
def test_omega_vs_hermitian_definite_pencil(n, solve):
    """Eq. (1)-(3): H1 = Sigma Hcal1; the pencil Sigma v = mu Hcal1 v (Hcal1 PD,
    solved by LAPACK through scipy.linalg.eigh) has mu = 1/lambda."""
    A, B = inputs.base(n, seed=100 + n)
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    Hc = np.block([[Af, Bf], [Bf, Af]])
    S = np.diag(np.concatenate([np.ones(n), -np.ones(n)]))
    mu = sla.eigh(S, Hc, eigvals_only=True)
    ref = np.sort(1.0 / mu[mu > 0])
    omega, _, _ = solve(A, B, vectors=False)
    assert np.max(np.abs(omega - ref)) <= 1e-13 * ref.max()
    assert np.max(np.abs(omega - ref) / ref) <= 1e-13


@pytest.mark.parametrize("solve", SOLVERS)
def test_commuting_closed_form(solve):
    """A = Q diag(a) Q^H, B = Q diag(b) Q^H commute: omega_i = sqrt(a_i^2 - b_i^2),
    x_i = alpha_i q_i, y_i = beta_i q_i with beta = (omega - a) alpha / b and
    alpha^2 - beta^2 = 1 (from H [x; y] = omega [x; y] and Sigma-normalisation)."""
    n = 96
    A, B, a, b, Q = inputs.commuting(n, seed=1)
    omega, X, Y = solve(A, B)
    om_exact = np.sqrt(a * a - b * b)
    order = np.argsort(om_exact)
    assert np.max(np.abs(omega - om_exact[order]) / om_exact[order]) < 1e-13
    r = (om_exact - a) / b
    alpha = 1.0 / np.sqrt(1.0 - r * r)
    beta = r * alpha
    Xe = Q[:, order] * alpha[order][None, :]
    Ye = Q[:, order] * beta[order][None, :]
    Xe, Ye = phase_align(Xe, Ye)
    Xo, Yo = phase_align(X, Y)
    assert np.max(np.abs(Xo - Xe)) < 1e-10 and np.max(np.abs(Yo - Ye)) < 1e-10


def test_paper_e1_closed_form_and_table1():
    """Section 4 accuracy workload: omega = sqrt(3)/2 d.  The SVD oracle's relative error
    of the smallest eigenvalue stays within the accuracy class the paper prints for
    CHOL+SVD (Table 1) -- a bound, since the paper's random Q is not reproducible."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_table1.json")))
    n = g["n"]
    for kappa, paper_err in zip(g["kappa"], g["rel_err"]["CHOL+SVD"]):
        A, B, d = inputs.paper_e1(n, kappa, seed=7)
        omega, _, _ = oracle.solve_svd(A, B, vectors=False)
        exact = np.sqrt(3.0) / 2.0 * d
        err_small = abs(omega[0] - exact[0]) / exact[0]
        assert err_small <= max(100 * paper_err, 1e-13), (kappa, err_small, paper_err)
        assert np.max(np.abs(omega - exact)) <= 1e-12 * exact.max()


def test_tamm_dancoff_b_zero():
    """B = 0 (Tamm-Dancoff, Section 4 LiF discussion): omega = eig(A), Y = 0."""
    n = 48
    A, _ = inputs.base(n, seed=3)
    B = np.zeros_like(A)
    lam = np.linalg.eigvalsh(inputs.hermitian_full(A))
    for solve in SOLVERS:
        omega, X, Y = solve(A, B)
        assert np.max(np.abs(omega - lam)) < 1e-13 * lam.max()
        assert np.max(np.abs(Y)) < 1e-13
        assert np.max(np.abs(X.conj().T @ X - np.eye(n))) < 1e-13


@pytest.mark.parametrize("ab", [(2.0, 1.0), (3.0, -2.5), (1.0, 0.0)])
def test_scalar_case(ab):
    """n = 1: H = [a b; -b -a] has eigenvalues +-sqrt(a^2 - b^2)."""
    a, b = ab
    A = np.array([[a]], dtype=np.complex128)
    B = np.array([[b]], dtype=np.complex128)
    for solve in SOLVERS:
        omega, X, Y = solve(A, B)
        assert abs(omega[0] - np.sqrt(a * a - b * b)) < 1e-15 * a
        assert abs(abs(X[0, 0]) ** 2 - abs(Y[0, 0]) ** 2 - 1) < 1e-14


# --- invariants -------------------------------------------------------------------

@pytest.mark.parametrize("solve", SOLVERS)
def test_trace_and_logdet_invariants(solve):
    """Thm. ProdEig: omega^2 are the eigenvalues of M1 M2, hence
    sum omega^2 = tr(M1 M2) and sum 2 log omega = log det M1 + log det M2."""
    n = 128
    A, B = inputs.base(n, seed=11)
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    M1, M2 = Af + Bf, Af - Bf
    omega, _, _ = solve(A, B, vectors=False)
    tr = np.real(np.trace(M1 @ M2))
    assert abs(np.sum(omega ** 2) - tr) < 1e-12 * tr
    ld = np.linalg.slogdet(M1)[1] + np.linalg.slogdet(M2)[1]
    assert abs(np.sum(2 * np.log(omega)) - ld) < 1e-11 * max(1.0, abs(ld))


@pytest.mark.parametrize("solve", SOLVERS)
def test_sigma_orthogonality_pairing_and_lemmas(solve):
    """Thm. ProdEig Eq. (13): X^H X - Y^H Y = I; cross pairs X^H Y - Y^H X = 0;
    Lemma ComputeNegEvecs: [Y; X] is the eigenvector of -omega; the Lemmas for
    Alg. 2 / Alg. 3: with V1 = X - Y and V2 = X + Y, V1^H V2 = I and
    M1 V2 M2 V1 relate by Lambda (M2 V1 = V2 Lambda^{a}, M1 V2 = V1 Lambda^{2-a})."""
    n = 96
    A, B = inputs.base(n, seed=5)
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    omega, X, Y = solve(A, B)
    assert sigma_residual(X, Y) < 1e-12
    assert np.max(np.abs(X.conj().T @ Y - Y.conj().T @ X)) < 1e-12
    assert eig_residual(A, B, omega, X, Y) < 1e-15 * np.sqrt(n) * 10
    # negative half
    R1 = Af @ Y + Bf @ X + Y * omega
    R2 = -Bf @ Y - Af @ X + X * omega
    assert max(np.abs(R1).max(), np.abs(R2).max()) < 1e-12 * omega.max()
    V1, V2 = X - Y, X + Y
    assert np.max(np.abs(V1.conj().T @ V2 - np.eye(n))) < 1e-12
    # both scalings satisfy M2 V1 Lambda^{-1/2} ... : the product form is scaling-free
    lhs = (Af - Bf) @ V1
    rhs = V2 * omega[None, :]
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * omega.max()
    lhs = (Af + Bf) @ V2
    rhs = V1 * omega[None, :]
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * omega.max()


# --- the building blocks ----------------------------------------------------------

def test_cholesky_blocks_and_not_pd():
    n = 40
    A, B = inputs.base(n, seed=2)
    M = inputs.hermitian_full(A - B)
    L = oracle.cholesky(A - B)
    assert np.allclose(L, np.tril(L)) and np.all(np.real(np.diag(L)) > 0)
    assert np.max(np.abs(np.imag(np.diag(L)))) == 0
    assert np.max(np.abs(L @ L.conj().T - M)) < 1e-14 * np.abs(M).max() * n
    assert np.max(np.abs(L - np.linalg.cholesky(M))) < 1e-13
    bad = np.eye(6, dtype=np.complex128)
    bad[3, 3] = -1.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.cholesky(bad)
    assert e.value.info == 4
    nan = np.eye(5, dtype=np.complex128)
    nan[2, 2] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.cholesky(nan)
    assert e.value.info == 3


def test_solvers_report_not_pd():
    n = 8
    A = np.eye(n, dtype=np.complex128)
    B = np.eye(n, dtype=np.complex128) * 1.5  # A - B = -0.5 I: not PD
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve_chol(A, B)
    assert e.value.code == oracle.ERR_NOT_PD_AMINUSB and e.value.info == 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.solve_svd(A, -B)  # A + B = -0.5 I
    assert e.value.code == oracle.ERR_NOT_PD_APLUSB


def test_congruence_and_product_vs_dense_products():
    n = 37
    A, B = inputs.base(n, seed=9)
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    L1 = np.linalg.cholesky(Af + Bf)
    L2 = np.linalg.cholesky(Af - Bf)
    M = oracle.congruence(Af + Bf, L2)
    assert np.max(np.abs(M - L2.conj().T @ (Af + Bf) @ L2)) < 1e-13
    G = oracle.product(L1, L2)
    assert np.max(np.abs(G - L1.conj().T @ L2)) < 1e-13
    # singular values of L1^H L2 are omega (Lemma SVDScalarFactors); not those of L1 L2^H
    sv = np.linalg.svd(G, compute_uv=False)
    om = oracle.solve_svd(A, B, vectors=False)[0]
    assert np.max(np.abs(np.sort(sv) - om)) < 1e-13 * om.max()


def test_jacobi_svd_and_eigh_vs_lapack():
    n = 45
    rng = np.random.default_rng(4)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    s, U, V, sweeps = oracle.jacobi_svd(G)
    assert 1 <= sweeps <= 20
    assert np.max(np.abs(np.sort(s) - np.sort(np.linalg.svd(G, compute_uv=False)))) < 1e-13 * s.max()
    assert np.max(np.abs(U.conj().T @ U - np.eye(n))) < 1e-13
    assert np.max(np.abs(V.conj().T @ V - np.eye(n))) < 1e-13
    assert np.max(np.abs((U * s) @ V.conj().T - G)) < 1e-13 * s.max()
    M = G @ G.conj().T + np.eye(n)
    lam, W, sweeps = oracle.jacobi_eigh(M)
    assert np.max(np.abs(np.sort(lam) - np.linalg.eigvalsh(M))) < 1e-13 * lam.max()
    assert np.max(np.abs(W.conj().T @ W - np.eye(n))) < 1e-13
    assert np.max(np.abs((W * lam) @ W.conj().T - M)) < 1e-12 * lam.max()


def test_thread_count_does_not_change_bits():
    n = 50
    A, B = inputs.base(n, seed=21)
    t0 = oracle.get_threads()
    try:
        oracle.set_threads(1)
        r1 = oracle.solve_svd(A, B)
        c1 = oracle.solve_chol(A, B)
        oracle.set_threads(4)
        r4 = oracle.solve_svd(A, B)
        c4 = oracle.solve_chol(A, B)
    finally:
        oracle.set_threads(t0)
    for a, b in zip(r1 + c1, r4 + c4):
        assert np.array_equal(a, b)


# --- gradient -----------------------------------------------------------------------

def test_grad_vs_central_differences():
    """d omega = x^H dA x + y^H dA y + x^H dB y + y^H dB x (Thm. 3 item 3 with the
    Sigma-normalisation): compare <G, E> with central differences, h = 1e-6."""
    n, k = 24, 5
    A, B = inputs.base(n, seed=31)
    A, B = inputs.hermitian_full(A), inputs.hermitian_full(B)
    w = inputs.grad_weights(k, seed=1)
    omega, X, Y = oracle.solve_svd(A, B)
    dA, dB = oracle.grad(X[:, :k], Y[:, :k], w)
    assert np.max(np.abs(dA - dA.conj().T)) < 1e-14 and np.max(np.abs(dB - dB.conj().T)) < 1e-14
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(6):
        EA = inputs.hermitian_direction(n, rng)
        EB = inputs.hermitian_direction(n, rng)
        Lp = w @ oracle.solve_svd(A + h * EA, B + h * EB, vectors=False)[0][:k]
        Lm = w @ oracle.solve_svd(A - h * EA, B - h * EB, vectors=False)[0][:k]
        fd = (Lp - Lm) / (2 * h)
        an = np.real(np.vdot(dA, EA) + np.vdot(dB, EB))
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (fd, an)


def test_grad_commuting_closed_form():
    """Commuting A, B: d omega_i/d a_i = a_i/omega_i and d omega_i/d b_i = -b_i/omega_i,
    so G_A = sum w_i (a_i/omega_i) q_i q_i^H and G_B = sum w_i (-b_i/omega_i) q_i q_i^H."""
    n, k = 40, 6
    A, B, a, b, Q = inputs.commuting(n, seed=3)
    omega, X, Y = oracle.solve_chol(A, B)
    w = inputs.grad_weights(k, seed=1)
    dA, dB = oracle.grad(X[:, :k], Y[:, :k], w)
    om_exact = np.sqrt(a * a - b * b)
    order = np.argsort(om_exact)[:k]
    q = Q[:, order]
    GA = (q * (w * a[order] / om_exact[order])[None, :]) @ q.conj().T
    GB = (q * (w * -b[order] / om_exact[order])[None, :]) @ q.conj().T
    assert np.max(np.abs(dA - GA)) < 1e-11 and np.max(np.abs(dB - GB)) < 1e-11
