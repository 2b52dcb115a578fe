"""Shared pytest configuration.

Markers: ``gpu`` -- needs a CUDA GPU (sm_103a) and the built library; every
other test runs on the CPU.  Only tests may import the CPU oracle.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    return oracle.load()


def phase_align(X: np.ndarray, Y: np.ndarray):
    """Rotate each column pair (x_i, y_i) so that the largest-modulus entry of
    [x_i; y_i] (first index on ties) is real and positive."""
    V = np.vstack([X, Y])
    idx = np.argmax(np.abs(V) - 1e-300 * np.arange(V.shape[0])[:, None], axis=0)
    ph = V[idx, np.arange(V.shape[1])]
    ph = np.where(np.abs(ph) > 0, ph / np.abs(ph), 1.0)
    return X / ph[None, :], Y / ph[None, :]


def sigma_residual(X: np.ndarray, Y: np.ndarray) -> float:
    """||V^H Sigma V - I||_F for V = [X; Y] (the paper's Fig. 2 metric)."""
    S = X.conj().T @ X - Y.conj().T @ Y
    return float(np.linalg.norm(S - np.eye(S.shape[0])))


def eig_residual(A, B, omega, X, Y) -> float:
    """||H V - V Lambda||_F / (||H||_F ||V||_F) for H = [A B; -B -A]."""
    from paper_2008_08825_gb300.inputs import hermitian_full

    Af, Bf = hermitian_full(A), hermitian_full(B)
    R1 = Af @ X + Bf @ Y - X * omega[None, :]
    R2 = -Bf @ X - Af @ Y - Y * omega[None, :]
    nh = np.sqrt(2 * np.linalg.norm(Af) ** 2 + 2 * np.linalg.norm(Bf) ** 2)
    nv = np.sqrt(np.linalg.norm(X) ** 2 + np.linalg.norm(Y) ** 2)
    return float(np.sqrt(np.linalg.norm(R1) ** 2 + np.linalg.norm(R2) ** 2) / (nh * nv))
