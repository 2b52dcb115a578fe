"""The seeded input generators (CPU): the properties the workloads promise —
definiteness, the requested conditioning, the closed forms' structure,
determinism, and the prefix property of the batched sizes that the sharded
batched bench relies on (512 N instances for N ranks extend the 512 of one)."""
import numpy as np
import pytest

from paper_2008_08825_gb300 import inputs


@pytest.mark.parametrize("n", [1, 7, 64, 257])
def test_base_is_hermitian_definite_and_deterministic(n):
    A, B = inputs.base(n, seed=3)
    A2, B2 = inputs.base(n, seed=3)
    assert np.array_equal(A, A2) and np.array_equal(B, B2)
    assert A.flags.f_contiguous and B.flags.f_contiguous and A.dtype == np.complex128
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    assert np.allclose(Af, Af.conj().T) and np.allclose(Bf, Bf.conj().T)
    # Weyl: d >= 1 and ||0.1 G_A -+ 0.05 G_B|| ~ 0.3 keep A +- B positive definite
    for M in (Af + Bf, Af - Bf):
        assert np.linalg.eigvalsh(M).min() > 0.5
    assert not np.array_equal(A, inputs.base(n, seed=4)[0])


def test_commuting_instance_structure():
    n = 40
    A, B, a, b, Q = inputs.commuting(n, seed=1)
    assert np.allclose(Q.conj().T @ Q, np.eye(n), atol=1e-13)
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    assert np.allclose(Af, (Q * a) @ Q.conj().T, atol=1e-12)
    assert np.allclose(Bf, (Q * b) @ Q.conj().T, atol=1e-12)
    assert np.allclose(Af @ Bf, Bf @ Af, atol=1e-11)
    om = inputs.commuting_omega(a, b)
    assert np.all(np.diff(om) >= 0) and np.all(om > 0)


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_kappa_sweep_sets_the_condition_of_a_minus_b(kappa):
    n = 96
    A, B, est = inputs.kappa_sweep(n, kappa, seed=0)
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    ev = np.linalg.eigvalsh(Af - Bf)
    assert ev.min() > 0
    achieved = ev.max() / ev.min()
    assert abs(achieved / kappa - 1.0) < 0.05, achieved
    assert abs(est / achieved - 1.0) < 0.05
    # A + B keeps the base generator's spectrum away from zero
    assert np.linalg.eigvalsh(Af + Bf).min() > 0.5


def test_batched_sizes_range_and_prefix_property():
    s512 = inputs.batched_sizes()
    assert len(s512) == 512 and s512.min() >= 32 and s512.max() <= 1024
    s2048 = inputs.batched_sizes(count=2048)
    assert np.array_equal(s2048[:512], s512)
    # log-uniform: the median sits near the geometric mean of the range
    assert 120 < np.median(s512) < 260


def test_directions_and_weights():
    rng = np.random.default_rng(2)
    E = inputs.hermitian_direction(12, rng)
    assert np.allclose(E, E.conj().T) and abs(np.linalg.norm(E) - 1.0) < 1e-14
    w = inputs.grad_weights(16, seed=1)
    assert w.shape == (16,) and np.array_equal(w, inputs.grad_weights(16, seed=1))


def test_assemble_h1_is_form_one():
    A, B = inputs.base(5, seed=9)
    H = inputs.assemble_h1(A, B)
    n = 5
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    assert np.array_equal(H[:n, :n], Af) and np.array_equal(H[:n, n:], Bf)
    assert np.array_equal(H[n:, :n], -Bf) and np.array_equal(H[n:, n:], -Af)
