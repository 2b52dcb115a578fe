"""Out-of-core tile executor (bse_ooc_run) on the GPU against the oracle.

The BLAS3 stages of Alg. 2 -- A - B and A + B formed from tiles of A and B,
the Cholesky factorisation L L^H = A - B (step 1) and the congruence
M = L^H (A + B) L (step 2) -- run with A and B in host memory through a
device budget of a few tiles (heavy eviction) up to everything resident.
L and M are compared element by element with the oracle's Cholesky and
congruence, and omega = sqrt(eig(M)) (step 3) with the oracle's Alg. 2
eigenvalues.  A plan that breaks residency or the budget is refused before
anything runs; a non-positive-definite A - B reports its global column.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2008_08825_gb300 import bse, inputs, ooc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def _oracle_stages(A, B):
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    L = oracle.cholesky(Af - Bf)
    return L, oracle.congruence(Af + Bf, L)


@pytest.mark.parametrize("n,nb,budget", [(384, 64, 3), (768, 128, 5), (768, 192, 8), (512, 128, 100),
                                         (1024, 128, 6)])
def test_ooc_stages_vs_oracle(n, nb, budget):
    A, B = inputs.base(n, seed=21)
    plan = ooc.DevicePlan(A, B, nb, budget)
    plan.run()
    L, M = plan.results()
    stats = plan.stats
    # tasks overlap on several streams, ordered only by the tiles they share:
    # a second run gives the same bits
    plan.run()
    L2, M2 = plan.results()
    assert np.array_equal(L, L2) and np.array_equal(M, M2)
    L_ref, M_ref = _oracle_stages(A, B)
    assert np.max(np.abs(L - np.tril(L_ref))) <= 1e-12 * np.abs(L_ref).max()
    assert np.max(np.abs(M - np.tril(M_ref))) <= 1e-12 * np.abs(M_ref).max()
    if n <= 768:  # Alg. 2 step 3 on the executor's M against the oracle's eigenvalues
        omega = np.sqrt(np.linalg.eigvalsh(M, UPLO="L"))
        om_ref, _, _ = oracle.solve_chol(A, B, vectors=False)
        assert np.max(np.abs(omega - om_ref) / om_ref) <= 1e-11
    nt = n // nb
    if budget >= 100:  # everything fits: each input tile crosses once, each result once
        assert stats["loads"] == 2 * nt * (nt + 1) // 2 and stats["stores"] == 2 * nt * (nt + 1) // 2


def test_ooc_not_positive_definite_reports_global_column():
    n, nb = 256, 64
    A = np.eye(n, dtype=np.complex128)
    B = 0.5 * np.eye(n, dtype=np.complex128)
    B[170, 170] = 1.5  # A - B = 0.5 I with -0.5 at column 171 (tile row 2)
    with pytest.raises(bse.BseError) as e:
        ooc.run_device(A, B, nb, 4)
    assert e.value.code == 2 and e.value.info == 171


def test_ooc_inconsistent_plans_are_refused():
    nb = 16
    tiles = [torch.zeros((nb, nb), dtype=torch.complex128) for _ in range(3)]
    before = [t.clone() for t in tiles]
    task = [(ooc.TASK_KINDS["GEMM"], 2, 0, 1, 0)]
    bad_plans = [
        ([(2, 0)], 3),                                  # COMPUTE with nothing resident
        ([(0, 0), (0, 1), (0, 2)], 2),                  # more tiles resident than the budget
        ([(0, 0), (0, 0)], 3),                          # LOAD of a resident tile
        ([(3, 1)], 3),                                  # STORE of a tile that is not resident
        ([(0, 0), (0, 1), (0, 2), (2, 5)], 3),          # task index out of range
        ([(0, 7)], 3),                                  # tile index out of range
    ]
    for ops, budget in bad_plans:
        with pytest.raises(bse.BseError) as e:
            bse.ooc_run(nb, tiles, ops, task, budget)
        assert e.value.code == 1, ops
    for t, b in zip(tiles, before):
        assert torch.equal(t, b)
    # the same three tiles in a consistent plan: C -= A B^H
    rng = np.random.default_rng(3)
    a, b, c = (rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb)) for _ in range(3))
    for t, x in zip(tiles, (a, b, c)):
        t.copy_(torch.from_numpy(np.ascontiguousarray(x.T)))
    bse.ooc_run(nb, tiles, [(0, 0), (0, 1), (0, 2), (2, 0), (3, 2), (4, 0), (4, 1), (4, 2)], task, 3)
    got = tiles[2].numpy().T
    assert np.max(np.abs(got - (c - a @ b.conj().T))) <= 1e-13 * nb
