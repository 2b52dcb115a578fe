"""Out-of-core plans (paper_2008_08825_gb300/ooc.py) on the CPU: executed with
numpy tiles under a device budget of a few tiles, the tile Cholesky and the
congruence M = L^H (A + B) L reproduce the dense results; every plan keeps
within its budget; transfers fall as the budget grows and reach the
compulsory minimum when everything fits; and the planner's estimate for the
n = 1e5 problem (Section 4's size) is reported."""
import numpy as np
import pytest

from paper_2008_08825_gb300 import inputs, ooc


def _problem(n):
    A, B = inputs.base(n, seed=11)
    A, B = inputs.hermitian_full(A), inputs.hermitian_full(B)
    return A + B, A - B


@pytest.mark.parametrize("n,nb,budget", [(256, 64, 3), (256, 64, 5), (320, 64, 8), (256, 32, 6)])
def test_tile_cholesky_and_congruence_match_dense(n, nb, budget):
    M1, M2 = _problem(n)
    nt = n // nb
    tasks = ooc.cholesky_tasks(nt, nb, "L") + ooc.congruence_tasks(nt, nb, "M1", "L", "W", "M")
    ops = ooc.plan(tasks, budget, keep={"L", "M"})
    host = {**ooc.tiles_of(M2, nb, "L"), **ooc.tiles_of(M1, nb, "M1")}
    stats = ooc.simulate(tasks, ops, host, budget, nb)
    assert stats["peak"] <= budget
    L = np.tril(ooc.assemble(host, "L", nt, nb))
    L_ref = np.linalg.cholesky(M2)
    assert np.max(np.abs(L - L_ref)) <= 1e-12 * np.abs(L_ref).max()
    M = ooc.assemble(host, "M", nt, nb)
    M_ref = np.tril(L_ref.conj().T @ M1 @ L_ref)
    assert np.max(np.abs(np.tril(M) - M_ref)) <= 1e-12 * np.abs(M_ref).max()


def test_plans_respect_budget_and_transfer_monotone():
    nt, nb = 8, 16
    tasks = ooc.cholesky_tasks(nt, nb) + ooc.congruence_tasks(nt, nb)
    loads = []
    for budget in (3, 4, 6, 10, 20, 200):
        ops = ooc.plan(tasks, budget, keep={"L", "M"})
        res = 0
        for op in ops:
            res += {"LOAD": 1, "ALLOC": 1, "FREE": -1}.get(op.kind, 0)
            assert res <= budget
        loads.append(sum(o.kind == "LOAD" for o in ops))
    assert all(a >= b for a, b in zip(loads, loads[1:]))
    # everything resident: each input tile crosses once (L: nt(nt+1)/2, M1: the same)
    assert loads[-1] == nt * (nt + 1)


def test_budget_below_one_task_is_refused():
    tasks = ooc.cholesky_tasks(4, 8)
    with pytest.raises(ValueError):
        ooc.plan(tasks, 2)


def test_estimate_n1e5():
    """n = 102400 in 4096-wide tiles (25 x 25; one tile 268 MB) with 200 GB
    of HBM for tiles: the Cholesky and congruence stages move about the
    compulsory volume and are compute-bound at the FP64 engine's rate."""
    nt, nb = 25, 4096
    tasks = ooc.cholesky_tasks(nt, nb) + ooc.congruence_tasks(nt, nb)
    budget = int(200e9 // (16 * nb * nb))
    ops = ooc.plan(tasks, budget, keep={"L", "M"})
    est = ooc.estimate(tasks, ops, nb)
    print({k: (round(v, 3) if isinstance(v, float) else v) for k, v in est.items()})
    assert est["compute_bound"]
    compulsory = (nt * (nt + 1)) * est["tile_bytes"]  # L and M1 in, L and M out (lower tiles)
    assert est["bytes_moved"] <= 3.0 * compulsory


@pytest.mark.parametrize("budget", [3, 7, 100])
def test_alg2_stage_plan_from_a_and_b(budget):
    # the full tile list of the executor: A - B and A + B formed from tiles of
    # A and B (lower tiles only), then the factorisation and the congruence
    n, nb = 192, 32
    A, B = inputs.base(n, seed=12)
    nt = n // nb
    tasks = ooc.alg2_stage_tasks(nt, nb)
    ops = ooc.plan(tasks, budget, keep={"L", "M"})
    host = {**ooc.tiles_of(A, nb, "A"), **ooc.tiles_of(B, nb, "B")}
    stats = ooc.simulate(tasks, ops, host, budget, nb)
    assert stats["peak"] <= budget
    Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
    L_ref = np.linalg.cholesky(Af - Bf)
    L = np.tril(ooc.assemble(host, "L", nt, nb))
    assert np.max(np.abs(L - L_ref)) <= 1e-12 * np.abs(L_ref).max()
    M_ref = np.tril(L_ref.conj().T @ (Af + Bf) @ L_ref)
    M = np.tril(ooc.assemble(host, "M", nt, nb))
    assert np.max(np.abs(M - M_ref)) <= 1e-12 * np.abs(M_ref).max()


def test_encode_matches_the_executor_contract():
    # every COMPUTE names a task whose tiles the plan made resident, the flags
    # follow the tile positions (diagonal tiles Hermitian or triangular, tiles
    # above the diagonal read conjugate-transposed), POTRF carries its tile row
    nt, nb = 5, 16
    tasks = ooc.alg2_stage_tasks(nt, nb)
    ops = ooc.plan(tasks, 4, keep={"L", "M"})
    names, enc, eops = ooc.encode(tasks, ops)
    assert len(enc) == len(tasks) and len(eops) == len(ops)
    assert len(set(names)) == len(names)
    resident = set()
    for kind, arg in eops:
        if kind in (0, 1):
            assert arg not in resident
            resident.add(arg)
        elif kind == 4:
            resident.remove(arg)
        elif kind == 3:
            assert arg in resident
        else:
            tk, out, in0, in1, flags = enc[arg]
            assert out in resident and (in0 < 0 or in0 in resident) and (in1 < 0 or in1 in resident)
            assert out not in (in0, in1)
    assert not resident
    for t, (tk, out, in0, in1, flags) in zip(tasks, enc):
        a = t.args
        if t.kind == "POTRF":
            assert tk == 2 and flags >> 8 == a["k"] and names[out] == ("L", a["k"], a["k"])
        elif t.kind == "WGEMM":
            i, j, k = a["i"], a["j"], a["k"]
            assert tk == 6
            assert bool(flags & ooc.IN0_HERM) == (i == k) and bool(flags & ooc.IN0_CONJT) == (i < k)
            assert bool(flags & ooc.IN1_LOWER) == (k == j)
            assert names[in0] == ("M1", max(i, k), min(i, k))
        elif t.kind == "MGEMM":
            assert tk == 6 and flags & ooc.IN0_CONJT
            assert bool(flags & ooc.IN0_LOWER) == (a["k"] == a["i"])
        elif t.kind in ("FORM_SUM", "FORM_DIFF"):
            assert names[in0][0] == "A" and names[in1][0] == "B"
