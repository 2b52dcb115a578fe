"""The oracle's pins are sharp enough: each plausible slip, planted in a copy
of the oracle's C source (a dropped 1/2, a wrong sign, a missing conjugate, a
transposed product, a wrong power of Lambda, a wrong rotation sign), is
caught by a small battery of the pins in test_oracle_pins.py (CPU only; the
mutants are built with gcc into a temporary directory).
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2008_08825_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "bse_oracle.c")

MUTANTS = {
    "final setup drops the 1/2 in X": ("AT(X, i, jj, ldx) = 0.5 * (v1 + v2);", "AT(X, i, jj, ldx) = (v1 + v2);"),
    "final setup flips the sign of Y": ("AT(Y, i, jj, ldy) = 0.5 * (v2 - v1);", "AT(Y, i, jj, ldy) = 0.5 * (v1 - v2);"),
    "product L1^T conj(L2) instead of L1^H L2": (
        "s += conj(AT(L1, k, i, ld1)) * AT(L2, k, j, ld2);", "s += AT(L1, k, i, ld1) * conj(AT(L2, k, j, ld2));"),
    "CHOL scales V1 by Lambda instead of Lambda^(1/2)": ("double sc = sqrt(om[j]);\n    for (int64_t i = n - 1",
                                                         "double sc = om[j];\n    for (int64_t i = n - 1"),
    "Cholesky update without conjugate": ("zc lkj = conj(AT(L, k, j, ldl));", "zc lkj = AT(L, k, j, ldl);"),
    "one-sided rotation with a wrong sign": ("u[i] = r.c * up - se * vp;", "u[i] = r.c * up + se * vp;"),
    "two-sided row rotation without conjugate phase": ("zc e = conj(rt.eph);", "zc e = rt.eph;"),
    "M2 = A + B instead of A - B": ("form_m(n, A, lda, B, ldb, -1.0, M2);\n  int64_t col = oracle_cholesky(n, M2, n, L, n);",
                                    "form_m(n, A, lda, B, ldb, +1.0, M2);\n  int64_t col = oracle_cholesky(n, M2, n, L, n);"),
    "gradient dB with a wrong sign": ("gb += w[i] * (xa * conj(yb) + ya * conj(xb));",
                                      "gb += w[i] * (xa * conj(yb) - ya * conj(xb));"),
    "SVD recovery uses L2 U instead of L1 U": ("s1 += AT(L1, i, k, n) * AT(U, k, j, n);",
                                               "s1 += AT(L2, i, k, n) * AT(U, k, j, n);"),
}


def _pins_pass(lib) -> bool:
    """A compact battery of pins; False as soon as one fails."""
    for n, seed in ((1, 3), (8, 5)):
        A, B = inputs.base(n, seed=seed)
        H = inputs.assemble_h1(A, B)
        ev = np.linalg.eigvals(H)
        ref = np.sort(ev.real[ev.real > 0])
        for solve in (oracle.solve_chol, oracle.solve_svd):
            try:
                om, X, Y = solve(A, B, lib=lib)
            except oracle.OracleError:
                return False
            if not np.all(np.isfinite(om)) or np.max(np.abs(om - ref)) > 1e-12 * ref.max():
                return False
            S = X.conj().T @ X - Y.conj().T @ Y - np.eye(n)
            if np.linalg.norm(S) > 1e-12:
                return False
            Af, Bf = inputs.hermitian_full(A), inputs.hermitian_full(B)
            R1 = Af @ X + Bf @ Y - X * om
            R2 = -Bf @ X - Af @ Y - Y * om
            if max(np.abs(R1).max(), np.abs(R2).max()) > 1e-12 * om.max():
                return False
    # gradient against central differences
    n, k = 6, 3
    A, B = inputs.base(n, seed=9)
    A, B = inputs.hermitian_full(A), inputs.hermitian_full(B)
    w = inputs.grad_weights(k, seed=1)
    om, X, Y = oracle.solve_svd(A, B)  # reference build for the eigenvectors
    dA, dB = oracle.grad(X[:, :k], Y[:, :k], w, lib=lib)
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(2):
        EA, EB = inputs.hermitian_direction(n, rng), inputs.hermitian_direction(n, rng)
        fd = (w @ oracle.solve_svd(A + h * EA, B + h * EB, vectors=False)[0][:k]
              - w @ oracle.solve_svd(A - h * EA, B - h * EB, vectors=False)[0][:k]) / (2 * h)
        an = np.real(np.vdot(dA, EA) + np.vdot(dB, EB))
        if abs(fd - an) > 1e-7 * max(1.0, abs(an)):
            return False
    return True


def test_unmutated_oracle_passes_the_battery():
    assert _pins_pass(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mpath = tmp_path / "bse_oracle_mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(so), str(mpath), "-lm"],
                   check=True)
    lib = oracle.load(str(so))
    assert not _pins_pass(lib), f"pins did not catch: {name}"
