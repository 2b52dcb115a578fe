"""The stored full-size accuracy values (tests/golden/c3_*.npz) are what the
committed script writes: for the small copies (n = 256) the inputs rebuilt
from the generator and the stored shift hash to the stored digest on any
host, and the oracle, run again, gives the stored omega bit for bit on the
kind of machine that wrote them (its results do not depend on its thread
count).  On another architecture the C library's elementary functions may
round differently, so there the oracle agrees to rounding level only."""
import glob
import os
import platform
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_c3_oracle as mk  # noqa: E402

SMALL = sorted(glob.glob(os.path.join(HERE, "golden", "c3_n256_seed0_*.npz")))


def _load(path):
    z = np.load(path)
    case = str(z["case"])
    shift = (z["u"], float(z["c"])) if "u" in z.files else None
    return z, case, shift


@pytest.mark.parametrize("path", SMALL, ids=[os.path.basename(p) for p in SMALL])
def test_small_golden_reproduces(path):
    z, case, shift = _load(path)
    n, seed = int(z["n"]), int(z["seed"])
    A, B, _ = mk.build_inputs(n, seed, case, shift=shift)
    assert mk.input_hash(A, B) == str(z["sha256"])
    om, _, _ = oracle.solve_svd(A, B, vectors=False)
    ref = z["omega"]
    made_on = str(z["machine"]) if "machine" in z.files else "x86_64"
    if platform.machine() == made_on:
        assert np.array_equal(om, ref)
    else:
        assert np.max(np.abs(om - ref)) <= 1e-13 * ref.max()


def test_golden_cases_present():
    assert {os.path.basename(p) for p in SMALL} >= {"c3_n256_seed0_base.npz", "c3_n256_seed0_1e10.npz"}
