"""Write the oracle's omega for the full-size accuracy configuration.

The configuration is the base workload at n = 8192 (seed 0) and the kappa(A - B)
sweep 1e2 / 1e6 / 1e10 on it, the paper's accuracy experiment (Section 4,
Table 1) scaled to the benchmark's size.  The oracle's reference answer is its
Alg. 3 pipeline (Cholesky factors, G = L1^H L2, one-sided Jacobi), whose
singular values have high relative accuracy.  Nothing here runs the CUDA path.

One file per case, ``c3_n<n>_seed<seed>_<case>.npz``, holding:
  omega     the n positive eigenvalues, ascending (oracle.solve_svd)
  u, c      the kappa cases' rank-one shift, so that inputs.kappa_sweep(...,
            shift=(u, c)) rebuilds the same matrices bit for bit on any host
            (the shift itself comes from LAPACK and is platform dependent)
  sha256    hash of A and B (complex128, column-major bytes): the test checks
            that it rebuilt exactly the matrices the oracle saw
  seconds, threads, machine   metadata for the record

Usage (hours at n = 8192 on a few cores; each case is written when done):
    python tests/golden/make_c3_oracle.py --n 8192 --cases base,1e2,1e6,1e10
"""
from __future__ import annotations

import argparse
import hashlib
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2008_08825_gb300 import inputs  # noqa: E402


def case_path(n: int, seed: int, case: str) -> str:
    return os.path.join(HERE, f"c3_n{n}_seed{seed}_{case}.npz")


def input_hash(A: np.ndarray, B: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.asfortranarray(A).tobytes(order="F"))
    h.update(np.asfortranarray(B).tobytes(order="F"))
    return h.hexdigest()


def build_inputs(n: int, seed: int, case: str, shift=None):
    """(A, B, extra) for one case; extra holds the shift of a kappa case."""
    if case == "base":
        A, B = inputs.base(n, seed)
        return A, B, {}
    kappa = float(case)
    if shift is None:
        u, c, est = inputs.kappa_shift(n, kappa, seed)
    else:
        (u, c), est = shift, None
    A, B, _ = inputs.kappa_sweep(n, kappa, seed, shift=(u, c))
    extra = {"u": u, "c": np.float64(c), "kappa": np.float64(kappa)}
    if est is not None:
        extra["kappa_estimate"] = np.float64(est)
    return A, B, extra


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cases", default="base,1e2,1e6,1e10")
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    if args.threads:
        oracle.set_threads(args.threads)
    for case in [c for c in args.cases.split(",") if c]:
        out = case_path(args.n, args.seed, case)
        A, B, extra = build_inputs(args.n, args.seed, case)
        digest = input_hash(A, B)
        t0 = time.time()
        omega, _, _ = oracle.solve_svd(A, B, vectors=False)
        dt = time.time() - t0
        np.savez(out, omega=omega, sha256=np.array(digest), n=np.int64(args.n), seed=np.int64(args.seed),
                 case=np.array(case), seconds=np.float64(dt), threads=np.int64(oracle.get_threads()),
                 machine=np.array(platform.machine()), **extra)
        print(f"{case}: n={args.n} {dt:.0f} s, omega[0]={omega[0]:.17g} -> {os.path.basename(out)}", flush=True)


if __name__ == "__main__":
    main()
