"""GB300-native solvers for the form-I Bethe-Salpeter eigenproblem
H1 = [A B; -B -A] (Benner & Penke, arXiv 2008.08825): the Cholesky method
(Alg. 2) and the SVD method (Alg. 3), plus the eigenvalue gradient.

The compute path is the C-ABI library ``libbse_gb300.so`` (hand-written CUDA
for sm_103a); :mod:`paper_2008_08825_gb300.bse` is the thin ctypes binding.
Importing this package does not load the library; the first solver call
does, and fails loudly if it is missing.
"""

__all__ = ["solve", "grad", "Omega"]


def __getattr__(name):
    if name in ("solve", "grad", "Omega", "Handle", "BseError", "lib"):
        import importlib

        return getattr(importlib.import_module(__name__ + ".bse"), name)
    raise AttributeError(name)
