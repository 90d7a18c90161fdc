"""GB300 (sm_103a) sketch-and-solve approximate null space.

Park & Nakatsukasa, "A Fast Randomized Algorithm for Computing an Approximate
Null Space": Algorithm 1 (sketch, SVD of the sketch, trailing right singular
vectors) with SRHT, sparse-sign and Gaussian sketches, an FP64 Householder QR
and one-sided Jacobi SVD, and the adjoint of the trailing projector.

The compute path is libns.so (CUDA kernels behind the C ABI of include/ns.h);
``api`` holds the thin ctypes binding with the same names.
"""
from . import workloads  # noqa: F401  (seeded inputs; no method arithmetic)


def __getattr__(name):
    # the binding needs torch; import it lazily so workloads stay importable alone
    if name in ("api",):
        import importlib
        return importlib.import_module(".api", __name__)
    raise AttributeError(name)
