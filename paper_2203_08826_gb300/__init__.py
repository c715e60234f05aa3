"""GB300-native state-vector simulator: gate application by the contraction of
Eq. (1) of arXiv 2203.08826, plus probabilities, sampling, Pauli expectations,
fused k-qubit blocks, batched small circuits and an adjoint gradient.

The compute path is ``libqsim.so`` (hand-written CUDA for sm_103a behind a C
ABI declared in ``include/qsim.h``); the Python layer only marshals arguments.
The library is loaded on first use and raises if it has not been built.
"""
from . import inputs  # noqa: F401  (seeded workload generators; no GPU needed)

__all__ = ["inputs"]


def __getattr__(name):
    # the binding is imported lazily so that the generators work without the .so
    if name in ("qsim", "binding"):
        from . import binding
        return binding
    raise AttributeError(name)
