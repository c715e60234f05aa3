"""GB300-native state-vector simulator: gate application by the contraction of
Eq. (1) of arXiv 2203.08826, plus probabilities, sampling, Pauli expectations,
fused k-qubit blocks, batched small circuits and an adjoint gradient.

The compute path is ``libqsim.so`` (hand-written CUDA for sm_103a behind the C
ABI declared in ``include/qsim.h``); ``binding`` only marshals arguments and
loads the library on first use, raising if it has not been built.
"""
from . import inputs  # noqa: F401  (seeded workload generators; no GPU needed)
