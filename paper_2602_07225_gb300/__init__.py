"""GB300-native (sm_103a) block-preconditioned Newton-Krylov hot path of the
pseudo-4D DFN battery model (arXiv 2602.07225).

The compute lives in the C-ABI library ``libp4d.so`` (``include/p4d.h``);
this package only marshals arguments: torch tensors on the CUDA device supply
memory and streams.  There is no CPU fallback.
"""
from ._native import P4DError, load  # noqa: F401
from .solver import P4DSolver, default_params  # noqa: F401
from .adjoint import TerminalVoltage, terminal_voltage  # noqa: F401
from .batch import BatchSolver, Autotuner  # noqa: F401
