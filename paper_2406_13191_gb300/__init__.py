"""GB300-native Lagrange-dual DCOPF bounds (projected gradient ascent, arXiv 2406.13191).

The compute path is libdcopfdual.so (hand-written sm_103a CUDA behind the C ABI of
include/dcopf_dual.h).  ``DcopfDual`` marshals torch tensors into that ABI; torch is
used only for device memory and streams.
"""
from .dual import DcopfDual, SolveResult, solve_group  # noqa: F401
