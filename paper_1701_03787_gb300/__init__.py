"""Batched Shen-Galerkin wall-normal solves on NVIDIA GB300.

Hot path of the channel-flow solver of Mortensen, arXiv:1701.03787: per Fourier
mode one Helmholtz solve (Shen Dirichlet basis), one biharmonic solve (Shen
biharmonic basis) and the right-hand-side operators of Eqs. gfin / ufin, with the
paper's O(N) direct algorithms in hand-written sm_103a CUDA behind the C ABI of
``include/shensolve.h``.  ``binding`` is the Python view of that ABI.
"""
from .binding import BatchPlan, Plan, ShenError, lib, PRECISIONS, PROBLEMS  # noqa: F401

__all__ = ["BatchPlan", "Plan", "ShenError", "lib", "PRECISIONS", "PROBLEMS"]
