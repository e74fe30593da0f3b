"""Sparse-block-grid reaction-diffusion on B300 (sm_103a).

A from-scratch implementation of the time-stepping hot path of Stark &
Sbalzarini's image-based porous-media pipeline (arXiv 2304.11165): forward-
Euler FTCS of a reaction-diffusion PDE on a geometry-adapted sparse block
grid built from a level-set phi, with the no-flux rule at phi = 0, bulk and
surface reactions, FP64 monitoring reductions, effective diffusivity and
tortuosity.  All compute runs in the hand-written CUDA kernels of
``libsbg.so`` behind the C ABI of ``include/sbg.h``.
"""
from ._abi import SbgError, load  # noqa: F401
from .api import Grid, State, make_params, redistance, stability_limit  # noqa: F401
