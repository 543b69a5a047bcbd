"""GB300-native single-GPU solver for the 2D shallow-water equations on
unstructured triangular meshes: the time-explicit finite-volume step of
Delmas & Soulaimani (HLLC fluxes with hydrostatic reconstruction,
semi-implicit Manning friction, CFL min-reduction), as fused CUDA kernels for
sm_103a behind the C ABI in include/swe.h.

``capi`` is the binding of that ABI; ``meshgen`` holds the seeded synthetic
inputs; ``build`` compiles the library in-tree.
"""
from . import capi  # noqa: F401
from .capi import (SWE_BC_INFLOW, SWE_BC_STAGE, SWE_BC_TRANSMISSIVE, SWE_BC_WALL,  # noqa: F401
                   SWE_FP32, SWE_FP64, SWE_REORDER_HILBERT, SWE_REORDER_NONE, SWE_REORDER_RCM,
                   Mesh, SWEError)
