"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the bench.

This package only *generates inputs*: level-set fields phi on a voxel box,
initial concentration arrays and the physical parameters of each workload.
It holds none of the method's arithmetic (no stencil, no mask rule, no
reaction weight, no reduction), so that the FP64 oracle and the CUDA path can
both consume it without sharing any computation.

Array convention everywhere: dense numpy arrays shaped ``[Nz, Ny, Nx]``
(x fastest), float32 for phi, float64 for initial states.
"""
from .geometry import (  # noqa: F401
    make_rng,
    sphere_pack_nonoverlap,
    phi_spheres,
    boolean_sphere_pack,
    gaussian_random_field,
    threshold_to_porosity,
    phi_from_pore_mask,
    channel_phi,
    random_blob_phi,
)
from .configs import (  # noqa: F401
    FACE_XLO, FACE_XHI, FACE_YLO, FACE_YHI, FACE_ZLO, FACE_ZHI,
    Physics,
    spheres64,
    grf256,
    grf_geometry,
    reactive512,
    inhom512,
    frap256,
    centred_box,
    frap_initial,
    mms_disk,
    gradient_setup,
    batch_geometries,
)
