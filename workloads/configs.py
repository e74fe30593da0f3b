"""The five synthetic workloads: geometry, initial state and physical parameters.

Each workload is named by what it is:

* ``spheres64``    - 64^3 box, 20 non-overlapping spheres, FP64 plain diffusion, 100 steps.
* ``grf256``       - 256^3 thresholded Gaussian random field (porosity 0.35), steady-state
                     tortuosity solve between two Dirichlet faces.
* ``reactive512``  - 512^3 overlapping polydisperse sphere packing (porosity 0.40),
                     two species with a surface reaction A -> B and bulk decay of B, 2000 steps.
* ``gradient_setup`` - the grf256 geometry (or a corner crop of it) with a surface sink,
                     used for the adjoint.
* ``batch_geometries`` - 64 boxes of uneven size and porosity for the batched solve.

Face numbering: 0 = x-low, 1 = x-high, 2 = y-low, 3 = y-high, 4 = z-low, 5 = z-high.
Time steps are given as numbers; each one is 0.9 x the explicit limit
1 / (2 max_s D_s sum_a dx_a^-2 + max rate) (the 3-D form of Eq. 10 with the
largest linear sink rate added), and the tests check them against both
implementations' limit functions.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .geometry import (boolean_sphere_pack, gaussian_random_field, make_rng, phi_from_pore_mask,
                       phi_spheres, sphere_pack_nonoverlap, threshold_to_porosity)

FACE_XLO, FACE_XHI, FACE_YLO, FACE_YHI, FACE_ZLO, FACE_ZHI = range(6)

SEED_SPHERES64 = 1000
SEED_GRF256 = 1001
SEED_REACTIVE512 = 1002
SEED_BATCH_BASE = 2000

DT_PURE_DIFFUSION = 0.15              # 0.9 / (2 * 1 * 3)
DT_SURFACE_SINK = 0.9 / 6.05          # 0.9 / (2 * 1 * 3 + 0.05 * 1), band half-width 1


@dataclass
class Physics:
    """Parameters of one reaction-diffusion run (constant D per species).

    Species 0 ("A") loses k_surf * w(phi) * A per unit time at the surface and
    decay[0] * A in the bulk; with two species the surface loss of A is the
    gain of species 1 ("B"), which decays at decay[1].
    """
    dims: tuple                        # (Nx, Ny, Nz)
    dt: float
    dx: tuple = (1.0, 1.0, 1.0)
    nspecies: int = 1
    D: tuple = (1.0, 0.0)
    decay: tuple = (0.0, 0.0)
    k_surf: float = 0.0
    dirichlet: tuple = (False,) * 6    # per face
    face_value: tuple = (0.0,) * 6     # species-0 value held on each Dirichlet face
    band_eps: float = 1.0              # half-width of the smoothed surface delta, in units of phi
    steps: int = 0
    extra: dict = field(default_factory=dict)


def _dirichlet_x(lo=None, hi=None):
    d = [False] * 6
    v = [0.0] * 6
    if lo is not None:
        d[FACE_XLO], v[FACE_XLO] = True, float(lo)
    if hi is not None:
        d[FACE_XHI], v[FACE_XHI] = True, float(hi)
    return tuple(d), tuple(v)


def initial_with_faces(dims, interior: float, phys: Physics) -> np.ndarray:
    """Dense FP64 initial field [Nz, Ny, Nx]: `interior` everywhere, Dirichlet faces at their value."""
    nx, ny, nz = dims
    u = np.full((nz, ny, nx), float(interior))
    if phys.dirichlet[FACE_XLO]:
        u[:, :, 0] = phys.face_value[FACE_XLO]
    if phys.dirichlet[FACE_XHI]:
        u[:, :, nx - 1] = phys.face_value[FACE_XHI]
    if phys.dirichlet[FACE_YLO]:
        u[:, 0, :] = phys.face_value[FACE_YLO]
    if phys.dirichlet[FACE_YHI]:
        u[:, ny - 1, :] = phys.face_value[FACE_YHI]
    if phys.dirichlet[FACE_ZLO]:
        u[0, :, :] = phys.face_value[FACE_ZLO]
    if phys.dirichlet[FACE_ZHI]:
        u[nz - 1, :, :] = phys.face_value[FACE_ZHI]
    return u


# ---------------------------------------------------------------------------
def spheres64(n: int = 64, seed: int = SEED_SPHERES64):
    """FP64 plain-method case: 20 non-overlapping spheres (radius U(6, 10)),
    analytic phi, c = 1 held on the x-low face, D = 1, dt = 0.1, 100 steps.
    Returns (phi, u0, physics)."""
    centres, radii = sphere_pack_nonoverlap(n, 20, 6.0, 10.0, seed)
    phi = phi_spheres((n, n, n), centres, radii)
    d, v = _dirichlet_x(lo=1.0)
    phys = Physics(dims=(n, n, n), dt=0.1, D=(1.0, 0.0), dirichlet=d, face_value=v, steps=100)
    u0 = initial_with_faces(phys.dims, 0.0, phys)
    return phi, u0, phys


def grf_geometry(n: int, seed: int, porosity: float, ell: float = 8.0) -> np.ndarray:
    """phi of a thresholded Gaussian random field: pore = the top `porosity` fraction."""
    field_ = gaussian_random_field((n, n, n), ell, seed)
    pore = threshold_to_porosity(field_, porosity)
    return phi_from_pore_mask(pore)


def grf256(n: int = 256, seed: int = SEED_GRF256, porosity: float = 0.35):
    """Tortuosity case: GRF (correlation length 8) at porosity 0.35, c = 1 on the
    x-low face and c = 0 on the x-high face, zero initial interior, D = 1,
    dt = 0.15, run to a relative residual of 1e-8.  Returns (phi, u0, physics)."""
    phi = grf_geometry(n, seed, porosity)
    d, v = _dirichlet_x(lo=1.0, hi=0.0)
    phys = Physics(dims=(n, n, n), dt=DT_PURE_DIFFUSION, D=(1.0, 0.0), dirichlet=d, face_value=v,
                   extra={"tol_residual": 1e-8, "porosity_target": porosity})
    u0 = initial_with_faces(phys.dims, 0.0, phys)
    return phi, u0, phys


def reactive512(n: int = 512, seed: int = SEED_REACTIVE512, porosity: float = 0.40, steps: int = 2000):
    """Two-species reactive transport: Boolean polydisperse spheres (lognormal
    radii, median 12, sigma 0.3) at pore fraction 0.40; A: D = 1, surface
    reaction A -> B with k = 0.05 in the band 0 < phi < 1; B: D = 0.5, decay
    0.001; A = 1 for x < 32, B = 0; closed box; dt = 0.9 x limit.
    Returns (phi, u0 [2, Nz, Ny, Nx], physics)."""
    phi, count, psi = boolean_sphere_pack(n, 12.0, 0.3, porosity, seed)
    phys = Physics(dims=(n, n, n), dt=DT_SURFACE_SINK, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.001),
                   k_surf=0.05, steps=steps, extra={"spheres": count, "pore_fraction": psi})
    u0 = np.zeros((2, n, n, n))
    u0[0, :, :, :min(32, n)] = 1.0
    return phi, u0, phys


def inhom512(n: int = 512, seed: int = SEED_REACTIVE512, porosity: float = 0.40, steps: int = 2000):
    """Inhomogeneous diffusion of a solute entering from one face (the paper's
    fertilizer application, Sec. 3.4, on a synthetic packed bed): the
    reactive512 geometry (Boolean spheres, pore fraction 0.40); one species
    with diffusivity D * eps(phi) from Eq. 6 with D_min = 0, D_max = 1,
    gamma2 = 4 per voxel and gamma1 = gamma2 * min(phi over the pore space)
    (the paper's smoothing parameters, gamma2 = 4 read per grid spacing);
    c = 1 held on the x = 0 face, 0 elsewhere initially; dt = 0.9 x limit.
    Returns (phi, u0, physics, (d_min, d_max, gamma1, gamma2))."""
    phi, count, psi = boolean_sphere_pack(n, 12.0, 0.3, porosity, seed)
    pore = phi > np.float32(np.finfo(np.float32).eps)
    g2 = 4.0
    g1 = g2 * float(phi[pore].min())
    d, v = _dirichlet_x(lo=1.0)
    phys = Physics(dims=(n, n, n), dt=DT_PURE_DIFFUSION, D=(1.0, 0.0), dirichlet=d, face_value=v, steps=steps,
                   extra={"spheres": count, "pore_fraction": psi})
    u0 = initial_with_faces(phys.dims, 0.0, phys)
    return phi, u0, phys, (0.0, 1.0, g1, g2)


def centred_box(dims, side):
    """(lo, hi) of the cube of edge ``side`` centred in a box of ``dims`` (x, y, z)."""
    lo = tuple(max((int(n) - int(side)) // 2, 0) for n in dims)
    hi = tuple(min(l + int(side), int(n)) for l, n in zip(lo, dims))
    return lo, hi


def frap_initial(shape_zyx, lo, hi) -> np.ndarray:
    """Bleached initial state: 1 everywhere except 0 in lo <= (x, y, z) < hi."""
    u0 = np.ones(shape_zyx)
    u0[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 0.0
    return u0


def frap256(n: int = 256, seed: int = SEED_GRF256, porosity: float = 0.35, side: int = 64,
            steps_per_sample: int = 128, samples: int = 128):
    """Simulated FRAP (Sec. 3.3) in the grf256 geometry: closed box (no-flux
    on every face), D = 1, dt = 0.15, the centred cube of edge ``side``
    bleached (u = 0 there, 1 elsewhere), the box mass recorded every
    ``steps_per_sample`` steps for ``samples`` samples; the bulk reference is
    the same box with every voxel in the pore space.
    Returns (phi, u0, physics, lo, hi)."""
    phi = grf_geometry(n, seed, porosity)
    phys = Physics(dims=(n, n, n), dt=DT_PURE_DIFFUSION, D=(1.0, 0.0), steps=steps_per_sample * samples,
                   extra={"steps_per_sample": steps_per_sample, "samples": samples, "side": side})
    lo, hi = centred_box(phys.dims, side)
    return phi, frap_initial(phi.shape, lo, hi), phys, lo, hi


def mms_disk(n: int, B: float = 20.0, t_final: float = 0.025, dt_over_h2: float = 0.125):
    """The verification case of Sec. 3.1: diffusion (D = 1) inside the unit
    disk, no flux on r = 1, on an n x n grid of cell centres covering
    [-2, 2]^2 (nz = 1), phi = 1 - r (exact SDF), u0 = r^3/3 - r^4/4, and the
    manufactured source of the appendix, S(r) exp(-B t) with
    S = B r^4 / 4 - B r^3 / 3 + 4 r^2 - 3 r; dt = t_final / ceil(t_final /
    (dt_over_h2 h^2)).  Returns (phi [1, n, n], u0, S, r, physics, nsteps)."""
    h = 4.0 / n
    c = -2.0 + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(c, c, indexing="xy")
    r = np.sqrt(X ** 2 + Y ** 2)
    phi = (1.0 - r).astype(np.float32)[None]
    nsteps = int(np.ceil(t_final / (dt_over_h2 * h * h)))
    dt = t_final / nsteps
    phys = Physics(dims=(n, n, 1), dt=dt, D=(1.0, 0.0), dx=(h, h, 1.0), steps=nsteps,
                   extra={"B": B, "t_final": t_final, "h": h})
    u0 = (r ** 3 / 3 - r ** 4 / 4)[None]
    S = (B / 4 * r ** 4 - B / 3 * r ** 3 + 4 * r ** 2 - 3 * r)[None]
    return phi, u0, S, r, phys, nsteps


def gradient_setup(n: int = 256, crop: int | None = None, steps: int = 1000, seed: int = SEED_GRF256):
    """Adjoint case on the grf256 geometry (or its [0, crop)^3 corner).

    One species A with D = 1 and surface sink k = 0.05 w(phi); A = 1 initially,
    A = 0 held on the x-high face; 1000 steps at dt = 0.9 x limit.  The loss is
    the mean of A over the pore voxels with x > floor(224 * Nx / 256).
    Returns (phi, u0, physics, x_cut)."""
    phi = grf_geometry(n, seed, 0.35)
    if crop is not None:
        phi = np.ascontiguousarray(phi[:crop, :crop, :crop])
    nz, ny, nx = phi.shape
    d, v = _dirichlet_x(hi=0.0)
    phys = Physics(dims=(nx, ny, nz), dt=DT_SURFACE_SINK, D=(1.0, 0.0), k_surf=0.05,
                   dirichlet=d, face_value=v, steps=steps)
    u0 = initial_with_faces(phys.dims, 1.0, phys)
    x_cut = (224 * nx) // 256
    return phi, u0, phys, x_cut


def batch_geometries(count: int = 64, seed_base: int = SEED_BATCH_BASE, sides=(64, 96, 128, 192, 256)):
    """Uneven batch: geometry g has a cubic side drawn from `sides`, a pore
    fraction drawn from U(0.2, 0.6); even g are Boolean sphere packings
    (median radius 12, sigma 0.3), odd g thresholded GRFs (correlation length 8).
    Yields (g, phi, physics) with the grf256 physics (c = 1 / c = 0 on the x
    faces, run to a relative residual of 1e-6)."""
    for g in range(count):
        rng = make_rng(seed_base + g)
        side = int(rng.choice(np.array(sides)))
        psi = float(rng.uniform(0.2, 0.6))
        geo_seed = int(rng.integers(0, 2 ** 31 - 1))
        if g % 2 == 0:
            phi, _, _ = boolean_sphere_pack(side, 12.0, 0.3, psi, geo_seed)
        else:
            phi = grf_geometry(side, geo_seed, psi)
        d, v = _dirichlet_x(lo=1.0, hi=0.0)
        phys = Physics(dims=(side, side, side), dt=DT_PURE_DIFFUSION, D=(1.0, 0.0), dirichlet=d,
                       face_value=v, extra={"tol_residual": 1e-6, "porosity_target": psi,
                                            "kind": "spheres" if g % 2 == 0 else "grf"})
        yield g, phi, phys
