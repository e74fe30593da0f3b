"""Seeded synthetic porous geometries, returned as level-set fields phi.

The paper builds phi by Sussman redistancing of segmented micro-CT images
(Sec. 2.2, Eqs. 4-5).  The images are not available, so the workloads use
synthetic stand-ins with the porosities and grain shapes of the paper's
samples: sphere packings (granular beds like the CaCO3 packing of Sec. 3.3)
and thresholded Gaussian random fields.  phi follows the sign convention of
Eq. 3: positive in the pore space Omega, negative in the solid, zero on the
interface.

PRNG: numpy ``Generator(PCG64(seed))`` everywhere.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# ---------------------------------------------------------------------------
# sphere packings
# ---------------------------------------------------------------------------
def sphere_pack_nonoverlap(n: int, count: int, rmin: float, rmax: float, seed: int,
                           max_tries: int = 200000):
    """`count` non-overlapping spheres in the box [0, n-1]^3.

    Centres are uniform in the box, radii uniform in [rmin, rmax]; a candidate
    is rejected while it overlaps an accepted sphere (|c_i - c_j| < r_i + r_j).
    Returns (centres [count, 3] as (x, y, z), radii [count]).
    """
    rng = make_rng(seed)
    centres, radii = [], []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("sphere packing did not reach the requested count")
        c = rng.uniform(0.0, n - 1.0, size=3)
        r = rng.uniform(rmin, rmax)
        ok = True
        for cj, rj in zip(centres, radii):
            if np.linalg.norm(c - cj) < r + rj:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(r)
    return np.array(centres), np.array(radii)


def phi_spheres(dims, centres, radii) -> np.ndarray:
    """Exact phi = min_i(|x - c_i| - r_i) at integer voxel centres (FP64 -> FP32).

    `dims` = (Nx, Ny, Nz); the result is shaped [Nz, Ny, Nx].  Positive in the
    pore space between the spheres, negative inside them.
    """
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    phi = np.full((nz, ny, nx), np.inf)
    for c, r in zip(centres, radii):
        d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) - r
        np.minimum(phi, d, out=phi)
    return phi.astype(np.float32)


def boolean_sphere_pack(n: int, median: float, sigma_ln: float, porosity: float, seed: int,
                        cutoff: float = 4.0):
    """Overlapping (Boolean-model) polydisperse sphere packing in an n^3 box.

    Spheres with centres uniform in [0, n)^3 and radii lognormal (median
    `median`, log-standard-deviation `sigma_ln`) are added one by one until the
    pore fraction (phi > 0) drops to `porosity` or below.  phi is the minimum of
    the per-sphere signed distances, evaluated exactly wherever it is below
    `cutoff` and clamped to `cutoff` further away from every sphere (only the
    sign of phi and its values in the band 0 < phi < 1 enter the method).

    Returns (phi [n, n, n] float32, number of spheres, pore fraction).
    """
    rng = make_rng(seed)
    phi = np.full((n, n, n), np.float32(cutoff), dtype=np.float32)
    n_total = n ** 3
    n_pore = n_total
    count = 0
    ax = np.arange(n, dtype=np.float64)
    while n_pore > porosity * n_total:
        c = rng.uniform(0.0, n, size=3)
        r = float(np.exp(np.log(median) + sigma_ln * rng.standard_normal()))
        reach = r + cutoff
        lo = [max(0, int(np.floor(c[a] - reach))) for a in range(3)]
        hi = [min(n, int(np.ceil(c[a] + reach)) + 1) for a in range(3)]
        if any(h <= l for l, h in zip(lo, hi)):
            count += 1
            continue
        dx2 = (ax[lo[0]:hi[0]] - c[0]) ** 2
        dy2 = (ax[lo[1]:hi[1]] - c[1]) ** 2
        dz2 = (ax[lo[2]:hi[2]] - c[2]) ** 2
        d = (np.sqrt(dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]) - r).astype(np.float32)
        view = phi[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        was_pore = view > 0
        np.minimum(view, d, out=view)
        n_pore -= int(np.count_nonzero(was_pore & (view <= 0)))
        count += 1
    return phi, count, n_pore / n_total


# ---------------------------------------------------------------------------
# Gaussian random fields
# ---------------------------------------------------------------------------
def gaussian_random_field(dims, ell: float, seed: int) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field, shaped [Nz, Ny, Nx].

    i.i.d. N(0, 1) noise is convolved (periodic FFT) with a Gaussian kernel of
    standard deviation ell / sqrt(2); the field's covariance is then
    C(r) = exp(-r^2 / (2 ell^2)), i.e. a Gaussian covariance with correlation
    length ell voxels.
    """
    nx, ny, nz = dims
    rng = make_rng(seed)
    noise = rng.standard_normal((nz, ny, nx))
    s = ell / np.sqrt(2.0)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    kernel_hat = np.exp(-2.0 * np.pi ** 2 * s ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    field = np.fft.irfftn(np.fft.rfftn(noise) * kernel_hat, s=(nz, ny, nx), axes=(0, 1, 2))
    field -= field.mean()
    field /= field.std()
    return field


def threshold_to_porosity(field: np.ndarray, porosity: float) -> np.ndarray:
    """Boolean pore mask holding exactly round(porosity * N) voxels: the largest field values."""
    flat = field.ravel()
    k = int(round(porosity * flat.size))
    mask = np.zeros(flat.size, dtype=bool)
    if k > 0:
        idx = np.argpartition(-flat, k - 1)[:k]
        mask[idx] = True
    return mask.reshape(field.shape)


def phi_from_pore_mask(pore: np.ndarray) -> np.ndarray:
    """Signed distance from a binary image by an exact Euclidean distance transform.

    Pore voxel: (distance to the nearest solid voxel centre) - 0.5.
    Solid voxel: -((distance to the nearest pore voxel centre) - 0.5).
    The half-voxel offset puts phi = 0 on the voxel faces between the phases.
    A box without solid (or without pore) gets +/- (box diagonal).
    """
    pore = np.asarray(pore, dtype=bool)
    big = float(np.sqrt(sum(s * s for s in pore.shape))) + 1.0
    if pore.all():
        return np.full(pore.shape, big, dtype=np.float32)
    if not pore.any():
        return np.full(pore.shape, -big, dtype=np.float32)
    d_pore = ndimage.distance_transform_edt(pore)     # pore voxels: distance to the nearest solid
    d_solid = ndimage.distance_transform_edt(~pore)   # solid voxels: distance to the nearest pore
    phi = np.where(pore, d_pore - 0.5, -(d_solid - 0.5))
    return phi.astype(np.float32)


# ---------------------------------------------------------------------------
# small geometries for tests
# ---------------------------------------------------------------------------
def channel_phi(dims, y_range, z_range) -> np.ndarray:
    """Solid block pierced by one straight pore channel running along x.

    The pore is every voxel with y in [y0, y1) and z in [z0, z1), for all x.
    """
    nx, ny, nz = dims
    pore = np.zeros((nz, ny, nx), dtype=bool)
    pore[z_range[0]:z_range[1], y_range[0]:y_range[1], :] = True
    return phi_from_pore_mask(pore)


def random_blob_phi(dims, seed: int, porosity: float = 0.5, ell: float = 2.0) -> np.ndarray:
    """Small random geometry for brute-force comparisons: a thresholded GRF
    with a short correlation length, so that it has many isolated pores,
    thin throats and single-voxel features."""
    field = gaussian_random_field(dims, ell, seed)
    pore = threshold_to_porosity(field, porosity)
    return phi_from_pore_mask(pore)
