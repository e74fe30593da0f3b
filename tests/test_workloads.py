"""The seeded input generators: sign conventions, porosities, determinism,
and the time steps each workload states (checked against the oracle's limit)."""
import numpy as np

import oracle
from workloads import (Physics, boolean_sphere_pack, channel_phi, gaussian_random_field,
                       gradient_setup, phi_from_pore_mask, phi_spheres, spheres64,
                       sphere_pack_nonoverlap, threshold_to_porosity)
from workloads.configs import DT_PURE_DIFFUSION, DT_SURFACE_SINK


def test_phi_from_mask_matches_brute_force():
    rng = np.random.default_rng(0)
    pore = rng.uniform(size=(5, 6, 7)) < 0.5
    phi = phi_from_pore_mask(pore)
    pts = np.argwhere(np.ones_like(pore))
    for (z, y, x) in pts:
        other = np.argwhere(~pore if pore[z, y, x] else pore)
        d = np.sqrt(((other - np.array([z, y, x])) ** 2).sum(1)).min()
        expect = d - 0.5 if pore[z, y, x] else -(d - 0.5)
        assert abs(phi[z, y, x] - expect) < 1e-5


def test_sphere_phi_sign_and_exactness():
    c, r = sphere_pack_nonoverlap(24, 3, 3.0, 5.0, seed=3)
    phi = phi_spheres((24, 24, 24), c, r)
    for ci, ri in zip(c, r):
        z, y, x = (int(round(ci[2])), int(round(ci[1])), int(round(ci[0])))
        assert phi[z, y, x] < 0
    d = np.min([np.linalg.norm(np.array([5.0, 6.0, 7.0]) - ci) - ri for ci, ri in zip(c, r)])
    assert abs(phi[7, 6, 5] - d) < 1e-5
    for i in range(3):
        for j in range(i):
            assert np.linalg.norm(c[i] - c[j]) >= r[i] + r[j]


def test_grf_threshold_hits_porosity_exactly():
    f = gaussian_random_field((32, 32, 32), 4.0, seed=5)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1) < 1e-12
    pore = threshold_to_porosity(f, 0.35)
    assert pore.sum() == round(0.35 * 32 ** 3)
    np.testing.assert_array_equal(gaussian_random_field((32, 32, 32), 4.0, seed=5), f)


def test_boolean_pack_reaches_target():
    phi, count, psi = boolean_sphere_pack(64, 6.0, 0.3, 0.4, seed=9)
    assert psi <= 0.4 and psi > 0.37
    assert abs((phi > 0).mean() - psi) < 1e-12
    assert count > 10


def test_channel_geometry():
    phi = channel_phi((8, 6, 5), (2, 4), (1, 3))
    assert ((phi > 0).sum()) == 8 * 2 * 2


def test_stated_time_steps_are_point_nine_of_the_limit():
    box = np.full((8, 8, 8), 5.0, dtype=np.float32)
    p1 = Physics(dims=(8, 8, 8), dt=DT_PURE_DIFFUSION, D=(1.0, 0.0))
    assert abs(DT_PURE_DIFFUSION - 0.9 * oracle.Problem(box, p1).stability_limit()) < 1e-15
    p2 = Physics(dims=(8, 8, 8), dt=DT_SURFACE_SINK, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.001),
                 k_surf=0.05)
    assert abs(DT_SURFACE_SINK - 0.9 * oracle.Problem(box, p2).stability_limit()) < 1e-15


def test_small_workloads_build():
    phi, u0, p = spheres64()
    assert phi.shape == (64, 64, 64) and u0[:, :, 0].min() == 1.0 and p.steps == 100
    phi, u0, p, xc = gradient_setup(n=64, crop=48)
    assert phi.shape == (48, 48, 48) and xc == 42 and u0[:, :, -1].max() == 0.0
