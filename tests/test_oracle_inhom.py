"""Pins of the oracle's inhomogeneous-diffusion functions (Eq. 6 and the
face-mean update of the functor in Appendix B Listing 6), each against
something other than the oracle itself: the constant-D oracle where the two
must agree, conservation and symmetry of the face-mean flux form, the closed
form of a layered channel's steady state, and the closed values of Eq. 6."""
import numpy as np
import pytest

import oracle
from workloads import Physics, channel_phi, random_blob_phi


def blob(dims, seed, porosity=0.6):
    return random_blob_phi(dims, seed, porosity=porosity, ell=1.7)


def test_unit_factor_equals_constant_diffusivity():
    dims = (14, 12, 10)
    phi = blob(dims, 3)
    ph = Physics(dims=dims, dt=0.04, D=(0.8, 0.0), decay=(0.01, 0.0), dx=(1.0, 0.9, 1.2),
                 dirichlet=(True, False, False, False, False, False), face_value=(1.0, 0, 0, 0, 0, 0))
    u0 = np.random.default_rng(0).uniform(0, 1, phi.shape)
    a = oracle.Problem(phi, ph).run(u0[None], 60)
    b = oracle.Problem(phi, ph, eps=np.ones(phi.shape)).run(u0[None], 60)
    assert np.max(np.abs(a - b)) <= 1e-14


def test_constant_factor_scales_the_diffusivity():
    dims = (13, 11, 9)
    phi = blob(dims, 4)
    ph = Physics(dims=dims, dt=0.05, D=(1.0, 0.0), dx=(1.0, 1.1, 0.9))
    ph2 = Physics(dims=dims, dt=0.05, D=(0.37, 0.0), dx=(1.0, 1.1, 0.9))
    u0 = np.random.default_rng(1).uniform(0, 1, phi.shape)
    a = oracle.Problem(phi, ph, eps=np.full(phi.shape, 0.37)).run(u0[None], 80)
    b = oracle.Problem(phi, ph2).run(u0[None], 80)
    assert np.max(np.abs(a - b)) <= 1e-13


def test_mass_conserved_with_a_varying_factor():
    """Closed box: the face-mean flux leaves one voxel exactly as it enters the other."""
    dims = (16, 14, 12)
    phi = blob(dims, 5)
    eps = np.random.default_rng(2).uniform(0.1, 1.0, phi.shape)
    ph = Physics(dims=dims, dt=0.1, D=(1.0, 0.0))
    P = oracle.Problem(phi, ph, eps=eps)
    u0 = P.shape_state(np.random.default_rng(3).uniform(0, 1, phi.shape))
    m0 = P.reduce(u0)[0]["mass"]
    u = P.run(u0, 500)
    assert abs(P.reduce(u)[0]["mass"] - m0) <= 1e-12 * m0


def test_step_operator_is_symmetric():
    """<M v, w> = <v, M w> for the step map of a closed box (face coefficients
    D (eps_i + eps_j)/2 are symmetric); using the neighbour's eps alone, or the
    centre's, would break it."""
    dims = (12, 11, 10)
    phi = blob(dims, 6)
    eps = np.random.default_rng(4).uniform(0.2, 1.0, phi.shape)
    ph = Physics(dims=dims, dt=0.05, D=(1.0, 0.0), dx=(1.0, 1.2, 0.8))
    P = oracle.Problem(phi, ph, eps=eps)
    rng = np.random.default_rng(5)
    v = P.shape_state(rng.standard_normal(phi.shape))
    w = P.shape_state(rng.standard_normal(phi.shape))
    lhs = float((P.step(v) * w).sum())
    rhs = float((v * P.step(w)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


def test_layered_channel_steady_state_closed_form():
    """A full channel whose factor varies along x: the steady flux is the same
    through every face, so u drops across face k in proportion to 1/eps_face(k),
    eps_face = (eps_k + eps_{k+1}) / 2; D_eff is the harmonic mean of the face
    diffusivities."""
    nx, ny, nz = 24, 3, 2
    phi = np.full((nz, ny, nx), 5.0, np.float32)
    ex = np.random.default_rng(7).uniform(0.2, 1.0, nx)
    eps = np.broadcast_to(ex[None, None, :], phi.shape).copy()
    ph = Physics(dims=(nx, ny, nz), dt=0.1, D=(0.7, 0.0),
                 dirichlet=(True, True, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    P = oracle.Problem(phi, ph, eps=eps)
    u0 = np.zeros(phi.shape)
    u0[:, :, 0] = 1.0
    u, rel, _ = P.steady_cg(u0[None])
    assert rel < 1e-13
    ef = 0.5 * (ex[:-1] + ex[1:])
    drop = np.cumsum(1.0 / ef) / np.sum(1.0 / ef)
    expect = np.concatenate([[1.0], 1.0 - drop])
    assert np.max(np.abs(u[0, 0, :] - expect)) <= 1e-12
    d_eff, tau, psi = P.effective_D(u[None])
    assert abs(d_eff - 0.7 * (nx - 1) / np.sum(1.0 / ef)) <= 1e-12


def test_eq6_closed_values():
    phi = np.array([-50.0, -0.25, 0.0, 0.25, 50.0], np.float32)
    eps = oracle.eps_sigmoid(phi, 0.1, 0.9, 1.0, 4.0)
    assert abs(eps[0] - 0.1) < 1e-15 and abs(eps[-1] - 1.0) < 1e-15
    # g1 + g2 phi = 0 at phi = -0.25: the midpoint d_min + d_max / 2
    assert abs(eps[1] - (0.1 + 0.45)) < 1e-15
    assert abs(eps[2] - (0.1 + 0.9 / (1.0 + np.exp(-1.0)))) < 1e-15
    assert np.all(np.diff(eps) > 0)


def test_maximum_principle_with_a_varying_factor():
    dims = (15, 13, 11)
    phi = blob(dims, 8)
    eps = np.random.default_rng(9).uniform(0.05, 1.0, phi.shape)
    dx = (1.0, 1.0, 1.0)
    dt = 1.0 / (2.0 * 1.0 * 3.0)  # the limit for D max(eps) <= 1
    ph = Physics(dims=dims, dt=dt, D=(1.0, 0.0), dx=dx,
                 dirichlet=(True, False, False, False, False, False), face_value=(1.0, 0, 0, 0, 0, 0))
    P = oracle.Problem(phi, ph, eps=eps)
    u = P.shape_state(np.random.default_rng(10).uniform(0, 1, phi.shape))
    for _ in range(20):
        u = P.run(u, 10)
        act = P.active > 0
        assert u[0][act].min() >= -1e-15 and u[0][act].max() <= 1.0 + 1e-15


def test_inhomogeneous_reduction_terms_against_their_definitions():
    """Fluxes with the face-mean factor and the residual (u' - u) / dt over the
    free voxels, by numpy, for a random factor and held x faces."""
    dims = (10, 8, 7)
    phi = blob(dims, 12)
    eps = np.random.default_rng(12).uniform(0.2, 1.3, phi.shape)
    ph = Physics(dims=dims, dt=0.03, D=(0.7, 0.0), decay=(0.03, 0.0), dx=(0.9, 1.0, 1.2),
                 dirichlet=(True, True, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    P = oracle.Problem(phi, ph, eps=eps)
    u = P.shape_state(np.random.default_rng(13).uniform(0, 1, phi.shape)[None])
    red = P.reduce(u)[0]
    act = P.active > 0
    free = act & (P.fixed == 0)
    lhs = (P.step(u)[0] - u[0]) / 0.03
    res = float(np.sqrt(np.sum(lhs[free] ** 2)))
    assert abs(red["residual"] - res) <= 1e-9 * res
    for key, p0 in (("J_in", 0), ("J_out", dims[0] - 2)):
        both = act[:, :, p0] & act[:, :, p0 + 1]
        f = 0.5 * (eps[:, :, p0] + eps[:, :, p0 + 1])
        j = 0.7 * float(np.sum((f * (u[0][:, :, p0] - u[0][:, :, p0 + 1]))[both])) / 0.9 * (1.0 * 1.2)
        assert abs(red[key] - j) <= 1e-12 * max(1.0, abs(j)), (key, red[key], j)
