"""Pins of the oracle's simulated-FRAP functions (Sec. 3.3): the box sum
against brute force and additivity, the recovery curve of a bleached cube in
a bulk box against the closed form of the discrete no-flux problem (cosine
modes of the 7-point Laplacian), and the time-scale fit against curves whose
scale is known exactly."""
import numpy as np
import pytest

import oracle
from workloads import Physics, centred_box, frap_initial, random_blob_phi


def test_box_sum_is_the_plain_masked_sum():
    rng = np.random.default_rng(5)
    dims = (9, 7, 6)
    phi = random_blob_phi(dims, 5, porosity=0.6, ell=1.5)
    P = oracle.Problem(phi, Physics(dims=dims, dt=0.05))
    u = rng.uniform(-1, 1, phi.shape)
    pore = phi > np.finfo(np.float32).eps
    for lo, hi in [((0, 0, 0), (9, 7, 6)), ((2, 1, 3), (7, 5, 6)), ((-3, -2, -1), (4, 40, 3)), ((5, 5, 5), (5, 7, 6)),
                   ((8, 0, 0), (20, 20, 20))]:
        s, c = P.box_sum(u[None], lo, hi)
        box = np.zeros(phi.shape, bool)
        box[max(lo[2], 0):hi[2], max(lo[1], 0):hi[1], max(lo[0], 0):hi[0]] = True
        m = box & pore
        assert c == int(m.sum())
        assert abs(s - float(np.sum(u[m]))) <= 1e-13 * max(1.0, float(np.sum(np.abs(u[m]))))


def test_box_sum_is_additive_and_the_whole_box_is_the_mass():
    dims = (12, 10, 8)
    phi = random_blob_phi(dims, 6, porosity=0.5, ell=1.7)
    P = oracle.Problem(phi, Physics(dims=dims, dt=0.05))
    u = np.random.default_rng(6).uniform(0, 1, phi.shape)
    whole, n = P.box_sum(u[None], (0, 0, 0), dims)
    a, na = P.box_sum(u[None], (0, 0, 0), (5, 10, 8))
    b, nb = P.box_sum(u[None], (5, 0, 0), (12, 10, 8))
    assert n == na + nb and abs(whole - (a + b)) <= 1e-13 * whole
    red = P.reduce(u[None])[0]
    assert n == red["n_active"] and abs(whole - red["mass"]) <= 1e-13 * whole


def closed_form_curve(dims, dx, D, dt, lo, hi, box_lo, box_hi, steps_per_sample, n_samples):
    """Box sums of a bleached cube (u = 1 outside [lo, hi), 0 inside) in a
    closed bulk box, from the cosine eigenmodes of the cell-centred no-flux
    Laplacian: mode k along an axis of n cells is cos(pi k (i + 1/2) / n) with
    eigenvalue -(2 - 2 cos(pi k / n)) / h^2, and forward Euler multiplies a
    3-D mode by 1 + D dt (sum of its three eigenvalues) per step."""
    coef, bsum, mu = [], [], []
    for a in range(3):
        n, h = dims[a], dx[a]
        i = np.arange(n) + 0.5
        k = np.arange(n)
        v = np.cos(np.pi * np.outer(k, i) / n)  # [k, i]
        chi = np.zeros(n)
        chi[lo[a]:hi[a]] = 1.0
        coef.append(v @ chi / np.sum(v * v, axis=1))
        bsum.append(v[:, box_lo[a]:box_hi[a]].sum(axis=1))
        mu.append(-(2.0 - 2.0 * np.cos(np.pi * k / n)) / (h * h))
    lam = 1.0 + D * dt * (mu[0][:, None, None] + mu[1][None, :, None] + mu[2][None, None, :])
    w = np.einsum("i,j,k->ijk", coef[0] * bsum[0], coef[1] * bsum[1], coef[2] * bsum[2])
    nbox = np.prod([box_hi[a] - box_lo[a] for a in range(3)])
    return np.array([nbox - np.sum(w * lam ** (s * steps_per_sample)) for s in range(n_samples + 1)])


@pytest.mark.parametrize("dx", [(1.0, 1.0, 1.0), (1.0, 0.8, 1.3)])
def test_bulk_recovery_matches_the_closed_form(dx):
    dims = (14, 12, 11)
    phi = np.full(tuple(reversed(dims)), 5.0, np.float32)
    ph = Physics(dims=dims, dt=0.1, dx=dx, D=(0.9, 0.0))
    lo, hi = (4, 3, 2), (9, 8, 7)
    u0 = frap_initial(phi.shape, lo, hi)
    sums, count = oracle.Problem(phi, ph).frap_curve(u0[None], lo, hi, 7, 12)
    assert count == 125
    ref = closed_form_curve(dims, dx, 0.9, 0.1, lo, hi, lo, hi, 7, 12)
    np.testing.assert_allclose(sums, ref, rtol=0, atol=1e-11)
    assert sums[0] == 0.0 and np.all(np.diff(sums) > 0)
    # another box than the bleached one
    blo, bhi = (0, 0, 0), (6, 12, 4)
    sums2, _ = oracle.Problem(phi, ph).frap_curve(u0[None], blo, bhi, 5, 6)
    np.testing.assert_allclose(sums2, closed_form_curve(dims, dx, 0.9, 0.1, lo, hi, blo, bhi, 5, 6), atol=1e-11)


def test_fit_recovers_a_known_scale():
    t = np.linspace(0, 10, 41)
    tr = np.linspace(0, 10, 4001)
    s, rss = oracle.frap_fit(t, 1 - np.exp(-0.37 * t), tr, 1 - np.exp(-tr))
    assert abs(s - 0.37) <= 1e-10 and rss <= 1e-20
    # off the reference grid the interpolation error bounds the fit
    s, _ = oracle.frap_fit(t, 1 - np.exp(-0.4137 * t), tr, 1 - np.exp(-tr))
    assert abs(s - 0.4137) <= 1e-5


def test_fit_of_half_the_diffusivity_is_one_half():
    """Forward Euler at (D / 2, dt) makes the same steps as (D, dt / 2), so the
    bulk curve at D / 2 sampled at t equals the curve at D sampled at t / 2:
    the fitted scale is 1/2 exactly."""
    dims = (12, 12, 12)
    phi = np.full(dims, 5.0, np.float32)
    lo, hi = centred_box(dims, 4)
    u0 = frap_initial(phi.shape, lo, hi)
    half = oracle.Problem(phi, Physics(dims=dims, dt=0.12, D=(0.5, 0.0)))
    full = oracle.Problem(phi, Physics(dims=dims, dt=0.06, D=(1.0, 0.0)))
    f, n = half.frap_curve(u0[None], lo, hi, 4, 20)
    fr, _ = full.frap_curve(u0[None], lo, hi, 4, 40)
    t = 0.12 * 4 * np.arange(21)
    tr = 0.06 * 4 * np.arange(41)
    s, rss = oracle.frap_fit(t, f / n, tr, fr / n, 0.05, 1.0)
    assert abs(s - 0.5) <= 1e-9 and rss <= 1e-20


def test_porous_recovery_is_slower_than_bulk():
    """Obstacles hinder the recovery (tortuosity >= 1, Eq. 2): the fitted
    scale lies in (0, 1); a pore space that fills the box gives exactly 1."""
    dims = (16, 16, 16)
    phi = random_blob_phi(dims, 9, porosity=0.7, ell=1.8)
    bulk = np.full(phi.shape, 5.0, np.float32)
    lo, hi = centred_box(dims, 6)
    u0 = frap_initial(phi.shape, lo, hi)
    ph = Physics(dims=dims, dt=0.15, D=(1.0, 0.0))
    P, B = oracle.Problem(phi, ph), oracle.Problem(bulk, ph)
    f, n = P.frap_curve(u0[None], lo, hi, 4, 30)
    total, nact = P.box_sum(P.shape_state(u0[None]), (0, 0, 0), dims)
    fb, nbk = B.frap_curve(u0[None], lo, hi, 4, 30)
    tb, nb = B.box_sum(B.shape_state(u0[None]), (0, 0, 0), dims)
    t = 0.15 * 4 * np.arange(31)
    F = f / (total / nact * n)
    Fb = fb / (tb / nb * nbk)
    s, _ = oracle.frap_fit(t, F, t, Fb, 0.01, 1.0)
    assert 0.05 < s < 1.0
    s1, rss1 = oracle.frap_fit(t, Fb, t, Fb, 0.01, 1.0)
    assert abs(s1 - 1.0) <= 1e-12 and rss1 == 0.0
