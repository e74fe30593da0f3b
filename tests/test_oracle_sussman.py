"""Pins of the oracle's Sussman redistancing (Sec. 2.1: the redistancing PDE
with the smoothed sign, first-order Godunov differences): exact distance
fields are fixed points, a step indicator relaxes to the exact distance from
the voxel face between its phases, the scheme is odd in phi and never
changes a voxel's sign, and the unit ball's error in the narrow band of
width 4h is first order in h (the appendix's convergence figure)."""
import math

import numpy as np
import pytest

import oracle


def test_planar_distance_fields_are_fixed_points():
    nz, ny, nx = 6, 9, 11
    dx = (0.5, 0.7, 1.0)
    z, y, x = np.meshgrid(*(np.arange(n) * d for n, d in zip((nz, ny, nx), dx[::-1])), indexing="ij")
    # axis-aligned: the upwind neighbour never lies beyond the box (an oblique
    # plane loses a gradient component at the zero-gradient box faces)
    for n in [(1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0)]:
        phi = n[0] * (x - 2.3) + n[1] * (y - 3.1) + n[2] * (z - 2.2)
        out = oracle.sussman(phi, dx=dx, cfl=0.3, iters=25)
        assert np.max(np.abs(out - phi)) <= 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_step_indicator_relaxes_to_the_exact_distance(axis):
    n, m, h = 30, 11, 0.5
    shape = [1, 1, 1]
    shape[2 - axis] = n
    idx = np.arange(n)
    phi0 = np.where(idx < m, -1.0, 1.0).reshape(shape)
    dx = [1.0, 1.0, 1.0]
    dx[axis] = h
    out = oracle.sussman(phi0, dx=tuple(dx), cfl=0.3, iters=400)
    exact = ((idx - m + 0.5) * h).reshape(shape)
    assert np.max(np.abs(out - exact)) <= 1e-10
    # the same in a 3-D box (a half-space indicator)
    phi3 = np.broadcast_to(phi0, tuple(5 if s == 1 else s for s in shape)).copy()
    out3 = oracle.sussman(phi3, dx=tuple(dx), cfl=0.3, iters=400)
    assert np.max(np.abs(out3 - np.broadcast_to(exact, phi3.shape))) <= 1e-10


def test_odd_symmetry_and_sign_preservation():
    rng = np.random.default_rng(3)
    phi0 = np.where(rng.uniform(size=(9, 10, 12)) < 0.5, -1.0, 1.0)
    phi0[2, 3, 4] = 0.0
    a = oracle.sussman(phi0, dx=(1.0, 0.9, 1.1), cfl=0.3, iters=30)
    b = oracle.sussman(-phi0, dx=(1.0, 0.9, 1.1), cfl=0.3, iters=30)
    np.testing.assert_array_equal(a, -b)
    assert np.all(np.sign(a) == np.sign(phi0))
    assert a[2, 3, 4] == 0.0


def ball(n):
    h = 4.0 / n
    c = -2.0 + (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    return np.where(r < 1.0, 1.0, -1.0), 1.0 - r, h


def test_unit_ball_error_is_first_order_in_the_band():
    l2 = []
    for n in (32, 64, 128):
        ind, sdf, h = ball(n)
        out = oracle.sussman(ind, dx=(h, h, h), cfl=0.3, iters=60)
        band = np.abs(sdf) < 2 * h
        e = out[band] - sdf[band]
        l2.append(math.sqrt(np.mean(e * e)))
        assert np.max(np.abs(e)) <= 0.35 * h and l2[-1] <= 0.2 * h, (n, l2[-1] / h)
    assert math.log(l2[0] / l2[-1], 2.0) / 2.0 >= 0.9, l2


def test_smoothed_sign_does_not_depend_on_the_steepness_of_phi():
    """The smoothed sign phi / sqrt(phi^2 + |grad phi|^2 h^2) is the same for
    phi and a*phi, the property it is chosen for (the form phi / sqrt(phi^2 +
    h^2) is not).  On a linear field of slope s along x, |grad phi| = s at
    every voxel, so one iteration moves each voxel by dalpha sigma (1 - s):
    the sigma recovered from a*phi (slope a*s) equals that from phi."""
    nx, h, cfl = 16, 1.0, 0.3
    x = np.arange(nx, dtype=np.float64) * h
    base = 0.5 * (x - 7.3)
    sig = []
    for a in (1.0, 3.0):
        phi = (a * base).reshape(1, 1, nx)
        out = oracle.sussman(phi, dx=(h, 1.0, 1.0), cfl=cfl, iters=1)
        move = (out - phi).ravel()
        sig.append(move / (cfl * h * (1.0 - a * 0.5)))
    np.testing.assert_allclose(sig[0], sig[1], rtol=1e-12, atol=0)
    assert np.all(np.sign(sig[0]) == np.sign(base))


def test_a_zero_field_stays_zero():
    """phi = 0 everywhere (no interface to measure from) is left unchanged and
    finite: a voxel with phi = 0 does not move."""
    phi = np.zeros((4, 5, 6))
    out = oracle.sussman(phi, cfl=0.3, iters=5)
    assert np.all(out == 0.0)
