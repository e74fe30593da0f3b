"""Pins of the FP64 oracle to things other than itself: closed forms, exact
invariants, an independent (edge-list) formulation of the masked voxel
graph, finite differences and the numbers the paper prints.

Each test is built so that a plausible slip in the oracle (a dropped term, a
wrong sign, a swapped axis or dx, a mirror rule applied on the wrong side)
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import erfc

import oracle
from workloads import Physics, channel_phi, random_blob_phi

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def phys(dims, dt, **kw):
    return Physics(dims=tuple(dims), dt=dt, **kw)


def open_box(dims):
    nx, ny, nz = dims
    return np.full((nz, ny, nx), 10.0, dtype=np.float32)


def dirich(*faces, values=None):
    d = [False] * 6
    v = [0.0] * 6
    for i, f in enumerate(faces):
        d[f] = True
        if values is not None:
            v[f] = values[i]
    return tuple(d), tuple(v)


# ---------------------------------------------------------------------------
# 1-D reduction and continuum erfc
# ---------------------------------------------------------------------------
def test_open_box_reduces_to_1d_recurrence():
    """A y/z-uniform run in an open box with c = 1 held on x = 0 equals the
    1-D FTCS recurrence with a reflecting far end, built as an explicit
    tridiagonal matrix."""
    nx, ny, nz = 40, 3, 2
    dt, D, n = 0.2, 1.1, 150
    d, v = dirich(0, values=[1.0])
    p = phys((nx, ny, nz), dt, D=(D, 0.0), dirichlet=d, face_value=v)
    P = oracle.Problem(open_box((nx, ny, nz)), p)
    u0 = np.zeros((nz, ny, nx))
    u0[:, :, 0] = 1.0
    u = P.run(u0, n)[0]
    M = np.zeros((nx, nx))
    M[0, 0] = 1.0
    for i in range(1, nx):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < nx]
        M[i, i] = 1.0 - dt * D * len(nb)
        for j in nb:
            M[i, j] = dt * D
    ref = np.linalg.matrix_power(M, n) @ u0[0, 0]
    for z in range(nz):
        for y in range(ny):
            np.testing.assert_allclose(u[z, y], ref, rtol=1e-13, atol=1e-15)


def test_open_box_converges_to_erfc():
    """Half-space diffusion from a held c = 1 plane: the discrete solution
    approaches erfc(x / (2 sqrt(D t))) at second order (dt tied to h^2)."""
    D, t_end, length = 1.0, 0.5, 12.0
    errs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        nx = int(round(length / h)) + 1
        dt0 = 0.2 * h * h / D
        nsteps = int(math.ceil(t_end / dt0))
        dt = t_end / nsteps
        d, v = dirich(0, values=[1.0])
        p = phys((nx, 1, 1), dt, D=(D, 0.0), dx=(h, 1.0, 1.0), dirichlet=d, face_value=v)
        P = oracle.Problem(open_box((nx, 1, 1)), p)
        u0 = np.zeros((1, 1, nx))
        u0[0, 0, 0] = 1.0
        u = P.run(u0, nsteps)[0, 0, 0]
        x = np.arange(nx) * h
        errs.append(np.max(np.abs(u - erfc(x / (2.0 * math.sqrt(D * t_end))))))
    orders = [math.log(errs[i] / errs[i + 1]) / math.log(2.0) for i in range(len(errs) - 1)]
    assert errs[-1] < 2e-3
    assert all(1.7 < o < 2.3 for o in orders), (errs, orders)


# ---------------------------------------------------------------------------
# closed box: discrete cosine modes are exact eigenvectors of the no-flux rule
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, 1, 1)])
def test_closed_box_cosine_modes(k):
    nx, ny, nz = 12, 10, 8
    dx = (1.0, 0.7, 1.3)
    D, dt, n = 0.8, 0.05, 40
    p = phys((nx, ny, nz), dt, D=(D, 0.0), dx=dx)
    P = oracle.Problem(open_box((nx, ny, nz)), p)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.cos(np.pi * k[0] * (x + 0.5) / nx) * np.cos(np.pi * k[1] * (y + 0.5) / ny)
            * np.cos(np.pi * k[2] * (z + 0.5) / nz))
    lam = sum(4.0 * D / dx[a] ** 2 * math.sin(math.pi * k[a] / (2 * N)) ** 2
              for a, N in enumerate((nx, ny, nz)))
    u = P.run(mode, n)[0]
    np.testing.assert_allclose(u, (1.0 - dt * lam) ** n * mode, atol=1e-13)


# ---------------------------------------------------------------------------
# independent formulation: the step as a sparse matrix built from the edge list
# of the active-voxel graph
# ---------------------------------------------------------------------------
def edge_matrix(active, fixed, w, dims, dx, dt, D, decay, k, ns):
    nx, ny, nz = dims
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    act = active.astype(bool)
    free = act & ~fixed.astype(bool)
    blocks = []
    for s in range(ns):
        A = sp.lil_matrix((n, n))
        diag = np.ones(n)
        for a, (sl_lo, sl_hi) in enumerate((
                ((slice(None), slice(None), slice(0, -1)), (slice(None), slice(None), slice(1, None))),
                ((slice(None), slice(0, -1), slice(None)), (slice(None), slice(1, None), slice(None))),
                ((slice(0, -1), slice(None), slice(None)), (slice(1, None), slice(None), slice(None))))):
            c = D[s] / dx[a] ** 2
            both = act[sl_lo] & act[sl_hi]
            i_lo, i_hi = idx[sl_lo][both], idx[sl_hi][both]
            for i, j in zip(i_lo, i_hi):
                A[i, j] += dt * c
                A[j, i] += dt * c
                diag[i] -= dt * c
                diag[j] -= dt * c
        rate = decay[s] + (k * w.ravel() if s == 0 else 0.0)
        diag = diag - dt * rate
        A = A.tocsr() + sp.diags(diag)
        keep = sp.diags(free.ravel().astype(float))
        A = keep @ A + sp.diags((act & ~free).ravel().astype(float))
        blocks.append(A)
    if ns == 1:
        return blocks[0]
    coupling = sp.diags(free.ravel() * dt * k * w.ravel())
    return sp.bmat([[blocks[0], None], [coupling, blocks[1]]]).tocsr()


@pytest.mark.parametrize("seed", [1, 2])
def test_step_equals_edge_list_matrix(seed):
    dims = (9, 7, 6)
    phi = random_blob_phi(dims, seed, porosity=0.55, ell=1.5)
    # add a band of small positive phi so that w varies
    phi = np.where(phi > 0, phi * 0.6, phi).astype(np.float32)
    d, v = dirich(0, 3, values=[1.0, 0.3])
    p = phys(dims, 0.07, nspecies=2, D=(1.0, 0.45), decay=(0.02, 0.3), k_surf=0.9,
             dx=(1.0, 0.8, 1.2), dirichlet=d, face_value=v)
    P = oracle.Problem(phi, p)
    rng = np.random.default_rng(seed)
    u = rng.uniform(0, 1, size=(2,) + phi.shape) * P.active[None]
    M = edge_matrix(P.active, P.fixed, P.w, dims, p.dx, p.dt, p.D, p.decay, p.k_surf, 2)
    ref = (M @ u.ravel()).reshape(u.shape)
    np.testing.assert_allclose(P.step(u), ref, rtol=1e-13, atol=1e-15)
    assert (P.w > 0).sum() > 10 and P.fixed.sum() > 0


def test_active_set_is_strictly_above_the_threshold():
    """A voxel is in Omega only when phi exceeds the FP32 machine epsilon
    (Sec. 3.2; the insertion test of Appendix B Listing 5): phi equal to it,
    zero and negative values are outside, the next FP32 value above is in."""
    eps = np.float32(np.finfo(np.float32).eps)
    vals = np.array([-1.0, 0.0, eps, np.nextafter(eps, np.float32(1)), 0.5], dtype=np.float32)
    phi = vals.reshape(1, 1, 5)
    P = oracle.Problem(phi, phys((5, 1, 1), 0.1, D=(1.0, 0.0)))
    assert P.active.ravel().tolist() == [0, 0, 0, 1, 1]


# ---------------------------------------------------------------------------
# conservation and balance
# ---------------------------------------------------------------------------
def test_mass_conserved_closed_box():
    dims = (24, 24, 24)
    phi = random_blob_phi(dims, 7, porosity=0.5, ell=2.0)
    p = phys(dims, 0.15, D=(1.0, 0.0))
    P = oracle.Problem(phi, p)
    u0 = np.random.default_rng(3).uniform(0, 1, size=phi.shape)
    m0 = P.reduce(u0)[0]["mass"]
    u = P.run(u0, 1000)
    m1 = P.reduce(u)[0]["mass"]
    assert abs(m1 - m0) / m0 < 1e-12


def test_mass_balance_with_held_face():
    """Free mass changes by exactly dt * sum over (held, free) neighbour pairs
    of c (u_held - u_free) dV per step."""
    dims = (16, 12, 10)
    phi = random_blob_phi(dims, 11, porosity=0.6, ell=2.0)
    d, v = dirich(0, values=[1.0])
    p = phys(dims, 0.12, D=(0.9, 0.0), dx=(1.0, 1.1, 0.9), dirichlet=d, face_value=v)
    P = oracle.Problem(phi, p)
    u = np.zeros(phi.shape)
    u[:, :, 0] = 1.0
    u = P.shape_state(u)[0]
    free = (P.active > 0) & (P.fixed == 0)
    dv = np.prod(p.dx)
    c = 0.9 / p.dx[0] ** 2
    for _ in range(30):
        flux = ((P.fixed[:, :, 0] > 0) & free[:, :, 1]) * (u[:, :, 0] - u[:, :, 1])
        expected = p.dt * c * flux.sum() * dv
        un = P.step(u)[0]
        dm = (un[free].sum() - u[free].sum()) * dv
        assert abs(dm - expected) <= 1e-12 * max(1.0, abs(expected))
        u = un


def test_reaction_closed_form_without_diffusion():
    dims = (8, 6, 5)
    phi = random_blob_phi(dims, 5, porosity=0.6, ell=1.5)
    phi = np.where(phi > 0, phi * 0.5, phi).astype(np.float32)
    lam_b = 0.05
    p = phys(dims, 0.3, nspecies=2, D=(0.0, 0.0), decay=(0.0, lam_b), k_surf=0.4)
    P = oracle.Problem(phi, p)
    rng = np.random.default_rng(0)
    u = rng.uniform(0, 1, size=(2,) + phi.shape) * P.active[None]
    a0 = u[0].copy()
    for n in range(1, 25):
        un = P.step(u)
        tot_before = u.sum()
        assert abs(un.sum() - (tot_before - p.dt * lam_b * u[1].sum())) < 1e-12 * tot_before
        u = un
        np.testing.assert_allclose(u[0], (1.0 - p.dt * p.k_surf * P.w) ** n * a0, rtol=1e-12,
                                   atol=1e-15)


def test_maximum_principle_at_the_limit():
    dims = (14, 13, 12)
    phi = random_blob_phi(dims, 21, porosity=0.5, ell=1.2)
    d, v = dirich(0, 1, values=[1.0, 0.0])
    p = phys(dims, 1.0, D=(1.0, 0.0), dirichlet=d, face_value=v)
    P = oracle.Problem(phi, p)
    dt = P.stability_limit()
    u = np.random.default_rng(4).uniform(0, 1, size=phi.shape)
    u[:, :, 0], u[:, :, -1] = 1.0, 0.0
    for _ in range(100):
        u = P.step(u, dt=dt)[0]
        assert u.min() >= -1e-15 and u.max() <= 1 + 1e-15


# ---------------------------------------------------------------------------
# steady state, flux and effective diffusivity
# ---------------------------------------------------------------------------
def test_channel_steady_profile_and_deff():
    """A straight channel between c = 1 and c = 0 has the exact linear steady
    profile and D_eff = D * psi (tau = 1)."""
    dims = (32, 9, 9)
    phi = channel_phi(dims, (3, 6), (2, 7))
    d, v = dirich(0, 1, values=[1.0, 0.0])
    D = 0.7
    dx = (0.7, 1.3, 0.9)
    p = phys(dims, 0.9 / (6 * D), D=(D, 0.0), dx=dx, dirichlet=d, face_value=v)
    P = oracle.Problem(phi, p)
    u0 = np.zeros(phi.shape)
    u0[:, :, 0] = 1.0
    u, rel, it = P.steady_cg(u0)
    assert rel < 1e-13
    lin = 1.0 - np.arange(32) / 31.0
    act = P.active > 0
    np.testing.assert_allclose(u[act], np.broadcast_to(lin, u.shape)[act], atol=1e-12)
    r = P.reduce(u)[0]
    psi_expected = 3 * 5 / (9 * 9)
    deff, tau, psi = P.effective_D(u)
    assert abs(psi - psi_expected) < 1e-15
    assert abs(deff - D * psi_expected) < 1e-12 * D
    assert abs(tau - 1.0) < 1e-12
    assert abs(r["J_in"] - r["J_out"]) < 1e-12


@pytest.mark.parametrize("dx", [(1.0, 1.0, 1.0), (1.0, 0.8, 1.3)])
def test_cg_equals_time_stepping_steady_state(dx):
    """The steady state by CG equals the limit of time stepping, also with a
    different spacing per axis (so that each axis's coefficient is pinned)."""
    dims = (16, 14, 12)
    phi = random_blob_phi(dims, 31, porosity=0.6, ell=2.0)
    d, v = dirich(0, 1, values=[1.0, 0.0])
    p = phys(dims, 0.15, D=(1.0, 0.0), dx=dx, dirichlet=d, face_value=v)
    P = oracle.Problem(phi, p)
    u0 = np.zeros(phi.shape)
    u0[:, :, 0] = 1.0
    u_cg, rel, _ = P.steady_cg(u0)
    assert rel < 1e-13
    u = P.shape_state(u0)[0]
    r0 = P.reduce(u)[0]["residual"]
    for _ in range(200):
        u = P.run(u, 500)[0]
        if P.reduce(u)[0]["residual"] < 1e-13 * r0:
            break
    act = P.active > 0
    assert np.max(np.abs(u[act] - u_cg[act])) < 1e-10
    r = P.reduce(u_cg)[0]
    assert r["J_in"] > 0 and abs(r["J_in"] - r["J_out"]) < 1e-10 * r["J_in"]


def test_tau_orientation_matches_paper_example():
    """tau = D / D_eff,intrinsic (Eq. 2); the paper's 1.0 / 0.55 = 1.82."""
    g = GOLDEN["tortuosity_caco3"]
    dims = np.array([11, 4, 5])
    psi = 0.4
    deff_superficial = g["D_eff_intrinsic"] * psi
    # choose fluxes that give this superficial D_eff: J = D_eff * dC * A / L
    A, L = 4 * 5, 10
    J = deff_superficial * 1.0 * A / L
    import ctypes
    lib = oracle._load()
    out = [ctypes.c_double() for _ in range(3)]
    lib.oracle_effective_D(oracle._p(dims.astype(np.int64)), oracle._p(np.ones(3)), J, J, 1.0,
                           g["D"], psi * 11 * 4 * 5, *[ctypes.byref(o) for o in out])
    assert abs(out[0].value - deff_superficial) < 1e-14
    assert abs(out[1].value - g["tau"]) < 0.005
    assert abs(out[2].value - psi) < 1e-15


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------
def adjoint_problem(seed=3):
    dims = (10, 8, 7)
    phi = random_blob_phi(dims, seed, porosity=0.6, ell=1.5)
    phi = np.where(phi > 0, phi * 0.6, phi).astype(np.float32)
    d, v = dirich(1, values=[0.0])
    p = phys(dims, 0.08, nspecies=2, D=(1.0, 0.5), decay=(0.01, 0.2), k_surf=0.7,
             dirichlet=d, face_value=v)
    return phi, p


def test_adjoint_dot_product():
    phi, p = adjoint_problem()
    P = oracle.Problem(phi, p)
    rng = np.random.default_rng(9)
    free = ((P.active > 0) & (P.fixed == 0))[None]
    v = rng.standard_normal((2,) + phi.shape) * free
    w = rng.standard_normal((2,) + phi.shape) * free
    Mv = P.step(v)
    lam, _ = P.adjoint_step(np.zeros_like(v), w)
    lhs, rhs = float((Mv * w).sum()), float((v * lam).sum())
    assert abs(lhs - rhs) < 1e-13 * max(abs(lhs), 1.0)


def test_adjoint_matches_central_differences():
    phi, p = adjoint_problem(5)
    P = oracle.Problem(phi, p)
    rng = np.random.default_rng(1)
    nsteps = 30
    u0 = rng.uniform(0.2, 1.0, size=(2,) + phi.shape)
    u0[:, :, :, -1] = 0.0
    weights = rng.uniform(0, 1, size=(2,) + phi.shape) * P.active[None]

    def loss_of(prob, u_init):
        return float((prob.run(u_init, nsteps) * weights).sum())

    lam0, grad, _ = P.adjoint_run(u0, nsteps, weights)
    import dataclasses
    for which, base in (("D0", p.D[0]), ("D1", p.D[1]), ("k", p.k_surf)):
        h = 1e-3 * base

        def perturbed(delta):
            q = dataclasses.replace(p)
            if which == "D0":
                q.D = (base + delta, p.D[1])
            elif which == "D1":
                q.D = (p.D[0], base + delta)
            else:
                q.k_surf = base + delta
            return loss_of(oracle.Problem(phi, q), u0)

        fd = (perturbed(h) - perturbed(-h)) / (2 * h)
        g = {"D0": grad[0], "D1": grad[1], "k": grad[2]}[which]
        assert abs(g - fd) <= 1e-6 * abs(fd), (which, g, fd)
    free = ((P.active > 0) & (P.fixed == 0))[None]
    direction = rng.standard_normal(u0.shape) * free
    h = 1e-3
    fd = (loss_of(P, u0 + h * direction) - loss_of(P, u0 - h * direction)) / (2 * h)
    assert abs(float((lam0 * direction).sum()) - fd) <= 1e-6 * abs(fd)


def test_adjoint_sink_gradient_at_zero_rate():
    """One species without a sink (k = 0): dL/dk is the first-order effect of
    switching a surface sink on, nonzero and equal to the central difference
    of the forward over k = +-h (k < 0 is a surface source; the update is
    affine in k, so the difference is exact up to rounding and the O(h^2)
    term)."""
    import dataclasses
    phi, p2 = adjoint_problem(7)
    p = dataclasses.replace(p2, nspecies=1, D=(1.0, 0.0), decay=(0.01, 0.0), k_surf=0.0)
    P = oracle.Problem(phi, p)
    rng = np.random.default_rng(4)
    nsteps = 25
    u0 = rng.uniform(0.2, 1.0, size=(1,) + phi.shape)
    weights = rng.uniform(0, 1, size=(1,) + phi.shape) * P.active[None]
    _, grad, _ = P.adjoint_run(u0, nsteps, weights)
    assert grad[1] < 0  # a sink lowers a positive-weighted sum of a positive field

    def loss(k):
        q = dataclasses.replace(p, k_surf=k)
        return float((oracle.Problem(phi, q).run(u0, nsteps) * weights).sum())

    h = 1e-4
    fd = (loss(h) - loss(-h)) / (2 * h)
    assert abs(grad[1] - fd) <= 1e-6 * abs(fd), (grad, fd)


# ---------------------------------------------------------------------------
# symmetry: the operator commutes with reflections and axis swaps
# ---------------------------------------------------------------------------
def test_reflection_and_axis_swap_symmetry():
    dims = (10, 8, 6)
    phi = random_blob_phi(dims, 44, porosity=0.6, ell=1.5)
    u0 = np.random.default_rng(2).uniform(0, 1, size=phi.shape)
    p = phys(dims, 0.1, D=(1.0, 0.0), dx=(1.0, 1.0, 1.0))
    base = oracle.Problem(phi, p).run(u0, 20)[0]
    flipped = oracle.Problem(np.ascontiguousarray(phi[:, :, ::-1]), p).run(u0[:, :, ::-1].copy(), 20)[0]
    np.testing.assert_allclose(flipped, base[:, :, ::-1], rtol=1e-13, atol=1e-15)
    pt = phys((8, 10, 6), 0.1, D=(1.0, 0.0))
    swapped = oracle.Problem(np.ascontiguousarray(phi.transpose(0, 2, 1)), pt).run(
        np.ascontiguousarray(u0.transpose(0, 2, 1)), 20)[0]
    np.testing.assert_allclose(swapped, base.transpose(0, 2, 1), rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------------------
# the paper's printed numbers
# ---------------------------------------------------------------------------
def test_stability_limit_reduces_to_eq_10():
    """In 2-D with one species and no reaction the limit is Eq. 10's
    1/(2 D (dx^-2 + dy^-2)), above the dt = h^2/8 of Sec. 3.1; the 3-D
    reactive form adds each species' loss rate."""
    g = GOLDEN["stability_2d"]
    h = 0.05
    p = phys((16, 16, 1), 0.0, D=(1.0, 0.0), dx=(h, h, 1.0))
    lim = oracle.Problem(open_box((16, 16, 1)), p).stability_limit()
    assert abs(lim - g["limit_over_h2_for_D1"] * h * h) < 1e-15
    assert g["paper_dt_over_h2"] * h * h < lim
    p3 = phys((8, 8, 8), 0.0, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.001), k_surf=0.05)
    lim3 = oracle.Problem(open_box((8, 8, 8)), p3).stability_limit()
    assert abs(lim3 - 1.0 / 6.05) < 1e-15


def test_manufactured_disk_converges_at_the_papers_order():
    """Sec. 3.1: diffusion in the unit disk with no flux on r = 1, manufactured
    source of appendix A.1, dt = h^2/8, t = 0.025; the paper reports an
    empirical order of about 1.5 (between the first-order boundary and the
    second-order interior)."""
    g = GOLDEN["mms_disk"]
    B, t_end = g["B"], g["t_final"]
    errs = []
    sizes = [32, 64, 128]
    for N in sizes:
        h = 4.0 / N
        c = -2.0 + (np.arange(N) + 0.5) * h
        X, Y = np.meshgrid(c, c, indexing="xy")
        r = np.sqrt(X ** 2 + Y ** 2)
        phi = (1.0 - r).astype(np.float32)[None]
        nsteps = int(math.ceil(t_end / (g["dt_over_h2"] * h * h)))
        dt = t_end / nsteps
        p = phys((N, N, 1), dt, D=(g["D"], 0.0), dx=(h, h, 1.0))
        P = oracle.Problem(phi, p)
        u = ((r ** 3 / 3 - r ** 4 / 4))[None]
        u = P.shape_state(u)
        for n in range(nsteps):
            t = n * dt
            f = (B / 4 * r ** 4 - B / 3 * r ** 3 + 4 * r ** 2 - 3 * r) * math.exp(-B * t)
            u = P.step(u, src=f[None])
        exact = (r ** 3 / 3 - r ** 4 / 4) * math.exp(-B * t_end)
        act = P.active[0] > 0
        e = u[0, 0][act] - exact[act]
        errs.append(math.sqrt(np.mean(e ** 2)))
    orders = [math.log(errs[i] / errs[i + 1]) / math.log(2.0) for i in range(len(errs) - 1)]
    lo, hi = g["order_band"]
    assert all(lo <= o <= hi for o in orders), (errs, orders)


def test_surface_weight_is_half_a_unit_delta():
    """The smoothed delta has unit integral across the interface; the pore side
    alone carries one half.  w(eps_b / 2) = 1 / (2 eps_b); w = 0 beyond eps_b."""
    h = 1e-3
    n = 4000
    x = (np.arange(n) + 0.5) * h
    phi = x.astype(np.float32).reshape(1, 1, n)
    P = oracle.Problem(phi, phys((n, 1, 1), 0.0))
    integral = P.w.sum() * h
    assert abs(integral - 0.5) < 1e-6
    phi2 = np.array([0.5, 1.0, 1.5, -0.2], dtype=np.float32).reshape(1, 1, 4)
    P2 = oracle.Problem(phi2, phys((4, 1, 1), 0.0))
    np.testing.assert_allclose(P2.w[0, 0], [0.5, 0.0, 0.0, 0.0], atol=1e-7)
    assert list(P2.active[0, 0]) == [1, 1, 1, 0]


# ---------------------------------------------------------------------------
# the monitoring reductions against their plain definitions
# ---------------------------------------------------------------------------
def test_reduction_terms_against_their_definitions():
    """Mass, active count, inlet/outlet x-fluxes and the residual of a
    two-species reactive state with held x faces, against numpy brute force
    over the active voxels; the residual against the step (pinned above on
    its own): L_h u = (u' - u) / dt on the free voxels."""
    dims = (11, 9, 8)
    phi = random_blob_phi(dims, 71, porosity=0.6, ell=1.5)
    d, v = dirich(0, 1, values=(1.0, 0.0))
    ph = phys(dims, 0.04, nspecies=2, D=(0.9, 0.4), decay=(0.02, 0.05), k_surf=0.7, dx=(0.8, 1.1, 1.3),
              dirichlet=d, face_value=v)
    P = oracle.Problem(phi, ph)
    u = P.shape_state(np.random.default_rng(71).uniform(0, 1, (2,) + phi.shape))
    red = P.reduce(u)
    act = P.active > 0
    free = act & (P.fixed == 0)
    step = P.step(u)
    dv = 0.8 * 1.1 * 1.3
    for s in range(2):
        r = red[s]
        assert r["n_active"] == int(act.sum())
        assert abs(r["mass"] - float(np.sum(u[s][act])) * dv) <= 1e-12 * r["mass"]
        lhs = (step[s] - u[s]) / 0.04
        res = math.sqrt(float(np.sum(lhs[free] ** 2)))
        assert abs(r["residual"] - res) <= 1e-9 * res
        for key, p0 in (("J_in", 0), ("J_out", dims[0] - 2)):
            both = act[:, :, p0] & act[:, :, p0 + 1]
            j = (0.9, 0.4)[s] * float(np.sum((u[s][:, :, p0] - u[s][:, :, p0 + 1])[both])) / 0.8 * (1.1 * 1.3)
            assert abs(r[key] - j) <= 1e-12 * max(1.0, abs(j)), (s, key, r[key], j)
