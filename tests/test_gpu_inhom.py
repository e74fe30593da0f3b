"""Inhomogeneous diffusion on the GPU (per-voxel diffusivity factor, Eq. 6,
face means of the Listing 6 functor) against the FP64 oracle, element by
element, plus the consistency of the kernels and the argument checks."""
import numpy as np
import pytest

import oracle
from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, State, make_params  # noqa: E402
from paper_2304_11165_b300 import _abi  # noqa: E402


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def case(dims, seed, dirichlet=True, decay=0.02, dt=0.04):
    phi = random_blob_phi(dims, seed, porosity=0.6, ell=1.7)
    eps = np.random.default_rng(seed).uniform(0.1, 1.0, phi.shape)
    d = (True, False, False, False, False, False) if dirichlet else (False,) * 6
    ph = Physics(dims=dims, dt=dt, D=(0.9, 0.0), decay=(decay, 0.0), dx=(1.0, 0.9, 1.1), dirichlet=d,
                 face_value=(1.0, 0, 0, 0, 0, 0))
    u0 = np.random.default_rng(seed + 1).uniform(0, 1, phi.shape)
    return phi, eps, ph, u0


@pytest.mark.parametrize("block", [4, 8])
def test_fp64_matches_the_oracle(block):
    phi, eps, ph, u0 = case((23, 19, 17), 11)
    ref = oracle.Problem(phi, ph, eps=eps).run(u0[None], 60)[0]
    g = Grid(phi, block=block).set_diffusivity(eps)
    st = State(g, 1, "f64").set(u0)
    st.step(make_params(ph), 60)
    assert rel_err(st.get(), ref) < 1e-13


@pytest.mark.parametrize("block", [4, 8])
def test_fp32_kernels_match_the_oracle_and_each_other(block):
    phi, eps, ph, u0 = case((37, 29, 23), 12)
    ref = oracle.Problem(phi, ph, eps=eps).run(u0[None], 150)[0]
    outs = []
    for variant in ("plain", "pipelined", "prefetch", "async", "stream"):
        g = Grid(phi, block=block).set_diffusivity(eps.astype(np.float32))
        st = State(g, 1, "f32").set_kernel(variant).set(u0)
        st.step(make_params(ph), 150)
        outs.append(st.get())
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)
    # eps is rounded to FP32 on both sides here (the oracle gets the same rounded values)
    ref32 = oracle.Problem(phi, ph, eps=eps.astype(np.float32).astype(np.float64)).run(u0[None], 150)[0]
    assert rel_err(outs[0], ref32) < 1e-5
    assert rel_err(outs[0], ref) < 2e-5


@pytest.mark.parametrize("block", [4, 8])
def test_two_row_kernel_with_few_ctas(block):
    """u and the factor on the two-row kernel (cp.async halos) with one and two
    persistent CTAs per SM: many groups per CTA, the same field as the
    one-thread-per-voxel kernel."""
    phi, eps, ph, u0 = case((64, 60, 56), 14)
    g = Grid(phi, block=block).set_diffusivity(eps.astype(np.float32))
    p = make_params(ph)
    a = State(g, 1, "f32").set_kernel("plain").set(u0).step(p, 33).get()
    for per_sm in (1, 2, 0):
        b = State(g, 1, "f32").set_kernel("async", ctas_per_sm=per_sm).set(u0).step(p, 33).get()
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("order", ["tiled", "planes"])
@pytest.mark.parametrize("per_sm", [1, 0])
def test_streaming_kernel_with_a_factor(order, per_sm):
    """u and the factor read by the streaming kernel (rows through L1, absent
    neighbour blocks from the ghost blocks: sentinels for u, zeros for the
    factor), with one or all CTAs per SM: the plain kernel's field bitwise."""
    phi, eps, ph, u0 = case((64, 60, 56), 15)
    g = Grid(phi, block=4, order=order).set_diffusivity(eps.astype(np.float32))
    p = make_params(ph)
    a = State(g, 1, "f32").set_kernel("plain").set(u0).step(p, 33).get()
    b = State(g, 1, "f32").set_kernel("stream", ctas_per_sm=per_sm).set(u0).step(p, 33).get()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims", [(1, 1, 1), (6, 1, 1), (1, 1, 9), (4, 4, 4), (17, 3, 2)])
def test_streaming_kernel_with_a_factor_on_thin_boxes(dims):
    rng = np.random.default_rng(sum(dims))
    phi = np.where(rng.uniform(size=dims[::-1]) < 0.8, 1.0, -1.0).astype(np.float32)
    phi.flat[0] = 1.0
    eps = rng.uniform(0.2, 1.0, phi.shape).astype(np.float32)
    ph = Physics(dims=dims, dt=0.02, D=(1.0, 0.0), decay=(0.01, 0.0))
    u0 = rng.uniform(size=phi.shape)
    g = Grid(phi, block=4).set_diffusivity(eps)
    p = make_params(ph)
    a = State(g, 1, "f32").set_kernel("plain").set(u0).step(p, 13).get()
    b = State(g, 1, "f32").set_kernel("stream").set(u0).step(p, 13).get()
    np.testing.assert_array_equal(a, b)
    ref = oracle.Problem(phi, ph, eps=eps.astype(np.float64)).run(u0[None], 13)[0]
    assert rel_err(b, ref) < 1e-5


def test_eq6_factor_on_the_device_matches_the_oracle():
    phi, _, ph, u0 = case((21, 18, 15), 13)
    args = (0.05, 0.95, -0.8, 2.5)
    eps = oracle.eps_sigmoid(phi, *args)
    ref = oracle.Problem(phi, ph, eps=eps).run(u0[None], 50)[0]
    g = Grid(phi, block=8).set_diffusivity_sigmoid(phi, *args)
    st = State(g, 1, "f64").set(u0)
    st.step(make_params(ph), 50)
    assert rel_err(st.get(), ref) < 1e-13


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_reductions_match_the_oracle(dtype, tol):
    phi, eps, ph, u0 = case((26, 21, 19), 14, dirichlet=False)
    ph = Physics(dims=ph.dims, dt=ph.dt, D=ph.D, decay=ph.decay, dx=ph.dx,
                 dirichlet=(True, True, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    epsd = eps if dtype == "f64" else eps.astype(np.float32).astype(np.float64)
    P = oracle.Problem(phi, ph, eps=epsd)
    g = Grid(phi, block=4).set_diffusivity(eps if dtype == "f64" else eps.astype(np.float32))
    st = State(g, 1, dtype).set(u0)
    p = make_params(ph)
    st.step(p, 30)
    field = st.get()
    red = st.reduce(p)[0]
    ref = P.reduce(field[None])[0]  # the oracle's reductions of the GPU's field
    for key in ("mass", "J_in", "J_out", "residual"):
        scale = max(abs(ref[key]), 1.0)
        assert abs(red[key] - ref[key]) <= tol * scale, (key, red[key], ref[key])
    assert red["n_active"] == ref["n_active"]


def test_closed_box_mass_is_conserved_in_fp64():
    phi, eps, ph, u0 = case((24, 20, 18), 15, dirichlet=False, decay=0.0, dt=0.1)
    g = Grid(phi, block=4).set_diffusivity(eps)
    st = State(g, 1, "f64").set(u0)
    p = make_params(ph)
    m0 = st.reduce(p)[0]["mass"]
    st.step(p, 400)
    assert abs(st.reduce(p)[0]["mass"] - m0) <= 1e-12 * m0


def test_layered_channel_effective_diffusivity():
    """Steady state of a full channel with a factor varying along x: D_eff is
    the harmonic mean of the face diffusivities (closed form)."""
    nx, ny, nz = 20, 4, 4
    phi = np.full((nz, ny, nx), 5.0, np.float32)
    ex = np.random.default_rng(16).uniform(0.3, 1.0, nx)
    eps = np.broadcast_to(ex[None, None, :], phi.shape).copy()
    ph = Physics(dims=(nx, ny, nz), dt=0.15, D=(1.0, 0.0), dirichlet=(True, True, False, False, False, False),
                 face_value=(1.0, 0.0, 0, 0, 0, 0))
    g = Grid(phi, block=4).set_diffusivity(eps)
    u0 = np.zeros(phi.shape)
    u0[:, :, 0] = 1.0
    st = State(g, 1, "f64").set(u0)
    p = make_params(ph)
    st.run_to_steady(p, 1e-13, check_every=1000, max_steps=400_000)
    d_eff, _, _ = st.effective_D(p)
    ef = 0.5 * (ex[:-1] + ex[1:])
    assert abs(d_eff - (nx - 1) / np.sum(1.0 / ef)) <= 1e-10


def test_argument_checks_and_clearing():
    phi, eps, ph, u0 = case((16, 14, 12), 17)
    p = make_params(ph)
    g = Grid(phi, block=4).set_diffusivity(eps)
    with pytest.raises(SbgError) as e:
        State(g, 1, "f32x2").set(u0).step(p, 1)
    assert e.value.status == _abi.SBG_ERR_INVALID_ARG
    ph2 = Physics(dims=ph.dims, dt=ph.dt, nspecies=2, D=(0.9, 0.5), dx=ph.dx)
    with pytest.raises(SbgError):
        State(g, 2, "f32").set_all(np.stack([u0, u0])).step(make_params(ph2), 1)
    # the stability limit follows D_0 * max(eps)
    g2 = Grid(phi, block=4).set_diffusivity(np.full(phi.shape, 3.0))
    with pytest.raises(SbgError) as e:
        State(g2, 1, "f32").set(u0).step(make_params(Physics(dims=ph.dims, dt=0.1, D=(1.0, 0.0))), 1)
    assert e.value.status == _abi.SBG_ERR_UNSTABLE_DT
    with pytest.raises(SbgError):
        Grid(phi, block=4).set_diffusivity(-np.ones(phi.shape))
    # clearing restores the constant-D step bitwise
    g.clear_diffusivity()
    a = State(g, 1, "f32").set(u0).step(p, 20).get()
    b = State(Grid(phi, block=4), 1, "f32").set(u0).step(p, 20).get()
    np.testing.assert_array_equal(a, b)
