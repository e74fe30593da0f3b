"""Degenerate boxes against the oracle: a single voxel, lines and planes of
voxels (one or two axes of extent 1), a box thinner than a block in every
direction, and a pore space of isolated voxels (every neighbour mirrored), in
every state type and both block edges, with held faces and reactions where
they make sense; plus the F32R / batch paths on the same shapes."""
import numpy as np
import pytest

import oracle
from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402

SHAPES = [(1, 1, 1), (1, 1, 13), (1, 11, 1), (9, 1, 1), (1, 7, 9), (3, 3, 3), (2, 5, 6)]


def tol(dtype):
    # SBG_F32X2 keeps the state to ~48 bits, but each step's increment is formed in FP32
    # arithmetic (differences of the hi and of the lo parts), so its error grows by about an
    # FP32 ulp of the increment per step
    return {"f64": 1e-13, "f32": 2e-6, "f32x2": 1e-8, "f32r": 1e-6}[dtype]


@pytest.mark.parametrize("zyx", SHAPES)
@pytest.mark.parametrize("block", [4, 8])
@pytest.mark.parametrize("dtype", ["f64", "f32", "f32x2", "f32r"])
def test_thin_boxes_match_the_oracle(zyx, block, dtype):
    nz, ny, nx = zyx
    dims = (nx, ny, nz)
    phi = np.full(zyx, 3.0, np.float32)
    held = nx > 1
    ph = Physics(dims=dims, dt=0.1, D=(1.0, 0.0), decay=(0.02, 0.0), dx=(1.0, 0.8, 1.2),
                 dirichlet=(held, held, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    u0 = np.random.default_rng(sum(zyx)).uniform(0, 1, zyx)
    ref = oracle.Problem(phi, ph).run(u0[None], 90)[0]
    for variant in (["plain", "async"] if dtype != "f64" else ["plain"]):
        st = State(Grid(phi, block=block), 1, dtype).set_kernel(variant).set(u0)
        st.step(make_params(ph), 90)
        out = st.get()
        assert np.max(np.abs(out - ref)) <= tol(dtype) * max(1.0, np.max(np.abs(ref))), (variant, zyx)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f32r"])
def test_isolated_voxels_only_react(dtype):
    """A checkerboard pore space: no two pore voxels share a face, so every
    neighbour is mirrored and each voxel decays on its own, u (1 - dt decay)^n."""
    zyx = (6, 7, 9)
    z, y, x = np.indices(zyx)
    phi = np.where((x + y + z) % 2 == 0, 1.5, -1.0).astype(np.float32)
    ph = Physics(dims=zyx[::-1], dt=0.15, D=(1.0, 0.0), decay=(0.05, 0.0))
    u0 = np.random.default_rng(3).uniform(0.5, 1, zyx)
    st = State(Grid(phi, block=4), 1, dtype).set(u0)
    st.step(make_params(ph), 40)
    out = st.get()
    pore = phi > 0
    expected = u0 * (1.0 - 0.15 * 0.05) ** 40
    assert np.max(np.abs(out[pore] - expected[pore])) <= tol(dtype)
    assert np.all(out[~pore] == 0.0)


@pytest.mark.parametrize("dtype", ["f32", "f32r"])
def test_batch_with_empty_and_one_voxel_geometries(dtype):
    """A batch holding an empty geometry (no pore voxel), a one-voxel box and
    a line next to ordinary boxes steps every geometry as its own grid does,
    and the batched steady solve leaves the empty one alone."""
    rng = np.random.default_rng(81)
    geos = [random_blob_phi((14, 12, 10), 81, porosity=0.6, ell=1.6),
            np.full((6, 7, 8), -1.0, np.float32),
            np.full((1, 1, 1), 2.0, np.float32),
            np.full((1, 1, 19), 2.0, np.float32),
            random_blob_phi((9, 11, 13), 82, porosity=0.5, ell=1.5)]
    d = (True, True, False, False, False, False)
    p = make_params(Physics(dims=(8, 8, 8), dt=0.1, D=(1.0, 0.0), decay=(0.01, 0.0), dirichlet=d,
                            face_value=(1.0, 0.0, 0, 0, 0, 0)))
    gb = Grid.batch(geos, block=4)
    na, _, count = gb.geometry_info()
    assert na[1] == 0 and count[1] == 0 and na[2] == 1
    sb = State(gb, 1, dtype)
    u0s = [rng.uniform(0, 1, phi.shape) for phi in geos]
    for i, u in enumerate(u0s):
        sb.set(u, geom=i)
    sb.step(p, 90)
    for i, phi in enumerate(geos):
        st = State(Grid(phi, block=4), 1, dtype).set(u0s[i]).step(p, 90)
        np.testing.assert_array_equal(sb.get(0, geom=i, out=np.zeros(phi.shape)), st.get())
    # plain FP32 stalls near a 1e-5 relative residual (the reason SBG_F32R exists)
    tol = 1e-6 if dtype == "f32r" else 2e-4
    steps, rel = sb.batch_run_to_steady(p, tol, check_every=128, max_steps=200_000, raise_on_max=False)
    assert steps[1] == 0 and np.all(rel[[0, 2, 3, 4]] < tol), (steps, rel)


@pytest.mark.parametrize("zyx", [(1, 1, 17), (1, 9, 11), (3, 3, 3)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_adjoint_on_thin_boxes_matches_the_oracle(zyx, dtype, tol):
    from paper_2304_11165_b300.autograd import adjoint, forward_record
    nz, ny, nx = zyx
    phi = np.full(zyx, 0.6, np.float32)  # every voxel in the surface band: the reaction acts everywhere
    ph = Physics(dims=(nx, ny, nz), dt=0.05, nspecies=2, D=(1.0, 0.5), decay=(0.01, 0.1), k_surf=0.5,
                 dirichlet=(nx > 1, False, False, False, False, False), face_value=(0.0,) * 6)
    rng = np.random.default_rng(sum(zyx))
    u0 = rng.uniform(0.2, 1.0, (2,) + zyx)
    if nx > 1:
        u0[:, :, :, 0] = 0.0
    lamN = rng.uniform(0, 1, (2,) + zyx)
    P = oracle.Problem(phi, ph)
    lam0_ref, grad_ref, _ = P.adjoint_run(u0, 25, lamN * P.active[None])
    g = Grid(phi, block=4)
    st = State(g, 2, dtype).set_all(u0)
    tape = forward_record(st, make_params(ph), 25, 6)
    lam = State(g, 2, dtype).set_all(lamN * P.active[None])
    grad = adjoint(tape, lam)
    lam0 = lam.get_all()
    assert np.max(np.abs(lam0 - lam0_ref)) <= tol * np.max(np.abs(lam0_ref))
    for s in range(2):
        assert abs(grad[s] - grad_ref[s]) <= tol * max(abs(grad_ref[s]), 1e-12), (s, grad, grad_ref)
    assert abs(grad[2] - grad_ref[2]) <= tol * max(abs(grad_ref[2]), 1e-12)


@pytest.mark.parametrize("zyx", [(1, 1, 15), (1, 8, 10), (2, 5, 6), (1, 1, 1)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_inhomogeneous_thin_boxes_match_the_oracle(zyx, dtype, tol):
    nz, ny, nx = zyx
    phi = np.full(zyx, 3.0, np.float32)
    eps = np.random.default_rng(sum(zyx) + 1).uniform(0.2, 1.0, zyx)
    if dtype == "f32":
        eps = eps.astype(np.float32).astype(np.float64)
    ph = Physics(dims=(nx, ny, nz), dt=0.1, D=(1.0, 0.0), decay=(0.02, 0.0),
                 dirichlet=(nx > 1, False, False, False, False, False), face_value=(1.0, 0, 0, 0, 0, 0))
    u0 = np.random.default_rng(sum(zyx)).uniform(0, 1, zyx)
    ref = oracle.Problem(phi, ph, eps=eps).run(u0[None], 60)[0]
    for variant in (["plain", "async"] if dtype == "f32" else ["plain"]):
        g = Grid(phi, block=4).set_diffusivity(eps if dtype == "f64" else eps.astype(np.float32))
        st = State(g, 1, dtype).set_kernel(variant).set(u0)
        st.step(make_params(ph), 60)
        assert np.max(np.abs(st.get() - ref)) <= tol * max(1.0, np.max(np.abs(ref))), (variant, zyx)


@pytest.mark.parametrize("block", [4, 8])
def test_activity_threshold_is_strict(block):
    """phi equal to the FP32 epsilon is outside Omega, the next FP32 value is
    inside (the same test as the oracle's): the grid counts and the state
    reads back accordingly."""
    eps = np.float32(np.finfo(np.float32).eps)
    vals = np.array([-1.0, 0.0, eps, np.nextafter(eps, np.float32(1)), 0.5], dtype=np.float32)
    phi = vals.reshape(1, 1, 5)
    g = Grid(phi, block=block)
    P = oracle.Problem(phi, Physics(dims=(5, 1, 1), dt=0.1, D=(1.0, 0.0)))
    assert g.n_active == int(P.active.sum()) == 2
    out = State(g, 1, "f64").set(np.ones(phi.shape)).get()
    np.testing.assert_array_equal(out.ravel(), [0.0, 0.0, 0.0, 1.0, 1.0])
