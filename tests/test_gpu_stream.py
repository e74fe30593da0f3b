"""The streaming step kernel (SBG_KERNEL_STREAM: groups of 16 blocks, 12 for
two species, taken by the CTAs in turn, one x-row per thread, neighbour rows
read through L1, an L2 prefetch of the next group's rows) against the one-thread-per-voxel kernel,
bitwise, and against the FP64 oracle; on grids in tiled and in plane order,
with ragged box edges, Dirichlet faces, the surface transfer of two species,
few CTAs walking many groups, and the degenerate geometries."""
import numpy as np
import pytest

import oracle
from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402


def case(dims, ns, k, faces, seed, porosity=0.55):
    phi = random_blob_phi(dims, seed, porosity=porosity, ell=1.7)
    phi = np.where(phi > 0, phi * 0.7, phi).astype(np.float32)
    d = [False] * 6
    v = [0.0] * 6
    for f in faces:
        d[f] = True
        v[f] = 1.0
    phys = Physics(dims=dims, dt=0.05, nspecies=ns, D=(1.0, 0.45), decay=(0.01, 0.2), k_surf=k,
                   dx=(1.0, 0.9, 1.1), dirichlet=tuple(d), face_value=tuple(v))
    u0 = np.random.default_rng(seed).uniform(0, 1, size=(ns,) + phi.shape)
    return phi, phys, u0


def run(phi, phys, u0, nsteps, variant, order="tiled", block=4, dtype="f32", ctas_per_sm=0):
    g = Grid(phi, block=block, order=order)
    st = State(g, phys.nspecies, dtype).set_kernel(variant, ctas_per_sm).set_all(u0)
    st.step(make_params(phys), nsteps)
    return st.get_all()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("order", ["tiled", "planes"])
@pytest.mark.parametrize("ns,k,faces", [(1, 0.0, (0, 1)), (1, 0.4, ()), (2, 0.6, (0, 1)), (2, 0.0, (3, 4)),
                                        (2, 0.6, ())])
def test_stream_kernel_is_bitwise_the_plain_kernel(order, ns, k, faces):
    phi, phys, u0 = case((37, 29, 23), ns, k, faces, 21)
    a = run(phi, phys, u0, 77, "plain", order)
    b = run(phi, phys, u0, 77, "stream", order)
    np.testing.assert_array_equal(a, b)
    ref = oracle.Problem(phi, phys).run(u0, 77)
    assert rel_err(b, ref) < 1e-5


def test_block_order_does_not_change_the_fields():
    """Plane order and tiled order list the same blocks differently; every
    voxel's update is the same expression, so the fields are bitwise equal."""
    phi, phys, u0 = case((45, 38, 41), 2, 0.6, (0,), 22)
    a = run(phi, phys, u0, 50, "stream", "tiled")
    b = run(phi, phys, u0, 50, "stream", "planes")
    c = run(phi, phys, u0, 50, "async", "planes")
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("per_sm", [1, 2, 0])
def test_stream_kernel_with_few_ctas_walks_many_groups(per_sm):
    """One or two CTAs per SM over a grid of many groups: each CTA takes
    dozens of groups in turn and its L2 prefetches run past the end of the
    list; the fields stay the plain kernel's."""
    phi, phys, u0 = case((96, 90, 84), 2, 0.6, (0, 1), 23)
    a = run(phi, phys, u0, 21, "plain", "planes")
    b = run(phi, phys, u0, 21, "stream", "planes", ctas_per_sm=per_sm)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 1, 1), (1, 6, 1), (1, 1, 7), (4, 4, 4), (3, 5, 9), (17, 2, 3)])
def test_stream_kernel_on_degenerate_boxes(dims):
    """Single voxels, lines, one block, thin boxes (every neighbour block
    absent: the ghost block)."""
    rng = np.random.default_rng(sum(dims))
    phi = np.where(rng.uniform(size=dims[::-1]) < 0.8, 1.0, -1.0).astype(np.float32)
    phi.flat[0] = 1.0
    phys = Physics(dims=dims, dt=0.02, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.1), k_surf=0.3)
    u0 = rng.uniform(size=(2,) + phi.shape)
    for order in ("tiled", "planes"):
        a = run(phi, phys, u0, 13, "plain", order)
        b = run(phi, phys, u0, 13, "stream", order)
        np.testing.assert_array_equal(a, b)
    ref = oracle.Problem(phi, phys).run(u0, 13)
    assert rel_err(b, ref) < 1e-5


def test_stream_variant_falls_back_where_it_does_not_apply():
    """FP64, compensated and 8^3-block states asked for the streaming kernel
    run the automatic choice (the same fields)."""
    phi, phys, u0 = case((21, 19, 17), 1, 0.3, (0,), 24)
    for dtype, block in (("f64", 4), ("f32x2", 4), ("f32", 8)):
        a = run(phi, phys, u0, 30, "auto", block=block, dtype=dtype)
        b = run(phi, phys, u0, 30, "stream", block=block, dtype=dtype)
        np.testing.assert_array_equal(a, b)


def test_empty_geometry_and_all_solid_state():
    phi = np.full((12, 10, 9), -1.0, np.float32)
    phys = Physics(dims=(9, 10, 12), dt=0.05, nspecies=2, D=(1.0, 0.5), k_surf=0.1)
    g = Grid(phi, block=4, order="planes")
    st = State(g, 2, "f32").set_kernel("stream").set_all(np.zeros((2,) + phi.shape))
    st.step(make_params(phys), 5)
    assert np.all(st.get_all() == 0)


def test_kernels_can_be_mixed_on_a_copied_state():
    """A state filled by a copy (its other buffer never written), stepped by
    the streaming kernel, then by the plain kernel (which reads every slot
    the streaming kernel wrote), then by the streaming kernel again, gives
    the plain kernel's fields bitwise, and its check counts no non-finite
    voxel."""
    phi, phys, u0 = case((45, 38, 41), 2, 0.6, (0,), 26, porosity=0.35)
    p = make_params(phys)
    g = Grid(phi, block=4, order="planes")
    ref = State(g, 2, "f32").set_kernel("plain").set_all(u0).step(p, 19).get_all()
    src = State(g, 2, "f32").set_all(u0)
    st = State(g, 2, "f32").copy_from(src)
    st.set_kernel("stream").step(p, 7)
    st.set_kernel("plain").step(p, 5)
    st.set_kernel("stream").step(p, 7)
    np.testing.assert_array_equal(st.get_all(), ref)
    r = st.reduce(p)
    assert r[0]["nonfinite"] == 0 and r[1]["nonfinite"] == 0


@pytest.mark.parametrize("order", ["tiled", "planes"])
@pytest.mark.parametrize("k", [0.0, 0.4])
def test_stream_kernel_runs_the_f32r_correction_bitwise(order, k):
    """SBG_F32R states (FP32 correction d on a compensated base, source
    r = L_h b refreshed every 256 steps): the streaming kernel reads d with its
    neighbour rows and r for the row itself, bitwise the plain kernel, over
    several refresh intervals with held faces; with a surface reaction the
    state falls back to the automatic choice (the same fields)."""
    phi, phys, u0 = case((37, 29, 23), 1, k, (0, 1), 27)
    a = run(phi, phys, u0, 600, "plain", order, dtype="f32r")
    b = run(phi, phys, u0, 600, "stream", order, dtype="f32r")
    np.testing.assert_array_equal(a, b)
    ref = oracle.Problem(phi, phys).run(u0, 600)
    # the correction carries up to 256 steps of change in FP32 (2.4e-7 of the maximum on this
    # random field, the plain kernel's error as well); the stated FP32 field bar is 1e-5
    assert rel_err(b, ref) < 1e-6

