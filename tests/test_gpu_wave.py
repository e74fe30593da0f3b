"""The wavefront step kernel (SBG_KERNEL_WAVE: 2 steps per launch,
SBG_KERNEL_WAVE4: 4) against the streaming kernel, bitwise, and against the
FP64 oracle: plane-ordered grids with ragged box edges, Dirichlet faces, one
and two species with the surface transfer, step counts that leave a
remainder and that use the cached graph, few CTAs taking many tickets (so
that tickets wait on one another), degenerate boxes, fallback where the
kernel does not apply, and a bounded wait made to run out."""
import numpy as np
import pytest

import oracle
from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, State, _abi, make_params  # noqa: E402


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


def run(phi, phys, u0, nsteps, variant, order="planes", ctas_per_sm=0, chunks=None):
    g = Grid(phi, block=4, order=order)
    st = State(g, phys.nspecies, "f32").set_kernel(variant, ctas_per_sm).set_all(u0)
    p = make_params(phys)
    for n in (chunks or [nsteps]):
        st.step(p, n)
    return st.get_all()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("variant", ["wave", "wave4"])
@pytest.mark.parametrize("ns,k,faces", [(1, 0.0, (0, 1)), (1, 0.4, ()), (2, 0.6, (0, 1)), (2, 0.0, (3, 4)),
                                        (2, 0.6, ())])
def test_wave_kernel_is_bitwise_the_streaming_kernel(variant, ns, k, faces):
    phi, phys, u0 = case((37, 29, 43), ns, k, faces, 21)
    a = run(phi, phys, u0, 77, "stream")
    b = run(phi, phys, u0, 77, variant)
    np.testing.assert_array_equal(a, b)
    ref = oracle.Problem(phi, phys).run(u0, 77)
    assert rel_err(b, ref) < 1e-5


@pytest.mark.parametrize("variant", ["wave", "wave4"])
def test_graph_replays_and_remainders(variant):
    """130 steps: two graph replays of 64 steps plus a remainder of 2, then
    chunks of 1, 3 and 5 steps (the odd ones end with a streaming step)."""
    phi, phys, u0 = case((40, 33, 52), 2, 0.6, (0,), 22)
    a = run(phi, phys, u0, 139, "stream", chunks=[130, 1, 3, 5])
    b = run(phi, phys, u0, 139, variant, chunks=[130, 1, 3, 5])
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("per_sm", [1, 2])
@pytest.mark.parametrize("variant", ["wave", "wave4"])
def test_few_ctas_take_many_tickets(per_sm, variant):
    """One or two CTAs per SM over a grid of thousands of tickets: tickets wait on
    one another often, and the counters are cleared and reused across launches."""
    phi, phys, u0 = case((96, 90, 84), 2, 0.6, (0, 1), 23)
    a = run(phi, phys, u0, 22, "stream")
    b = run(phi, phys, u0, 22, variant, ctas_per_sm=per_sm)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 1, 1), (1, 6, 1), (1, 1, 7), (4, 4, 4), (3, 5, 9), (17, 2, 3),
                                  (9, 8, 30)])
def test_wave_kernel_on_degenerate_boxes(dims):
    """Single voxels, lines, one plane, one block, thin boxes, planes without
    active blocks."""
    rng = np.random.default_rng(sum(dims))
    phi = np.where(rng.uniform(size=dims[::-1]) < 0.8, 1.0, -1.0).astype(np.float32)
    if dims[2] >= 30:
        phi[8:16] = -1.0  # two planes of blocks with no active block
    phi.flat[0] = 1.0
    phys = Physics(dims=dims, dt=0.02, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.1), k_surf=0.3)
    u0 = rng.uniform(size=(2,) + phi.shape)
    a = run(phi, phys, u0, 13, "stream")
    for v in ("wave", "wave4"):
        b = run(phi, phys, u0, 13, v)
        np.testing.assert_array_equal(a, b)
    ref = oracle.Problem(phi, phys).run(u0, 13)
    assert rel_err(b, ref) < 1e-5


def test_wave_variant_falls_back_where_it_does_not_apply():
    """A tiled-order grid, FP64 and SBG_F32R states asked for the wavefront
    kernel run the automatic choice (the same fields)."""
    phi, phys, u0 = case((21, 19, 17), 1, 0.3, (0,), 24)
    a = run(phi, phys, u0, 30, "auto", order="tiled")
    b = run(phi, phys, u0, 30, "wave", order="tiled")
    np.testing.assert_array_equal(a, b)
    for dtype in ("f64", "f32r"):
        g = Grid(phi, block=4, order="planes")
        x = State(g, 1, dtype).set_kernel("auto").set_all(u0).step(make_params(phys), 30).get_all()
        y = State(g, 1, dtype).set_kernel("wave").set_all(u0).step(make_params(phys), 30).get_all()
        np.testing.assert_array_equal(x, y)


def test_a_wave_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    """The stall hook keeps one ticket from publishing its completion: the
    tickets that wait on it give up after the short bound, SBG_ERR_TIMEOUT is
    reported by the next synchronising call, and the next launches (their
    counters cleared by the aborted launch's last CTA) give the right fields."""
    lib = _abi.load()
    phi, phys, u0 = case((48, 40, 64), 2, 0.6, (0,), 25)
    p = make_params(phys)
    g = Grid(phi, block=4, order="planes")
    st = State(g, 2, "f32").set_kernel("wave").set_all(u0)
    _abi.check(lib.sbg_debug_stall_stage(g.handle, 3, 1 << 20))
    try:
        st.step(p, 2)
        with pytest.raises(SbgError) as e:
            st.reduce(p)
        assert e.value.status == _abi.SBG_ERR_TIMEOUT
    finally:
        _abi.check(lib.sbg_debug_stall_stage(g.handle, -1, 0))
    ref = State(g, 2, "f32").set_kernel("stream").set_all(u0).step(p, 10).get_all()
    st.set_all(u0).step(p, 10)
    st.reduce(p)
    np.testing.assert_array_equal(st.get_all(), ref)
    assert torch.zeros(4, device="cuda").sum().item() == 0.0
