"""The slab decomposition on the GPU, with the ranks emulated in one process
(one grid and state per slab, the ghost planes exchanged between them after
every step through sbg_state_get_xplane / sbg_state_set_xplane): the owned
planes of all slabs equal the whole-box run bit for bit, in FP64 and in FP32
(the streaming kernel), and the owned box sums add up to the whole mass.
The ranks' kernels never wait on one another (the exchange runs on the host
between steps)."""
import numpy as np
import pytest

from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, State, _abi, make_params  # noqa: E402
from paper_2304_11165_b300 import slab as sl  # noqa: E402


def problem(dims=(53, 31, 27), seed=71):
    phi = random_blob_phi(dims, seed, porosity=0.6, ell=1.7)
    phys = Physics(dims=dims, dt=0.05, nspecies=2, D=(1.0, 0.5), decay=(0.01, 0.1), k_surf=0.4,
                   dirichlet=(True, True, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    u0 = np.random.default_rng(seed).uniform(0, 1, size=(2,) + phi.shape)
    u0[0, :, :, 0] = 1.0
    u0[0, :, :, -1] = 0.0
    return phi, phys, u0


@pytest.mark.parametrize("dtype,nslabs", [("f64", 3), ("f32", 3), ("f32", 2)])
def test_slabs_reproduce_the_whole_box_bit_for_bit(dtype, nslabs):
    phi, phys, u0 = problem()
    nsteps = 40
    whole = State(Grid(phi, block=4, order="planes"), 2, dtype).set_all(u0)
    whole.step(make_params(phys), nsteps)
    ref = whole.get_all()
    bounds = sl.partition(phi, nslabs, block=4)
    slabs = [sl.Slab.of(bounds, r) for r in range(nslabs)]
    engines = [sl.LibraryEngine(s, phi, phys, u0, dtype=dtype) for s in slabs]
    for _ in range(nsteps):
        for e in engines:
            e.step(1)
        sl.exchange_ghosts_local(slabs, engines, 2)
    joined = np.concatenate([e.owned() for e in engines], axis=-1)
    np.testing.assert_array_equal(joined, ref)
    red = whole.reduce(make_params(phys))
    for s in range(2):
        parts = [e.owned_sum(s, sb.first_owned, sb.last_owned + 1) for sb, e in zip(slabs, engines)]
        assert sum(c for _, c in parts) == red[s]["n_active"]
        assert abs(sum(m for m, _ in parts) - red[s]["mass"]) <= 1e-12 * abs(red[s]["mass"])


def test_xplane_get_and_set_round_trip_and_argument_checks():
    phi, phys, u0 = problem((20, 14, 11), 72)
    g = Grid(phi, block=8)
    st = State(g, 2, "f64").set_all(u0)
    act = phi > np.finfo(np.float32).eps
    eng = sl.LibraryEngine(sl.Slab(0, 1, 0, 20, 20), phi, phys, u0, dtype="f64", block=8)
    for x in (0, 7, 8, 19):
        p = eng.get_plane(1, x).cpu().numpy()
        np.testing.assert_array_equal(p, np.where(act[:, :, x], u0[1][:, :, x], 0.0))
        eng.set_plane(1, x, torch.full_like(eng.get_plane(1, x), 0.25))
    got = eng.state.get(1)
    for x in (0, 7, 8, 19):
        np.testing.assert_array_equal(got[:, :, x], np.where(act[:, :, x], 0.25, 0.0))
    lib = _abi.load()
    buf = torch.zeros((11, 14), dtype=torch.float64, device="cuda")
    import ctypes
    for bad in ((0, 20), (2, 0), (0, -1)):
        sp, x = bad
        rc = lib.sbg_state_get_xplane(g.handle, st.handle, 0, sp, x, ctypes.c_void_p(buf.data_ptr()), _abi.SBG_F64, 1,
                                      None)
        assert rc == _abi.SBG_ERR_INVALID_ARG
    rc = lib.sbg_state_get_xplane(g.handle, st.handle, 0, 0, 3, ctypes.c_void_p(buf.data_ptr()), _abi.SBG_F32, 1, None)
    assert rc == _abi.SBG_ERR_INVALID_ARG  # the plane's dtype must be the state's
    with pytest.raises(SbgError):
        sl.partition(phi, 0)
