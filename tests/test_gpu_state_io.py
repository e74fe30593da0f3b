"""Dense <-> block-layout transfers: setting a state from FP32 input (the
row kernel, with and without 16-byte dense loads) gives the same state as
setting it from the same values in FP64 (the per-slot kernel), for every
state type and ragged boxes; inactive voxels read back as 0 and NaN input
stays NaN."""
import numpy as np
import pytest

from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402


@pytest.mark.parametrize("dims", [(24, 19, 13), (23, 18, 11)])
@pytest.mark.parametrize("block", [4, 8])
@pytest.mark.parametrize("dtype", ["f32", "f32x2", "f32r"])
def test_fp32_input_equals_fp64_input(dims, block, dtype):
    phi = random_blob_phi(dims, 61, porosity=0.55, ell=1.6)
    rng = np.random.default_rng(61)
    u32 = rng.uniform(-1, 1, phi.shape).astype(np.float32)
    act = phi > np.finfo(np.float32).eps
    idx = np.argwhere(act)
    u32[tuple(idx[3])] = np.nan
    u32[tuple(idx[5])] = np.inf
    g = Grid(phi, block=block)
    a = State(g, 1, dtype).set(u32)                      # FP32 input: row kernel
    b = State(g, 1, dtype).set(u32.astype(np.float64))   # FP64 input: per-slot kernel
    ga, gb = a.get(), b.get()
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(ga[~act], 0.0)
    assert np.isnan(ga[tuple(idx[3])]) and np.isinf(ga[tuple(idx[5])])
    ok = act & np.isfinite(u32)
    np.testing.assert_array_equal(ga[ok], u32[ok].astype(np.float64))


def test_unaligned_device_input_and_steps_agree():
    dims = (32, 20, 17)
    phi = random_blob_phi(dims, 62, porosity=0.6, ell=1.7)
    rng = np.random.default_rng(62)
    u = rng.uniform(0, 1, phi.shape).astype(np.float32)
    ph = Physics(dims=dims, dt=0.05, D=(1.0, 0.0), dirichlet=(True, True, False, False, False, False),
                 face_value=(1.0, 0.0, 0, 0, 0, 0))
    p = make_params(ph)
    g = Grid(phi, block=4)
    flat = torch.zeros(u.size + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(u.ravel()).cuda()
    view = flat[1:].view(u.shape)  # 4-byte offset: no 16-byte loads
    for dtype in ("f32", "f32r"):
        a = State(g, 1, dtype).set(view).step(p, 40).get()
        b = State(g, 1, dtype).set(u.astype(np.float64)).step(p, 40).get()
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dtype,ns", [("f32", 2), ("f64", 1), ("f32r", 1), ("f32x2", 1)])
def test_async_reduction_equals_the_synchronous_one(dtype, ns):
    dims = (26, 22, 18)
    phi = random_blob_phi(dims, 63, porosity=0.6, ell=1.7)
    rng = np.random.default_rng(63)
    u0 = rng.uniform(0, 1, (ns,) + phi.shape)
    ph = Physics(dims=dims, dt=0.05, nspecies=ns, D=(1.0, 0.5)[:ns] + (0.0,) * (2 - ns),
                 decay=(0.01, 0.02), k_surf=0.2 if ns == 2 else 0.0,
                 dirichlet=(True, True, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    p = make_params(ph)
    g = Grid(phi, block=4)
    a = State(g, ns, dtype).set_all(u0 if ns == 2 else u0[0]).step(p, 70)
    b = State(g, ns, dtype).set_all(u0 if ns == 2 else u0[0]).step(p, 70)
    ref = a.reduce(p)
    host = torch.zeros(ns * 8, dtype=torch.float64).pin_memory()
    dev = torch.zeros(ns * 8, dtype=torch.float64, device="cuda")
    b.reduce_async(p, host)
    torch.cuda.synchronize()
    assert b.parse_reduction(host) == ref
    c = State(g, ns, dtype).set_all(u0 if ns == 2 else u0[0]).step(p, 70)
    c.reduce_async(p, dev)
    assert c.parse_reduction(dev.cpu()) == ref
    # the states go on identically after either call (SBG_F32R: the same refresh)
    np.testing.assert_array_equal(a.step(p, 30).get_all(), b.step(p, 30).get_all())


@pytest.mark.parametrize("dtype,ns,block", [("f32", 2, 4), ("f32", 2, 8), ("f32", 1, 4), ("f64", 2, 4),
                                            ("f32r", 1, 4), ("f32x2", 1, 8)])
def test_check_is_the_reduction_without_the_residual(dtype, ns, block):
    """sbg_check_async: every scalar bitwise that of the full reduction of the
    same state, the residual NaN, the state untouched."""
    dims = (29, 21, 17)
    phi = random_blob_phi(dims, 64, porosity=0.6, ell=1.7)
    rng = np.random.default_rng(64)
    u0 = rng.uniform(0, 1, (ns,) + phi.shape)
    ph = Physics(dims=dims, dt=0.05, nspecies=ns, D=(1.0, 0.5)[:ns] + (0.0,) * (2 - ns),
                 decay=(0.01, 0.02), k_surf=0.2,
                 dirichlet=(True, True, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    p = make_params(ph)
    g = Grid(phi, block=block)
    a = State(g, ns, dtype).set_all(u0 if ns == 2 else u0[0]).step(p, 50)
    before = a.get_all()
    dev = torch.full((ns * 8,), 7.0, dtype=torch.float64, device="cuda")
    a.check_async(p, dev)
    chk = a.parse_reduction(dev.cpu())
    host = torch.zeros(ns * 8, dtype=torch.float64).pin_memory()
    a.check_async(p, host)
    torch.cuda.synchronize()
    chk_host = a.parse_reduction(host)
    np.testing.assert_array_equal(a.get_all(), before)
    # (SBG_F32R: the full reduction then folds the correction into the base, so it comes last)
    ref = a.reduce(p)
    keys = ("mass", "J_in", "J_out", "min", "max", "nonfinite", "n_active")
    for s in range(ns):
        assert np.isnan(chk[s]["residual"]) and np.isnan(chk_host[s]["residual"])
        assert np.isfinite(ref[s]["residual"])
        for key in keys:
            assert chk[s][key] == ref[s][key], (s, key, chk[s][key], ref[s][key])
            assert chk_host[s][key] == chk[s][key]
