"""The allocation-free reduction entry point.

sbg_reduce_noalloc serves callers that may not allocate device memory (their
memory is owned by another allocator, or allocation latency is not allowed in
their loop).  It must give what sbg_reduce gives, call after call, although
every call reuses the same fixed scratch array inside the library.  This file
is collected last so that a run that stops at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402
from paper_2304_11165_b300 import _abi  # noqa: E402

REL = 1e-12  # FP64 sums in a different order


def noalloc(state, params, geom, species):
    """One call through the C ABI; returns the SBG_NRED results as numpy."""
    lib = _abi.load()
    out = torch.full((_abi.NRED,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.sbg_reduce_noalloc(state.grid.handle, state.handle, ctypes.byref(params), geom, species,
                                ctypes.c_void_p(out.data_ptr()), stream)
    _abi.check(rc)
    torch.cuda.current_stream().synchronize()
    return out.cpu().numpy()


def reference(state, params, geom):
    out = np.zeros(state.nspecies * _abi.NRED)
    _abi.check(_abi.load().sbg_reduce(state.grid.handle, state.handle, ctypes.byref(params), geom,
                                      out.ctypes.data_as(ctypes.c_void_p), 0))
    return out.reshape(state.nspecies, _abi.NRED)


def assert_same(a, b):
    for q in range(_abi.NRED):
        if q in (_abi.RED_MIN, _abi.RED_MAX, _abi.RED_NONFINITE, _abi.RED_NACTIVE):
            assert a[q] == b[q], (q, a[q], b[q])
        else:
            assert abs(a[q] - b[q]) <= REL * max(abs(b[q]), 1e-300), (q, a[q], b[q])


@pytest.mark.parametrize("dtype,block", [("f32", 8), ("f64", 4), ("f32x2", 8)])
def test_noalloc_reduction_equals_sbg_reduce_on_consecutive_calls(dtype, block):
    dims = (37, 30, 26)
    phi = random_blob_phi(dims, 21, porosity=0.55, ell=1.7)
    phi = np.where(phi > 0, phi * 0.7, phi).astype(np.float32)
    ns = 1 if dtype == "f32x2" else 2
    d = (True, True, False, False, False, False)
    phys = Physics(dims=dims, dt=0.05, nspecies=ns, D=(1.0, 0.5), decay=(0.01, 0.1), k_surf=0.4,
                   dirichlet=d, face_value=(1.0, 0.0, 0, 0, 0, 0))
    u0 = np.random.default_rng(3).uniform(0, 1, size=(ns,) + phi.shape)
    g = Grid(phi, block=block)
    st = State(g, ns, dtype).set_all(u0)
    p = make_params(phys)
    for call in range(2):
        ref = reference(st, p, 0)
        for s in range(ns):
            assert_same(noalloc(st, p, 0, s), ref[s])
        st.step(p, 7)  # the second call sees a different state and stale scratch contents
    again = [noalloc(st, p, -1, 0), noalloc(st, p, -1, 0)]
    np.testing.assert_array_equal(again[0], again[1])
    assert_same(again[0], reference(st, p, -1)[0])


def test_noalloc_f32r_state_is_read_only_and_multi_cta_ranges_follow_a_small_call():
    """The tortuosity solve's state type (SBG_F32R: FP32 correction on a
    compensated base): the entry point reduces b + d without refreshing the
    source or folding the correction, so the state's field stays bitwise the
    same; a 64^3 range of 8^3 blocks (several records of the fixed array)
    right after a small one (a single record) gives sbg_reduce's results,
    so records left by an earlier call do not leak into a later one."""
    small = random_blob_phi((13, 11, 9), 5, porosity=0.6, ell=1.5)
    big = random_blob_phi((64, 64, 64), 6, porosity=0.8, ell=4.0)
    d = (True, True, False, False, False, False)
    for phi in (small, big):
        dims = tuple(reversed(phi.shape))
        phys = Physics(dims=dims, dt=0.1, D=(1.0, 0.0), dirichlet=d, face_value=(1.0, 0.0, 0, 0, 0, 0))
        g = Grid(phi, block=8)
        st = State(g, 1, "f32r").set(np.random.default_rng(8).uniform(0, 1, phi.shape))
        p = make_params(phys)
        st.step(p, 37)  # a correction d that is not yet folded into the base
        before = st.get()
        a = noalloc(st, p, 0, 0)
        np.testing.assert_array_equal(st.get(), before)
        b = noalloc(st, p, 0, 0)
        np.testing.assert_array_equal(a, b)
        assert_same(a, reference(st, p, 0)[0])  # sbg_reduce refreshes and folds after it reduces
        assert_same(noalloc(st, p, 0, 0), reference(st, p, 0)[0])


def test_noalloc_reduction_of_one_geometry_of_a_batch():
    phis = [random_blob_phi((20, 17, 15), 9, porosity=0.5, ell=1.6),
            random_blob_phi((33, 25, 40), 10, porosity=0.6, ell=2.0)]
    gb = Grid.batch(phis, block=4)
    st = State(gb, 2, "f32")
    for i, phi in enumerate(phis):
        st.set_all(np.random.default_rng(i).uniform(0, 1, (2,) + phi.shape), geom=i)
    phys = Physics(dims=(20, 17, 15), dt=0.05, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.1), k_surf=0.3)
    p = make_params(phys)
    st.step(p, 9)
    for geom in (1, 0, -1):
        ref = reference(st, p, geom)
        for s in range(2):
            assert_same(noalloc(st, p, geom, s), ref[s])


def test_noalloc_reduction_rejects_a_range_beyond_its_fixed_array():
    """2^28 voxel slots is the stated limit: a 648^3 box with every voxel in
    the pore space has 81^3 blocks of 8^3 = 272M slots and is refused before
    any launch; the same call with sbg_reduce works."""
    lib = _abi.load()
    n = 648
    phi = torch.full((n, n, n), 2.0, dtype=torch.float32, device="cuda")
    g = Grid(phi, block=8)
    del phi
    assert g.n_blocks * 512 > 2 ** 28
    st = State(g, 1, "f32")
    p = make_params(Physics(dims=(n, n, n), dt=0.1))
    out = torch.zeros(_abi.NRED, dtype=torch.float64, device="cuda")
    rc = lib.sbg_reduce_noalloc(g.handle, st.handle, ctypes.byref(p), 0, 0, ctypes.c_void_p(out.data_ptr()), 0)
    assert rc == _abi.SBG_ERR_INVALID_ARG
    assert b"exceed the limit" in lib.sbg_last_error()
    st.close()
    g.close()


def test_noalloc_reduction_rejects_bad_arguments():
    lib = _abi.load()
    phi = np.full((8, 8, 8), 2.0, np.float32)
    g = Grid(phi, block=8)
    st = State(g, 1, "f32").set_all(np.ones((1, 8, 8, 8)))
    p = make_params(Physics(dims=(8, 8, 8), dt=0.1))
    out = torch.zeros(_abi.NRED, dtype=torch.float64, device="cuda")
    assert lib.sbg_reduce_noalloc(g.handle, st.handle, ctypes.byref(p), 0, 0, None, 0) == _abi.SBG_ERR_INVALID_ARG
    assert lib.sbg_reduce_noalloc(g.handle, st.handle, ctypes.byref(p), 0, 1,
                                  ctypes.c_void_p(out.data_ptr()), 0) == _abi.SBG_ERR_INVALID_ARG
    assert b"species" in lib.sbg_last_error()
