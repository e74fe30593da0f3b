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
