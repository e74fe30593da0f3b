"""Failure detection without a fault on the device.

* A bounded wait that runs out: the test hook sbg_debug_stall_stage makes the
  ring-buffer step kernels skip the bulk copy of one group, so the CTA that
  owns it gives up its wait after a short bound, records SBG_ERR_TIMEOUT in
  the grid's error word and exits.  The next synchronising call reports the
  status; the device context stays usable and a fresh run gives the plain
  kernel's fields.
* An allocation that fails: the hook sbg_debug_fail_alloc makes the n-th
  next allocation of the library fail.  For every n up to the number of
  allocations an entry point makes, the call returns SBG_ERR_OOM and the
  library's table of live allocations is back where it was (nothing leaked).
"""
import ctypes
import gc

import numpy as np
import pytest

from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, State, _abi, make_params  # noqa: E402
from paper_2304_11165_b300.autograd import forward_record  # noqa: E402


def case(dims=(40, 36, 30), ns=1, seed=31):
    phi = random_blob_phi(dims, seed, porosity=0.6, ell=1.8)
    phys = Physics(dims=dims, dt=0.05, nspecies=ns, D=(1.0, 0.5), decay=(0.01, 0.1), k_surf=0.3 if ns == 2 else 0.0,
                   dirichlet=(True, False, False, False, False, False), face_value=(1.0, 0, 0, 0, 0, 0))
    u0 = np.random.default_rng(seed).uniform(0, 1, size=(ns,) + phi.shape)
    return phi, phys, u0


def live():
    """The library's live allocations (count, bytes), after Python has released
    every unreachable grid, state and tape (their destructors free them)."""
    gc.collect()
    torch.cuda.synchronize()
    n, b = ctypes.c_int64(), ctypes.c_int64()
    _abi.check(_abi.load().sbg_debug_live_allocations(ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


@pytest.mark.parametrize("variant,ns", [("async", 1), ("pipelined", 1), ("async", 2), ("prefetch", 1)])
def test_a_wait_that_runs_out_is_reported_and_the_context_stays_usable(variant, ns):
    lib = _abi.load()
    phi, phys, u0 = case(ns=ns)
    p = make_params(phys)
    g = Grid(phi, block=4)
    st = State(g, ns, "f32").set_kernel(variant).set_all(u0)
    _abi.check(lib.sbg_debug_stall_stage(g.handle, 1, 1 << 20))  # ~0.5 ms at the SM clock
    try:
        st.step(p, 3)
        with pytest.raises(SbgError) as e:
            st.reduce(p)
        assert e.value.status == _abi.SBG_ERR_TIMEOUT
    finally:
        _abi.check(lib.sbg_debug_stall_stage(g.handle, -1, 0))
    # the error word was read and cleared; the same grid and a fresh state work
    ref = State(g, ns, "f32").set_kernel("plain").set_all(u0).step(p, 9).get_all()
    again = State(g, ns, "f32").set_kernel(variant).set_all(u0).step(p, 9)
    again.reduce(p)
    np.testing.assert_array_equal(again.get_all(), ref)
    assert torch.cuda.is_available() and torch.zeros(4, device="cuda").sum().item() == 0.0


def test_the_stall_hook_rejects_bad_bounds():
    lib = _abi.load()
    phi, _, _ = case()
    g = Grid(phi, block=4)
    assert lib.sbg_debug_stall_stage(g.handle, 0, 0) == _abi.SBG_ERR_INVALID_ARG
    assert lib.sbg_debug_stall_stage(g.handle, 0, 1 << 40) == _abi.SBG_ERR_INVALID_ARG
    assert lib.sbg_debug_stall_stage(None, -1, 0) == _abi.SBG_ERR_INVALID_ARG


def failing_until_success(call, limit=200):
    """Runs call() with the n-th allocation failing for n = 1, 2, ... until it
    succeeds; each failure must be SBG_ERR_OOM with nothing leaked.  Returns
    (the call's result, the number of allocations it made)."""
    lib = _abi.load()
    base = live()
    try:
        for n in range(1, limit):
            _abi.check(lib.sbg_debug_fail_alloc(n))
            try:
                out = call()
            except SbgError as e:
                assert e.status == _abi.SBG_ERR_OOM, (n, e)
                del e
                assert live() == base, (n, live(), base)
                continue
            _abi.check(lib.sbg_debug_fail_alloc(0))
            return out, n - 1
        raise AssertionError("the call kept failing")
    finally:
        _abi.check(lib.sbg_debug_fail_alloc(0))


def test_failed_allocations_in_build_state_and_tape_leak_nothing():
    phi, phys, u0 = case(ns=2)
    p = make_params(phys)
    base = live()
    g, n_build = failing_until_success(lambda: Grid(phi, block=4, order="planes"))
    assert n_build >= 10  # tables, hash, scratch, weights: every one of them was made to fail once
    st, n_state = failing_until_success(lambda: State(g, 2, "f32"))
    assert n_state >= 1
    # a first step makes the grid's table of held (Dirichlet) voxels, which the grid keeps
    # for later steps: made here, it is not counted against the tape below
    st.set_all(u0).step(p, 2)
    st.set_all(u0)
    tape, n_tape = failing_until_success(lambda: forward_record(st, p, 10, 4))
    assert n_tape >= 3
    def state_from_host():
        # the host-pointer set allocates a staging buffer too; a state whose set failed is
        # destroyed here (the exception's traceback would otherwise keep it alive)
        s2 = State(g, 2, "f32")
        try:
            return s2.set_all(u0)
        except SbgError:
            s2.close()
            raise

    st2, n_set = failing_until_success(state_from_host)
    assert n_set >= 2
    del tape, st, st2
    g.close()
    assert live() == base


def test_fail_alloc_hook_rejects_a_negative_count():
    assert _abi.load().sbg_debug_fail_alloc(-1) == _abi.SBG_ERR_INVALID_ARG
