"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares; host-side argument checks reject bad input before any
device work."""
import ctypes
import glob
import os
import re

import pytest

from paper_2304_11165_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(sbg_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("sbg_build", "sbg_step", "sbg_reduce", "sbg_effective_D", "sbg_state_create",
                 "sbg_run_to_steady", "sbg_stability_limit"):
        assert core in names


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in _abi.SIGNATURES}
    assert declared_functions() <= bound, declared_functions() - bound


def test_version_and_status_strings():
    lib = _abi.load()
    assert lib.sbg_abi_version() >= 1
    assert lib.sbg_status_string(0) == b"ok"
    assert b"stability" in lib.sbg_status_string(4)


def test_build_rejects_bad_block_edge_without_touching_the_device():
    lib = _abi.load()
    phi = (ctypes.c_float * 8)(*([1.0] * 8))
    dims = (ctypes.c_int64 * 3)(2, 2, 2)
    opts = _abi.BuildOpts(5, 0, 0.0, 1.0, 0)
    out = ctypes.c_void_p()
    rc = lib.sbg_build(phi, dims, ctypes.byref(opts), None, ctypes.byref(out))
    assert rc == _abi.SBG_ERR_INVALID_ARG
    assert b"block" in lib.sbg_last_error()
    dims_bad = (ctypes.c_int64 * 3)(0, 2, 2)
    opts.block = 8
    assert lib.sbg_build(phi, dims_bad, ctypes.byref(opts), None, ctypes.byref(out)) == _abi.SBG_ERR_INVALID_ARG
    assert lib.sbg_build(None, dims, ctypes.byref(opts), None, ctypes.byref(out)) == _abi.SBG_ERR_INVALID_ARG


def test_stability_limit_host_function():
    from paper_2304_11165_b300 import make_params, stability_limit
    from workloads import Physics
    p = make_params(Physics(dims=(8, 8, 8), dt=0.1, nspecies=2, D=(1.0, 0.5), decay=(0.0, 0.001),
                            k_surf=0.05))
    assert abs(stability_limit(p, (8, 8, 8), 1.0) - 1 / 6.05) < 1e-15
    p2 = make_params(Physics(dims=(16, 16, 1), dt=0.1, dx=(0.5, 0.5, 1.0)))
    assert abs(stability_limit(p2, (16, 16, 1), 1.0) - 0.25 * 0.25) < 1e-15


def test_null_handles_are_rejected():
    lib = _abi.load()
    p = _abi.Params()
    assert lib.sbg_step(None, None, ctypes.byref(p), 1, None) == _abi.SBG_ERR_INVALID_ARG
    assert lib.sbg_reduce(None, None, ctypes.byref(p), 0, None, None) == _abi.SBG_ERR_INVALID_ARG
    assert lib.sbg_state_create(None, 1, 0, ctypes.byref(ctypes.c_void_p())) == _abi.SBG_ERR_INVALID_ARG


def test_redistance_rejects_bad_arguments_before_touching_the_device():
    """sbg_redistance validates every argument on the host: null pointers,
    dims outside [1, 2^20], a non-positive spacing, an unknown dtype, options
    out of range, a step that breaks the upwind scheme's monotonicity, a
    launch grid beyond the y/z limits, and a host call that would write over
    its own input."""
    lib = _abi.load()
    buf_in = (ctypes.c_float * 8)()
    buf_out = (ctypes.c_float * 8)()
    ok_dims = (ctypes.c_int64 * 3)(2, 2, 2)
    ok_dx = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    ok = _abi.RedistOpts(0.3, 10, 1e-3, 2.0, 5)

    def call(dims=ok_dims, dx=ok_dx, a=buf_in, b=buf_out, dtype=_abi.SBG_F32, opts=ok):
        rc = lib.sbg_redistance(dims, dx, a, b, dtype, 0, ctypes.byref(opts) if opts is not None else None,
                                None, None, None)
        return rc, lib.sbg_last_error().decode()

    assert call(dims=None)[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(opts=None)[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(dims=(ctypes.c_int64 * 3)(0, 2, 2))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(dims=(ctypes.c_int64 * 3)(2, 2, (1 << 20) + 1))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(dx=(ctypes.c_double * 3)(1.0, 0.0, 1.0))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(dx=(ctypes.c_double * 3)(1.0, float("nan"), 1.0))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(dtype=7)[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(opts=_abi.RedistOpts(0.3, -1, 1e-3, 2.0, 5))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(opts=_abi.RedistOpts(0.3, 10, 1e-3, 2.0, 0))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(opts=_abi.RedistOpts(0.0, 10, 1e-3, 2.0, 5))[0] == _abi.SBG_ERR_INVALID_ARG
    assert call(opts=_abi.RedistOpts(0.3, 10, 1e-3, 0.0, 5))[0] == _abi.SBG_ERR_INVALID_ARG
    rc, msg = call(opts=_abi.RedistOpts(0.4, 10, 1e-3, 2.0, 5))  # 0.4 * 1 * 3 = 1.2 > 1
    assert rc == _abi.SBG_ERR_INVALID_ARG and "above 1" in msg
    # anisotropic spacing: cfl * min(dx) * sum(1/dx) = 0.3 * 0.5 * (2 + 1 + 1) = 0.6 passes the test
    assert "above 1" not in call(dx=(ctypes.c_double * 3)(0.5, 1.0, 1.0), a=buf_in, b=buf_in)[1]
    rc, msg = call(dims=(ctypes.c_int64 * 3)(2, 8 * 65536, 1))
    assert rc == _abi.SBG_ERR_INVALID_ARG and "Ny" in msg
    rc, msg = call(b=buf_in)
    assert rc == _abi.SBG_ERR_INVALID_ARG and "differ" in msg
