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
    opts = _abi.BuildOpts(5, 0, 0.0, 1.0)
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
