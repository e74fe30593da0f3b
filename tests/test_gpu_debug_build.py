"""The debug build of the library (libsbg_debug.so, compiled with SBG_DEBUG:
every face id and band-row index checked against its table inside the step
kernels).  It runs in a child process (SBG_LIB_VARIANT=debug selects it) and
must (1) give the release kernels' fields bitwise, with no error, and (2)
report an index outside the block list as SBG_ERR_BOUNDS instead of reading
outside the state.  The planted index is the block count itself: the first
block past the list, whose slots lie inside the state's allocation, so that
even a check that failed would not read outside device memory."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2304_11165_b300 import Grid, SbgError, State, _abi, make_params
from workloads import Physics, random_blob_phi
assert _abi.LIB_NAME == "libsbg_debug.so"
lib = _abi.load()
dims = (37, 29, 23)
phi = random_blob_phi(dims, 41, porosity=0.55, ell=1.7)
phys = Physics(dims=dims, dt=0.05, nspecies=2, D=(1.0, 0.45), decay=(0.01, 0.2), k_surf=0.6)
u0 = np.random.default_rng(41).uniform(0, 1, size=(2,) + phi.shape)
p = make_params(phys)
g = Grid(phi, block=4, order="planes")
fields = []
for variant in ("plain", "stream", "async"):
    st = State(g, 2, "f32").set_kernel(variant).set_all(u0).step(p, 25)
    st.reduce(p)  # raises if the error word was set
    fields.append(st.get_all())
for f in fields[1:]:
    np.testing.assert_array_equal(fields[0], f)
print("parity ok")
old = ctypes.c_int32()
block = 3
_abi.check(lib.sbg_debug_set_face(g.handle, block, 1, g.n_blocks, ctypes.byref(old)))
for variant in ("stream", "plain"):
    st = State(g, 2, "f32").set_kernel(variant).set_all(u0).step(p, 1)
    try:
        st.reduce(p)
        raise SystemExit("planted index not reported by the %s kernel" % variant)
    except SbgError as e:
        assert e.status == _abi.SBG_ERR_BOUNDS, e
print("bounds ok")
_abi.check(lib.sbg_debug_set_face(g.handle, block, 1, old.value, None))
st = State(g, 2, "f32").set_kernel("stream").set_all(u0).step(p, 25)
st.reduce(p)
np.testing.assert_array_equal(st.get_all(), fields[0])
print("restored ok")
'''


def test_debug_build_matches_the_release_kernels_and_reports_bad_indices():
    from paper_2304_11165_b300 import build
    build.build(debug=True)  # no-op when libsbg_debug.so is current
    env = dict(os.environ, SBG_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "parity ok" in r.stdout and "bounds ok" in r.stdout and "restored ok" in r.stdout, r.stdout
