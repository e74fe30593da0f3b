"""Degenerate boxes against the oracle: a single voxel, lines and planes of
voxels (one or two axes of extent 1), a box thinner than a block in every
direction, and a pore space of isolated voxels (every neighbour mirrored), in
every state type and both block edges, with held faces and reactions where
they make sense; plus the F32R / batch paths on the same shapes."""
import numpy as np
import pytest

import oracle
from workloads import Physics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402

SHAPES = [(1, 1, 1), (1, 1, 13), (1, 11, 1), (9, 1, 1), (1, 7, 9), (3, 3, 3), (2, 5, 6)]


def tol(dtype):
    # SBG_F32X2 keeps the state to ~48 bits, but each step's increment is formed in FP32
    # arithmetic (differences of the hi and of the lo parts), so its error grows by about an
    # FP32 ulp of the increment per step
    return {"f64": 1e-13, "f32": 2e-6, "f32x2": 1e-8, "f32r": 1e-6}[dtype]


@pytest.mark.parametrize("zyx", SHAPES)
@pytest.mark.parametrize("block", [4, 8])
@pytest.mark.parametrize("dtype", ["f64", "f32", "f32x2", "f32r"])
def test_thin_boxes_match_the_oracle(zyx, block, dtype):
    nz, ny, nx = zyx
    dims = (nx, ny, nz)
    phi = np.full(zyx, 3.0, np.float32)
    held = nx > 1
    ph = Physics(dims=dims, dt=0.1, D=(1.0, 0.0), decay=(0.02, 0.0), dx=(1.0, 0.8, 1.2),
                 dirichlet=(held, held, False, False, False, False), face_value=(1.0, 0.0, 0, 0, 0, 0))
    u0 = np.random.default_rng(sum(zyx)).uniform(0, 1, zyx)
    ref = oracle.Problem(phi, ph).run(u0[None], 90)[0]
    for variant in (["plain", "async"] if dtype != "f64" else ["plain"]):
        st = State(Grid(phi, block=block), 1, dtype).set_kernel(variant).set(u0)
        st.step(make_params(ph), 90)
        out = st.get()
        assert np.max(np.abs(out - ref)) <= tol(dtype) * max(1.0, np.max(np.abs(ref))), (variant, zyx)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f32r"])
def test_isolated_voxels_only_react(dtype):
    """A checkerboard pore space: no two pore voxels share a face, so every
    neighbour is mirrored and each voxel decays on its own, u (1 - dt decay)^n."""
    zyx = (6, 7, 9)
    z, y, x = np.indices(zyx)
    phi = np.where((x + y + z) % 2 == 0, 1.5, -1.0).astype(np.float32)
    ph = Physics(dims=zyx[::-1], dt=0.15, D=(1.0, 0.0), decay=(0.05, 0.0))
    u0 = np.random.default_rng(3).uniform(0.5, 1, zyx)
    st = State(Grid(phi, block=4), 1, dtype).set(u0)
    st.step(make_params(ph), 40)
    out = st.get()
    pore = phi > 0
    expected = u0 * (1.0 - 0.15 * 0.05) ** 40
    assert np.max(np.abs(out[pore] - expected[pore])) <= tol(dtype)
    assert np.all(out[~pore] == 0.0)
