"""Handle lifecycle on the device: building, stepping, reducing and
destroying grids and states (every state type, the source, FRAP and
redistancing calls) many times leaves the device's free memory where it was:
no allocation leaks per call."""
import numpy as np
import pytest

from workloads import Physics, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params, redistance  # noqa: E402


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def cycle(phi, u0, ph):
    p = make_params(ph)
    g = Grid(phi, block=4)
    g.set_diffusivity(np.ones(phi.shape))
    g.clear_diffusivity()
    for dtype in ("f32", "f64", "f32x2", "f32r"):
        st = State(g, 1, dtype).set(u0)
        st.step(p, 70)
        st.reduce(p)
        st.box_sum((0, 0, 0), (5, 5, 5))
        if dtype in ("f32", "f64"):
            st.set_source(u0)
            st.step_source(p, [1.0, 0.5])
        st.frap_curve(p, (2, 2, 2), (8, 8, 8), 2, 2)
        st.close()
    g.close()
    redistance(np.where(phi > 0, 1.0, -1.0).astype(np.float32), max_iter=3)


def test_repeated_create_and_destroy_does_not_leak_device_memory():
    dims = (40, 36, 30)
    phi = random_blob_phi(dims, 41, porosity=0.6, ell=1.7)
    u0 = np.random.default_rng(41).uniform(0, 1, phi.shape)
    ph = Physics(dims=dims, dt=0.05, D=(1.0, 0.0), dirichlet=(True, True, False, False, False, False),
                 face_value=(1.0, 0.0, 0, 0, 0, 0))
    cycle(phi, u0, ph)  # first use: library statics, pools, module loading
    before = free_bytes()
    for _ in range(12):
        cycle(phi, u0, ph)
    after = free_bytes()
    # the stream-ordered pool may keep a few MB cached; a leak per cycle would be
    # at least the grid and state arrays (~1 MB here) x 12
    assert before - after <= 4 << 20, (before, after)
