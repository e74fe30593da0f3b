"""Simulated FRAP on the GPU (Sec. 3.3): the box sum of every state type
against the oracle's, the device-recorded recovery curve against the
oracle's curve, the curve call against plain steps and box sums, and the
whole D_eff estimate against the oracle's composition of the same steps."""
import numpy as np
import pytest

import oracle
from workloads import Physics, centred_box, frap_initial, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, State, make_params  # noqa: E402
from paper_2304_11165_b300 import _abi, frap  # noqa: E402

BOXES = [((0, 0, 0), (1 << 30, 1 << 30, 1 << 30)), ((3, 2, 1), (17, 11, 9)), ((-4, 5, -2), (9, 40, 7)),
         ((6, 6, 6), (6, 9, 9)), ((30, 0, 0), (40, 5, 5)), ((1, 1, 1), (2, 2, 2))]


def blob(dims, seed, porosity=0.6):
    return random_blob_phi(dims, seed, porosity=porosity, ell=1.7)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f32x2", "f32r"])
@pytest.mark.parametrize("block", [4, 8])
def test_box_sum_matches_the_oracle(dtype, block):
    dims = (27, 21, 18)
    phi = blob(dims, 21)
    ph = Physics(dims=dims, dt=0.05, D=(1.0, 0.0), decay=(0.01, 0.0))
    P = oracle.Problem(phi, ph)
    u0 = np.random.default_rng(22).uniform(-1, 1, phi.shape)
    st = State(Grid(phi, block=block), 1, dtype).set(u0)
    st.step(make_params(ph), 37)   # an SBG_F32R state then holds an unfolded correction
    field = st.get()
    for lo, hi in BOXES:
        s, c = st.box_sum(lo, hi)
        so, co = P.box_sum(field[None], lo, hi)
        assert c == co, (lo, hi)
        assert abs(s - so) <= 1e-12 * max(1.0, abs(so)), (dtype, lo, hi, s, so)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32r", 2e-7), ("f32", 2e-5)])
def test_frap_curve_matches_the_oracle(dtype, tol):
    dims = (30, 26, 22)
    phi = blob(dims, 23, porosity=0.65)
    ph = Physics(dims=dims, dt=0.15, D=(1.0, 0.0))
    lo, hi = centred_box(dims, 9)
    u0 = frap_initial(phi.shape, lo, hi)
    ref, nref = oracle.Problem(phi, ph).frap_curve(u0[None], lo, hi, 16, 24)
    st = State(Grid(phi, block=4), 1, dtype).set(u0)
    sums, n = st.frap_curve(make_params(ph), lo, hi, 16, 24)
    assert n == nref
    assert np.max(np.abs(sums - ref)) <= tol * n


def test_frap_curve_equals_steps_and_box_sums():
    dims = (25, 20, 19)
    phi = blob(dims, 24)
    ph = Physics(dims=dims, dt=0.15, D=(0.8, 0.0))
    p = make_params(ph)
    lo, hi = centred_box(dims, 7)
    u0 = frap_initial(phi.shape, lo, hi)
    g = Grid(phi, block=8)
    a = State(g, 1, "f32r").set(u0)
    sums, _ = a.frap_curve(p, lo, hi, 66, 5)
    b = State(g, 1, "f32r").set(u0)
    loop = [b.box_sum(lo, hi)[0]]
    for _ in range(5):
        b.step(p, 66)
        loop.append(b.box_sum(lo, hi)[0])
    np.testing.assert_array_equal(sums, np.array(loop))
    np.testing.assert_array_equal(a.get(), b.get())


def oracle_effective_D(phi, ph, u0, lo, hi, sps, ns):
    """The same estimate composed from the oracle's steps, box sums and fit."""
    curves = []
    for field in (phi, np.full(phi.shape, 1.0e3, np.float32)):
        P = oracle.Problem(field, ph)
        total, nact = P.box_sum(P.shape_state(u0[None]), (0, 0, 0), ph.dims)
        sums, n = P.frap_curve(u0[None], lo, hi, sps, ns)
        curves.append(sums / (total / nact * n))
    t = ph.dt * sps * np.arange(ns + 1)
    return oracle.frap_fit(t, curves[0], t, curves[1], 1e-3, 1.0)


def test_effective_D_matches_the_oracle():
    dims = (32, 32, 32)
    phi = blob(dims, 25, porosity=0.7)
    ph = Physics(dims=dims, dt=0.15, D=(1.0, 0.0))
    lo, hi = centred_box(dims, 10)
    u0 = frap_initial(phi.shape, lo, hi)
    r = frap.effective_D(phi, ph, u0, lo, hi, 8, 40, dtype="f32r")
    s_ref, _ = oracle_effective_D(phi, ph, u0, lo, hi, 8, 40)
    assert 0.0 < r.scale < 1.0
    assert abs(r.scale - s_ref) <= 1e-5, (r.scale, s_ref)
    assert abs(r.tau - 1.0 / s_ref) <= 1e-5 * r.tau
    # a pore space that fills the box is the bulk box itself
    full = np.full(phi.shape, 2.0, np.float32)
    r1 = frap.effective_D(full, ph, u0, lo, hi, 8, 40, dtype="f32r")
    assert abs(r1.scale - 1.0) <= 1e-12 and r1.rss == 0.0


def test_recovery_is_normalised_by_the_library_like_the_oracle():
    """sbg_frap_recovery: t_i = i sps dt and F_i = M_box(t_i) / (c n_box) with c
    the conserved mean over the active voxels, against the oracle's box sums
    normalised the same way (Sec. 3.3); D_eff = s D for a D other than 1."""
    dims = (30, 27, 25)
    phi = blob(dims, 27, porosity=0.65)
    ph = Physics(dims=dims, dt=0.2, D=(0.7, 0.0))
    lo, hi = centred_box(dims, 8)
    u0 = frap_initial(phi.shape, lo, hi)
    st = State(Grid(phi, block=4), 1, "f64").set(u0)
    t, F, n_box = st.frap_recovery(make_params(ph), lo, hi, 6, 25)
    P = oracle.Problem(phi, ph)
    total, nact = P.box_sum(P.shape_state(u0[None]), (0, 0, 0), ph.dims)
    sums, n = P.frap_curve(u0[None], lo, hi, 6, 25)
    assert n_box == n
    np.testing.assert_allclose(t, ph.dt * 6 * np.arange(26), rtol=0, atol=1e-15)
    np.testing.assert_allclose(F, sums / (total / nact * n), rtol=1e-12, atol=1e-14)
    r = frap.effective_D(phi, ph, u0, lo, hi, 6, 25, dtype="f32r")
    assert abs(r.D_eff - r.scale * 0.7) <= 1e-15 and abs(r.tau * r.scale - 1.0) <= 1e-15


def test_argument_checks():
    dims = (12, 10, 9)
    phi = blob(dims, 26)
    ph = Physics(dims=dims, dt=0.1)
    st = State(Grid(phi, block=4), 1, "f32").set(np.ones(phi.shape))
    p = make_params(ph)
    for bad in (dict(species=1), dict(geom=1)):
        with pytest.raises(SbgError) as e:
            st.box_sum((0, 0, 0), (4, 4, 4), **bad)
        assert e.value.status == _abi.SBG_ERR_INVALID_ARG
        with pytest.raises(SbgError):
            st.frap_curve(p, (0, 0, 0), (4, 4, 4), 2, 2, **bad)
    with pytest.raises(SbgError):
        st.frap_curve(p, (0, 0, 0), (4, 4, 4), 0, 2)
    # an empty box sums to zero
    assert st.box_sum((5, 5, 5), (5, 9, 9)) == (0.0, 0)
