"""SBG_F32R states (FP32 correction d on a compensated base b, source
r = L_h b refreshed and d folded every 256 steps and at every reduction):
parity with the FP64 oracle, bitwise consistency across block sizes and step
kernels, steady states against the oracle's CG solve, and the batch solver."""
import numpy as np
import pytest

import oracle
from workloads import Physics, grf_geometry, random_blob_phi
from workloads.configs import initial_with_faces

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def blob_case(dims, k, seed, faces=(0, 1)):
    phi = random_blob_phi(dims, seed, porosity=0.55, ell=1.7)
    phi = np.where(phi > 0, phi * 0.7, phi).astype(np.float32)
    d = tuple(f in faces for f in range(6))
    v = tuple(1.0 if f == 0 else 0.0 for f in range(6))
    phys = Physics(dims=dims, dt=0.05, D=(1.0, 0.0), decay=(0.01, 0.0), k_surf=k, dx=(1.0, 0.9, 1.1),
                   dirichlet=d, face_value=v)
    u0 = np.random.default_rng(seed).uniform(0, 1, size=phi.shape)
    return phi, phys, u0


@pytest.mark.parametrize("block,k", [(4, 0.0), (8, 0.4), (4, 0.4)])
def test_f32r_steps_match_the_oracle(block, k):
    """600 steps cross two refreshes (at 256 and 512); the error is far below
    plain FP32's because d only carries the change since the last fold."""
    phi, phys, u0 = blob_case((29, 23, 19), k, 40 + block)
    ref = oracle.Problem(phi, phys).run(u0[None], 600)[0]
    g = Grid(phi, block=block)
    st = State(g, 1, "f32r").set(u0)
    st.step(make_params(phys), 600)
    assert rel_err(st.get(), ref) < 2e-7


def test_f32r_is_bitwise_independent_of_block_size_and_kernel():
    phi, phys, u0 = blob_case((37, 29, 23), 0.3, 51)
    p = make_params(phys)
    outs = []
    for block, variant in ((4, "plain"), (4, "pipelined"), (4, "prefetch"), (4, "async"), (8, "pipelined"),
                           (8, "async"), (8, "plain")):
        g = Grid(phi, block=block)
        st = State(g, 1, "f32r").set_kernel(variant).set(u0)
        st.step(p, 200)
        outs.append(st.get())
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)


def test_f32r_step_counts_do_not_depend_on_call_pattern():
    """One call of 300 steps equals 300 calls of one step (the refresh points
    follow the state's own step count)."""
    phi, phys, u0 = blob_case((21, 17, 13), 0.2, 52)
    p = make_params(phys)
    g = Grid(phi, block=8)
    a = State(g, 1, "f32r").set(u0).step(p, 300).get()
    st = State(g, 1, "f32r").set(u0)
    for _ in range(300):
        st.step(p, 1)
    np.testing.assert_array_equal(a, st.get())


@pytest.mark.parametrize("k,res_tol", [(0.0, 1e-10), (0.4, 1e-7)])
def test_f32r_reduction_matches_the_oracle_and_leaves_the_field(k, res_tol):
    """The reduction of an SBG_F32R state against the oracle's reduction of the
    same field (read back in FP64), and the field against the oracle's run.
    The first 256 steps after a set carry the whole change in d, so the field
    is FP32-accurate there; the reduction itself is double-float.  With a
    surface reaction the residual uses the FP32 surface weights the step uses
    (the oracle's are FP64), which bounds its agreement at ~1e-7."""
    phi, phys, u0 = blob_case((26, 21, 19), k, 53)
    P = oracle.Problem(phi, phys)
    ref_u = P.run(u0[None], 90)
    g = Grid(phi, block=4)
    st = State(g, 1, "f32r").set(u0)
    p = make_params(phys)
    st.step(p, 90)
    before = st.get()
    red = st.reduce(p)[0]
    after = st.get()
    # the fold changes the representation, not the field (double-float rounding)
    assert np.max(np.abs(after - before)) <= 1e-12
    assert rel_err(before, ref_u[0]) < 2e-7
    ref = P.reduce(before[None])[0]
    assert abs(red["mass"] - ref["mass"]) <= 1e-12 * abs(ref["mass"])
    assert abs(red["residual"] - ref["residual"]) <= res_tol * ref["residual"]
    for key in ("J_in", "J_out"):
        assert abs(red[key] - ref[key]) <= 1e-10 * max(abs(ref[key]), 1.0)
    assert red["n_active"] == ref["n_active"]


def test_f32r_steady_state_matches_the_oracle_cg():
    phi = grf_geometry(40, 77, 0.45, ell=4.0)
    d = (True, True, False, False, False, False)
    phys = Physics(dims=(40, 40, 40), dt=0.15, D=(1.0, 0.0), dirichlet=d, face_value=(1.0, 0.0, 0, 0, 0, 0))
    u0 = initial_with_faces(phys.dims, 0.0, phys)
    P = oracle.Problem(phi, phys)
    u_cg, relres, _ = P.steady_cg(u0)
    d_ref, tau_ref, psi_ref = P.effective_D(u_cg)
    g = Grid(phi, block=4)
    st = State(g, 1, "f32r").set(u0)
    p = make_params(phys)
    steps, rel = st.run_to_steady(p, 1e-11, check_every=256, max_steps=600_000)
    assert rel < 1e-11
    d_eff, tau, psi = st.effective_D(p)
    assert psi == psi_ref
    assert abs(d_eff - d_ref) <= 1e-8 * d_ref, (d_eff, d_ref)
    assert rel_err(st.get(), u_cg[0] if u_cg.ndim == 4 else u_cg) < 1e-8


def test_f32r_batch_steady_solve_matches_single_solves():
    geos = [grf_geometry(side, 700 + i, psi, ell=3.0) for i, (side, psi) in
            enumerate([(24, 0.5), (31, 0.6), (20, 0.45), (28, 0.55)])]
    d = (True, True, False, False, False, False)
    gb = Grid.batch(geos, block=4)
    sb = State(gb, 1, "f32r")
    for i, phi in enumerate(geos):
        phys = Physics(dims=tuple(reversed(phi.shape)), dt=0.15, D=(1.0, 0.0), dirichlet=d,
                       face_value=(1.0, 0.0, 0, 0, 0, 0))
        sb.set(initial_with_faces(phys.dims, 0.0, phys), geom=i)
    p = make_params(Physics(dims=(8, 8, 8), dt=0.15, D=(1.0, 0.0), dirichlet=d, face_value=(1.0, 0.0, 0, 0, 0, 0)))
    steps, rel = sb.batch_run_to_steady(p, 1e-9, check_every=128, max_steps=300_000, raise_on_max=False)
    assert np.all(rel < 1e-9), (steps, rel)
    for i, phi in enumerate(geos):
        phys = Physics(dims=tuple(reversed(phi.shape)), dt=0.15, D=(1.0, 0.0), dirichlet=d,
                       face_value=(1.0, 0.0, 0, 0, 0, 0))
        u_cg, _, _ = oracle.Problem(phi, phys).steady_cg(initial_with_faces(phys.dims, 0.0, phys))
        d_ref, _, _ = oracle.Problem(phi, phys).effective_D(u_cg)
        d_eff, _, _ = sb.effective_D(p, geom=i)
        if d_ref <= 1e-12:
            assert abs(d_eff) < 1e-9
            continue
        assert abs(d_eff - d_ref) <= 1e-7 * d_ref, (i, d_eff, d_ref)
