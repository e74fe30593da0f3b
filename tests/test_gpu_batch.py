"""Batched geometries: one concatenated block list, one launch per step.

The batch must reproduce what separate grids compute, geometry by geometry,
and the batched steady-state solve must give each geometry the effective
diffusivity of its own solve and of the FP64 oracle's CG steady state."""
import numpy as np
import pytest

import oracle
from workloads import Physics, boolean_sphere_pack, grf_geometry, random_blob_phi
from workloads.configs import initial_with_faces

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402


def tortuosity_physics(dims, dt=0.15):
    d = (True, True, False, False, False, False)
    return Physics(dims=dims, dt=dt, D=(1.0, 0.0), dirichlet=d, face_value=(1.0, 0.0, 0, 0, 0, 0))


def small_batch():
    """Uneven boxes, spheres and GRFs, porosities 0.3-0.6."""
    geos = []
    for i, (side, kind, psi) in enumerate([(24, "grf", 0.45), (17, "spheres", 0.5), (31, "grf", 0.6),
                                           (20, "spheres", 0.4), (28, "grf", 0.35), (12, "grf", 0.55)]):
        if kind == "grf":
            phi = grf_geometry(side, 500 + i, psi, ell=3.0)
        else:
            phi, _, _ = boolean_sphere_pack(side, 3.0, 0.3, psi, 600 + i)
        geos.append(phi)
    return geos


def dense_of(state, geom, phi):
    out = np.zeros(phi.shape)
    return state.get(0, geom=geom, out=out)


@pytest.mark.parametrize("block", [4, 8])
def test_batched_steps_equal_separate_grids_bitwise(block):
    geos = small_batch()
    gb = Grid.batch(geos, block=block)
    na, begin, count = gb.geometry_info()
    sb = State(gb, 1, "f32")
    u0s = []
    for i, phi in enumerate(geos):
        phys = tortuosity_physics(tuple(reversed(phi.shape)))
        u0 = initial_with_faces(phys.dims, 0.0, phys) + np.random.default_rng(i).uniform(0, 0.5, phi.shape)
        u0s.append(u0)
        sb.set(u0, geom=i)
    p = make_params(tortuosity_physics((8, 8, 8)))
    sb.step(p, 70)
    for i, phi in enumerate(geos):
        g = Grid(phi, block=block)
        assert g.n_active == na[i]
        st = State(g, 1, "f32").set(u0s[i]).step(p, 70)
        np.testing.assert_array_equal(dense_of(sb, i, phi), st.get())


def test_batched_steady_solve_matches_single_solves_and_the_oracle():
    geos = small_batch()
    gb = Grid.batch(geos, block=4)
    sb = State(gb, 1, "f32x2")
    for i, phi in enumerate(geos):
        phys = tortuosity_physics(tuple(reversed(phi.shape)))
        sb.set(initial_with_faces(phys.dims, 0.0, phys), geom=i)
    p = make_params(tortuosity_physics((8, 8, 8)))
    steps, rel = sb.batch_run_to_steady(p, 1e-8, check_every=200, max_steps=400_000, raise_on_max=False)
    assert np.all(rel < 1e-8), (steps, rel)
    assert len(set(steps.tolist())) > 1  # geometries left the work list at different steps
    for i, phi in enumerate(geos):
        phys = tortuosity_physics(tuple(reversed(phi.shape)))
        d_eff, tau, psi = sb.effective_D(p, geom=i)
        g = Grid(phi, block=8)
        st = State(g, 1, "f32x2").set(initial_with_faces(phys.dims, 0.0, phys))
        st.run_to_steady(p, 1e-8, check_every=200, max_steps=400_000)
        d1, _, psi1 = st.effective_D(p)
        P = oracle.Problem(phi, phys)
        u_cg, relres, _ = P.steady_cg(initial_with_faces(phys.dims, 0.0, phys))
        d_ref, tau_ref, psi_ref = P.effective_D(u_cg)
        assert psi == psi1 == psi_ref
        if d_ref <= 1e-12:  # no percolating path: both must see no flux
            assert abs(d_eff) < 1e-9 and abs(d1) < 1e-9
            continue
        assert abs(d_eff - d1) <= 1e-6 * d_ref
        assert abs(d_eff - d_ref) <= 1e-6 * d_ref, (i, d_eff, d_ref)
        # a converged geometry stays frozen while the others keep stepping
        field = dense_of(sb, i, phi)
        np.testing.assert_allclose(field, st.get(), rtol=0, atol=1e-6)


@pytest.mark.parametrize("dtype", ["f32", "f32x2"])
def test_segmented_check_equals_per_geometry_reductions(dtype):
    """One check of the batched solve (one segmented reduction over every
    unconverged geometry) gives each geometry's relative residual exactly as
    separate per-geometry reductions of the same states do."""
    geos = small_batch()
    gb = Grid.batch(geos, block=4)
    sa = State(gb, 1, dtype)
    sb = State(gb, 1, dtype)
    for i, phi in enumerate(geos):
        phys = tortuosity_physics(tuple(reversed(phi.shape)))
        u0 = initial_with_faces(phys.dims, 0.0, phys)
        sa.set(u0, geom=i)
        sb.set(u0, geom=i)
    p = make_params(tortuosity_physics((8, 8, 8)))
    r0 = [sb.reduce(p, geom=i)[0]["residual"] for i in range(len(geos))]
    steps, rel = sa.batch_run_to_steady(p, 1e-30, check_every=64, max_steps=64, raise_on_max=False)
    assert np.all(steps == 64)
    sb.step(p, 64)
    for i in range(len(geos)):
        r1 = sb.reduce(p, geom=i)[0]["residual"]
        assert rel[i] == r1 / r0[i], (i, rel[i], r1 / r0[i])


def test_autotuner_picks_the_fastest_and_a_cache_hit_skips_the_timing(tmp_path, monkeypatch):
    from paper_2304_11165_b300 import autotune
    monkeypatch.setenv("SBG_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    geos = small_batch()[:3]
    phys = tortuosity_physics((8, 8, 8))
    cands = [(4, "async", 0), (8, "pipelined", 0), (4, "pipelined", 2)]
    fake = {cands[0]: 3.0, cands[1]: 1.5, cands[2]: 2.0}
    calls = []

    def timer(c):
        calls.append(c)
        return fake[c]

    best, table = autotune.tune(geos, phys, "f32", candidates=cands, timer=timer)
    assert (best["block"], best["variant"], best["ctas_per_sm"]) == cands[1] and not best["cached"]
    assert len(table) == 3 and calls == cands
    again, t2 = autotune.tune(geos, phys, "f32", candidates=cands, timer=timer)
    assert again["cached"] and t2 is None and len(calls) == 3
    # a different species count or state type is another key: timed again
    autotune.tune(geos, phys, "f32x2", candidates=cands, timer=timer)
    assert len(calls) == 6
    # the real timing of two candidates, without the cache
    real, table = autotune.tune(geos, phys, "f32", candidates=cands[:2], steps=8, use_cache=False)
    assert all(r["ns_per_voxel_update"] > 0 for r in table)
    assert real["ns_per_voxel_update"] == min(r["ns_per_voxel_update"] for r in table)
