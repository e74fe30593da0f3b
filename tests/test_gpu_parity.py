"""Parity of the CUDA path with the FP64 oracle, element by element, on small
seeded inputs that span several blocks and ragged box edges, plus the
invariances the block layout must respect.  Every call goes through the C ABI."""
import numpy as np
import pytest

import oracle
from workloads import Physics, channel_phi, random_blob_phi, spheres64
from workloads.configs import initial_with_faces

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, State, make_params  # noqa: E402
from paper_2304_11165_b300 import _abi  # noqa: E402


def dirich(*faces, values=None):
    d = [False] * 6
    v = [0.0] * 6
    for i, f in enumerate(faces):
        d[f] = True
        if values is not None:
            v[f] = values[i]
    return tuple(d), tuple(v)


def gpu_run(phi, phys, u0, nsteps, block=8, dtype="f64"):
    g = Grid(phi, block=block)
    st = State(g, phys.nspecies, dtype)
    st.set_all(u0)
    st.step(make_params(phys), nsteps)
    out = st.get_all()
    return out, g, st


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


CASES = [
    # dims, block, nspecies, k, dirichlet faces
    ((13, 11, 9), 4, 1, 0.0, (0,)),
    ((21, 13, 10), 8, 1, 0.0, (0, 1)),
    ((17, 19, 12), 8, 2, 0.6, (3,)),
    ((24, 16, 16), 4, 2, 0.6, ()),
    ((9, 8, 33), 8, 1, 0.3, (5,)),
]


def make_case(dims, ns, k, faces, seed):
    phi = random_blob_phi(dims, seed, porosity=0.55, ell=1.7)
    phi = np.where(phi > 0, phi * 0.7, phi).astype(np.float32)
    d, v = dirich(*faces, values=[1.0] * len(faces))
    phys = Physics(dims=dims, dt=0.05, nspecies=ns, D=(1.0, 0.45), decay=(0.01, 0.2), k_surf=k,
                   dx=(1.0, 0.9, 1.1), dirichlet=d, face_value=v)
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(0, 1, size=(ns,) + phi.shape)
    return phi, phys, u0


@pytest.mark.parametrize("case", range(len(CASES)))
def test_grid_tables_match_brute_force(case):
    dims, block, ns, k, faces = CASES[case]
    phi, phys, u0 = make_case(dims, ns, k, faces, 100 + case)
    P = oracle.Problem(phi, phys)
    g = Grid(phi, block=block)
    nbr, blocks = g.tables()
    nx, ny, nz = dims
    nbx, nby, nbz = [(n + block - 1) // block for n in dims]
    act = np.zeros((nbz * block, nby * block, nbx * block), bool)
    act[:nz, :ny, :nx] = P.active > 0
    occ = act.reshape(nbz, block, nby, block, nbx, block).any(axis=(1, 3, 5))
    # tiled order: tiles of T^3 blocks (T = 32 / B, 32^3 voxels), tiles and blocks inside a tile x-fastest
    T = 32 // block
    ntx, nty, ntz = [(n + T - 1) // T for n in (nbx, nby, nbz)]
    expect = []
    for tz in range(ntz):
        for ty in range(nty):
            for tx in range(ntx):
                for iz in range(T):
                    for iy in range(T):
                        for ix in range(T):
                            bx, by, bz = tx * T + ix, ty * T + iy, tz * T + iz
                            if bx < nbx and by < nby and bz < nbz and occ[bz, by, bx]:
                                expect.append((bx, by, bz))
    assert [tuple(b[:3]) for b in blocks] == expect
    assert g.n_active == int(P.active.sum())
    index = {c: i for i, c in enumerate(expect)}
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)]
    for i, (bx, by, bz) in enumerate(expect):
        for kk, (dx, dy, dz) in enumerate(offs):
            assert nbr[i, kk] == index.get((bx + dx, by + dy, bz + dz), -1)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_steps_match_oracle(case):
    dims, block, ns, k, faces = CASES[case]
    phi, phys, u0 = make_case(dims, ns, k, faces, 200 + case)
    P = oracle.Problem(phi, phys)
    ref = P.run(u0, 40)
    out, _, _ = gpu_run(phi, phys, u0, 40, block=block, dtype="f64")
    assert rel_err(out, ref) < 1e-13


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp32_steps_match_oracle(case):
    dims, block, ns, k, faces = CASES[case]
    phi, phys, u0 = make_case(dims, ns, k, faces, 300 + case)
    P = oracle.Problem(phi, phys)
    ref = P.run(u0, 300)
    out, _, _ = gpu_run(phi, phys, u0, 300, block=block, dtype="f32")
    assert rel_err(out, ref) < 1e-5


def test_block_size_and_graph_path_are_bitwise_identical():
    phi, phys, u0 = make_case((30, 27, 22), 2, 0.5, (0,), 7)
    a, _, _ = gpu_run(phi, phys, u0, 130, block=4, dtype="f32")
    b, _, _ = gpu_run(phi, phys, u0, 130, block=8, dtype="f32")
    np.testing.assert_array_equal(a, b)
    # 130 steps = two captured 64-step graphs + 2 single launches; compare with 130 single launches
    g = Grid(phi, block=8)
    st = State(g, 2, "f32").set_all(u0)
    p = make_params(phys)
    for _ in range(130):
        st.step(p, 1)
    np.testing.assert_array_equal(st.get_all(), b)


def test_translation_invariance_bitwise():
    dims = (20, 18, 14)
    phi, phys, u0 = make_case(dims, 1, 0.0, (), 8)
    pad = np.full((14 + 10, 18 + 6, 20 + 5), -3.0, np.float32)
    pad[7:21, 3:21, 3:23] = phi
    up = np.zeros((1,) + pad.shape)
    up[:, 7:21, 3:21, 3:23] = u0
    phys2 = Physics(dims=(25, 24, 24), dt=phys.dt, D=phys.D, decay=phys.decay, dx=phys.dx)
    a, _, _ = gpu_run(phi, phys, u0, 60, block=8, dtype="f32")
    b, _, _ = gpu_run(pad, phys2, up, 60, block=8, dtype="f32")
    np.testing.assert_array_equal(a, b[:, 7:21, 3:21, 3:23])


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_reductions_match_oracle(dtype, tol):
    """Mass, fluxes and residual against the oracle.  Each difference is
    bounded by `tol` times the sum of the magnitudes that enter the quantity
    (the FP32 field error is relative to the field, and fluxes and residuals
    are differences of field values)."""
    phi, phys, u0 = make_case((26, 21, 19), 2, 0.4, (0, 1), 9)
    P = oracle.Problem(phi, phys)
    ref_u = P.run(u0, 25)
    ref = P.reduce(ref_u)
    g = Grid(phi, block=8)
    st = State(g, 2, dtype).set_all(u0)
    p = make_params(phys)
    st.step(p, 25)
    red = st.reduce(p)
    act = P.active > 0
    for s in range(2):
        u = np.abs(ref_u[s]) * act
        D = phys.D[s]
        rate = 4 * D * sum(1 / d ** 2 for d in phys.dx) + phys.decay[s] + phys.k_surf
        scale = {"mass": u.sum() * np.prod(phys.dx),
                 "J_in": D * (u[:, :, 0] + u[:, :, 1]).sum() * phys.dx[1] * phys.dx[2] / phys.dx[0],
                 "J_out": D * (u[:, :, -2] + u[:, :, -1]).sum() * phys.dx[1] * phys.dx[2] / phys.dx[0],
                 "residual": np.sqrt(((rate * u) ** 2).sum())}
        for key in ("mass", "J_in", "J_out", "residual"):
            assert abs(red[s][key] - ref[s][key]) <= tol * scale[key], (s, key, red[s][key], ref[s][key])
        assert red[s]["n_active"] == ref[s]["n_active"]
        assert red[s]["nonfinite"] == 0


@pytest.mark.parametrize("block,ns,k", [(4, 2, 0.4), (8, 2, 0.4), (4, 1, 0.3), (4, 2, 0.0)])
def test_fp32_reduction_of_a_state_matches_the_oracle_on_the_same_values(block, ns, k):
    """The reduction arithmetic alone: the FP32 state's checks against the
    oracle's FP64 checks of the very same stored values.  Mass and fluxes agree
    to the double-float accumulation (1e-12 of their scale); the residual also
    carries the FP32 rounding of the surface weights (the kernels read the
    weights the step uses), so it gets 1e-6 of the transfer term's scale."""
    phi, phys, u0 = make_case((27, 22, 18), ns, k, (0, 2), 12)
    P = oracle.Problem(phi, phys)
    g = Grid(phi, block=block)
    st = State(g, ns, "f32").set_all(u0)
    p = make_params(phys)
    st.step(p, 30)
    u = st.get_all()
    ref = P.reduce(u)
    red = st.reduce(p)
    act = P.active > 0
    for s in range(ns):
        a = np.abs(u[s]) * act
        D = phys.D[s]
        rate = 4 * D * sum(1 / d ** 2 for d in phys.dx) + phys.decay[s] + k
        scale = {"mass": a.sum() * np.prod(phys.dx),
                 "J_in": D * (a[:, :, 0] + a[:, :, 1]).sum() * phys.dx[1] * phys.dx[2] / phys.dx[0],
                 "J_out": D * (a[:, :, -2] + a[:, :, -1]).sum() * phys.dx[1] * phys.dx[2] / phys.dx[0]}
        for key in ("mass", "J_in", "J_out"):
            assert abs(red[s][key] - ref[s][key]) <= 1e-12 * scale[key], (s, key, red[s][key], ref[s][key])
        transfer = np.sqrt(((k * np.abs(u[0]) * act) ** 2).sum())
        res_tol = 1e-12 * np.sqrt(((rate * a) ** 2).sum()) + 1e-6 * transfer
        assert abs(red[s]["residual"] - ref[s]["residual"]) <= res_tol, (s, red[s]["residual"], ref[s]["residual"])
        assert red[s]["n_active"] == ref[s]["n_active"]
        assert red[s]["min"] == u[s][act].min() and red[s]["max"] == u[s][act].max()


def test_spheres64_fp64_matches_oracle():
    """64^3, 20 spheres, FP64, c = 1 held on x = 0, D = 1, dt = 0.1, 100 steps."""
    phi, u0, phys = spheres64()
    P = oracle.Problem(phi, phys)
    ref = P.run(u0, phys.steps)
    out, g, st = gpu_run(phi, phys, u0, phys.steps, block=8, dtype="f64")
    assert rel_err(out, ref) < 1e-13
    m_ref = P.reduce(ref)[0]["mass"]
    m = st.reduce(make_params(phys))[0]["mass"]
    assert abs(m - m_ref) <= 1e-13 * m_ref


def test_channel_steady_state_gives_exact_deff():
    dims = (40, 12, 12)
    phi = channel_phi(dims, (3, 8), (4, 9))
    d, v = dirich(0, 1, values=[1.0, 0.0])
    phys = Physics(dims=dims, dt=0.15, D=(1.0, 0.0), dirichlet=d, face_value=v)
    u0 = initial_with_faces(dims, 0.0, phys)
    g = Grid(phi, block=8)
    st = State(g, 1, "f32x2").set(u0)
    p = make_params(phys)
    steps, rel = st.run_to_steady(p, 1e-10, check_every=500, max_steps=2_000_000)
    d_eff, tau, psi = st.effective_D(p)
    assert abs(psi - 25 / 144) < 1e-15
    assert abs(d_eff - psi) < 1e-6 * psi
    assert abs(tau - 1.0) < 1e-6


def test_unstable_dt_is_rejected_and_nan_is_reported():
    phi, phys, u0 = make_case((16, 16, 16), 1, 0.0, (0,), 10)
    g = Grid(phi, block=8)
    st = State(g, 1, "f32").set_all(u0)
    p = make_params(phys, dt=1.0)
    with pytest.raises(SbgError) as e:
        st.step(p, 1)
    assert e.value.status == _abi.SBG_ERR_UNSTABLE_DT
    u_bad = u0.copy()
    P = oracle.Problem(phi, phys)
    z, y, x = np.argwhere((P.active > 0) & (P.fixed == 0))[0]
    u_bad[0, z, y, x] = np.nan
    st.set_all(u_bad)
    p = make_params(phys)
    assert st.reduce(p)[0]["nonfinite"] == 1
    with pytest.raises(SbgError) as e:
        st.run_to_steady(p, 1e-6, check_every=10, max_steps=100)
    assert e.value.status == _abi.SBG_ERR_NONFINITE


def test_empty_and_full_geometries():
    phys = Physics(dims=(10, 9, 8), dt=0.1)
    g = Grid(np.full((8, 9, 10), -1.0, np.float32), block=8)
    assert g.n_blocks == 0 and g.n_active == 0
    st = State(g, 1, "f32")
    st.step(make_params(phys), 3)
    assert st.reduce(make_params(phys))[0]["n_active"] == 0
    assert np.all(st.get() == 0)
    full = np.full((8, 9, 10), 2.0, np.float32)
    u0 = np.random.default_rng(0).uniform(size=(8, 9, 10))
    ref = oracle.Problem(full, phys).run(u0, 20)
    out, _, _ = gpu_run(full, phys, u0[None], 20, block=4, dtype="f64")
    assert rel_err(out, ref) < 1e-13


@pytest.mark.parametrize("block", [4, 8])
@pytest.mark.parametrize("dtype,ns,k", [("f32", 1, 0.0), ("f32", 1, 0.4), ("f32", 2, 0.6), ("f32", 2, 0.0),
                                        ("f32x2", 1, 0.0), ("f32x2", 1, 0.5)])
def test_pipelined_kernel_is_bitwise_the_plain_kernel(block, dtype, ns, k):
    """The bulk-copy pipelined kernel and the one-thread-per-voxel kernel give
    bitwise the same fields (same pinned per-voxel arithmetic), including a
    ragged last group and Dirichlet faces."""
    phi, phys, u0 = make_case((37, 29, 23), ns, k, (0, 1), 11)
    p = make_params(phys)
    outs = []
    for variant in ("plain", "pipelined", "prefetch", "async", "stream"):
        g = Grid(phi, block=block)
        st = State(g, ns, dtype).set_kernel(variant).set_all(u0)
        st.step(p, 77)
        outs.append(st.get_all())
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)
    ref = oracle.Problem(phi, phys).run(u0, 77)
    assert rel_err(outs[1], ref) < 1e-5


def test_pipelined_kernel_with_few_ctas_walks_long_ranges():
    """One persistent CTA per SM over a grid with many groups per CTA."""
    phi, phys, u0 = make_case((64, 60, 56), 1, 0.0, (0,), 12)
    p = make_params(phys)
    g = Grid(phi, block=4)
    a = State(g, 1, "f32").set_kernel("plain").set_all(u0).step(p, 20).get_all()
    b = State(g, 1, "f32").set_kernel("pipelined", ctas_per_sm=1).set_all(u0).step(p, 20).get_all()
    c = State(g, 1, "f32").set_kernel("prefetch", ctas_per_sm=1).set_all(u0).step(p, 20).get_all()
    d = State(g, 1, "f32").set_kernel("async", ctas_per_sm=1).set_all(u0).step(p, 20).get_all()
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(a, d)


@pytest.mark.parametrize("block", [4, 8])
def test_two_species_two_row_kernel_with_few_ctas(block):
    """Two species with the surface transfer on the two-row kernel (cp.async
    halos), one and two persistent CTAs per SM: many groups per CTA, both
    halo buffers reused, the same fields as the one-thread-per-voxel kernel."""
    phi, phys, u0 = make_case((64, 60, 56), 2, 0.6, (0, 1), 13)
    p = make_params(phys)
    g = Grid(phi, block=block)
    a = State(g, 2, "f32").set_kernel("plain").set_all(u0).step(p, 31).get_all()
    for per_sm in (1, 2, 0):
        b = State(g, 2, "f32").set_kernel("async", ctas_per_sm=per_sm).set_all(u0).step(p, 31).get_all()
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("block", [4, 8])
def test_compensated_two_row_kernel_with_few_ctas(block):
    """SBG_F32X2 (hi and lo, both with halos) with the surface sink on the
    two-row kernel, one and two persistent CTAs per SM and all that fit: the
    same hi and lo parts as the one-thread-per-voxel kernel (read back as
    hi + lo in FP64, which is exact)."""
    phi, phys, u0 = make_case((64, 60, 56), 1, 0.5, (0, 1), 14)
    p = make_params(phys)
    g = Grid(phi, block=block)
    a = State(g, 1, "f32x2").set_kernel("plain").set_all(u0).step(p, 29).get_all()
    for per_sm in (1, 2, 0):
        b = State(g, 1, "f32x2").set_kernel("async", ctas_per_sm=per_sm).set_all(u0).step(p, 29).get_all()
        np.testing.assert_array_equal(a, b)
        # the streaming kernel's compensated form (hi and lo rows at the same offsets)
        c = State(g, 1, "f32x2").set_kernel("stream", ctas_per_sm=per_sm).set_all(u0).step(p, 29).get_all()
        np.testing.assert_array_equal(a, c)
