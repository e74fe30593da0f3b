"""The slab decomposition's host logic (paper_2304_11165_b300.slab: partition,
local physics of a sub-box, ghost-plane exchange after every step, the
combination of the check scalars over the ranks) run as gloo ranks on CPU,
each rank computing its sub-box with the FP64 oracle as its engine.  The
owned planes of all ranks after the run must equal the whole-box oracle run
bit for bit (every owned voxel sees exactly its whole-box neighbourhood), and
the combined checks must equal the whole-box reductions (mass and residual up
to the order of the FP64 sums)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTEPS = 30


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem():
    sys.path.insert(0, ROOT)
    from workloads import Physics, random_blob_phi
    dims = (29, 17, 13)
    phi = random_blob_phi(dims, 61, porosity=0.6, ell=1.6)
    phys = Physics(dims=dims, dt=0.05, nspecies=2, D=(1.0, 0.5), decay=(0.01, 0.1), k_surf=0.4,
                   dirichlet=(True, False, False, False, True, False), face_value=(1.0, 0, 0, 0, 0, 0))
    u0 = np.random.default_rng(61).uniform(0, 1, size=(2,) + phi.shape)
    u0[0, :, :, 0] = 1.0
    return phi, phys, u0


class OracleEngine:
    """A rank's compute on the host: the oracle on the rank's sub-box."""

    def __init__(self, slab, phi, phys, u0):
        import oracle
        self.P = oracle.Problem(np.ascontiguousarray(slab.sub_field(phi)), slab.local_physics(phys))
        self.u = self.P.shape_state(np.ascontiguousarray(slab.sub_field(u0)))
        self.nz, self.ny = phi.shape[0], phi.shape[1]

    def empty_plane(self):
        return torch.zeros((self.nz, self.ny), dtype=torch.float64)

    def get_plane(self, s, x):
        return torch.from_numpy(np.ascontiguousarray(self.u[s][:, :, x]))

    def set_plane(self, s, x, plane):
        act = self.P.active[:, :, x] > 0
        self.u[s][:, :, x][act] = plane.numpy()[act]

    def step(self, n):
        self.u = self.P.run(self.u, n)

    def checks(self, s):
        from paper_2304_11165_b300 import _abi
        r = self.P.reduce(self.u)[s]
        out = np.zeros(_abi.NRED)
        out[_abi.RED_MASS], out[_abi.RED_JIN], out[_abi.RED_JOUT] = r["mass"], r["J_in"], r["J_out"]
        out[_abi.RED_RESIDUAL], out[_abi.RED_NACTIVE] = r["residual"], r["n_active"]
        vals = self.u[s][self.P.active > 0]
        out[_abi.RED_MIN], out[_abi.RED_MAX] = vals.min(), vals.max()
        out[_abi.RED_NONFINITE] = float(np.count_nonzero(~np.isfinite(vals)))
        return out

    def owned_sum(self, s, x0, x1):
        return self.P.box_sum(self.u, (x0, 0, 0), (x1, self.ny, self.nz), s)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    from paper_2304_11165_b300 import slab as sl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        phi, phys, u0 = problem()
        bounds = sl.partition(phi, world, block=4)
        slab = sl.Slab.of(bounds, rank)
        eng = OracleEngine(slab, phi, phys, u0)
        comm = sl.TorchComm()
        sl.run(slab, eng, comm, 2, NSTEPS)
        checks = sl.global_checks(slab, eng, comm, 2)
        out.put((rank, bounds.tolist(), slab.owned_field(eng.u), [c.tolist() for c in checks]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_over_gloo_ranks_reproduce_the_whole_box_bit_for_bit(world):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    phi, phys, u0 = problem()
    bounds = got[0][1]
    assert bounds[0] == 0 and bounds[-1] == phys.dims[0] and all(b % 4 == 0 for b in bounds[1:-1])
    assert all(g[1] == bounds for g in got)
    whole = oracle.Problem(phi, phys).run(u0, NSTEPS)
    joined = np.concatenate([g[2] for g in got], axis=-1)
    np.testing.assert_array_equal(joined, whole)
    ref = oracle.Problem(phi, phys).reduce(whole)
    for s in range(2):
        c = np.array(got[0][3][s])
        for g in got[1:]:
            np.testing.assert_array_equal(np.array(g[3][s]), c)  # every rank holds the same combination
        from paper_2304_11165_b300 import _abi
        assert c[_abi.RED_NACTIVE] == ref[s]["n_active"]
        assert abs(c[_abi.RED_MASS] - ref[s]["mass"]) <= 1e-12 * abs(ref[s]["mass"])
        assert c[_abi.RED_JIN] == ref[s]["J_in"] and c[_abi.RED_JOUT] == ref[s]["J_out"]
        assert abs(c[_abi.RED_RESIDUAL] - ref[s]["residual"]) <= 1e-12 * ref[s]["residual"]
        act = oracle.Problem(phi, phys).active > 0
        assert c[_abi.RED_MIN] == whole[s][act].min() and c[_abi.RED_MAX] == whole[s][act].max()


def test_partition_balances_active_blocks():
    """Bounds on block boundaries, every slab at least one block column, and
    active-block counts within one column's worth of the even share."""
    sys.path.insert(0, ROOT)
    from paper_2304_11165_b300 import slab as sl
    phi, _, _ = problem()
    big = np.concatenate([phi] * 4, axis=2)  # 116 planes
    for n in (1, 2, 3, 5, 29):
        b = sl.partition(big, n, block=4)
        assert b[0] == 0 and b[-1] == big.shape[2] and np.all(np.diff(b) >= 4) and np.all(b[1:-1] % 4 == 0)
    # an empty left half: the active blocks all lie right of x = 64, the cut follows them
    lop = np.where(np.arange(128)[None, None, :] < 64, -1.0, 1.0).astype(np.float32) * np.ones((8, 8, 1), np.float32)
    b = sl.partition(lop, 2, block=4)
    assert b.tolist() == [0, 96, 128]
    with pytest.raises(Exception):
        sl.partition(lop, 33, block=4)  # more slabs than block columns
