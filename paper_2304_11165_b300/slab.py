"""Slab decomposition along x: the domain decomposition with one ghost layer
that the paper runs across GPUs (Sec. 2.4; scaling results in Sec. 3.6).

Rank k owns the x planes [x_bounds[k], x_bounds[k+1]) of the box
(``partition``: bounds on block boundaries balancing the active blocks,
computed by ``sbg_slab_partition``).  It builds the sub-box of its planes
plus one ghost plane on each side where another slab lies; the ghost planes
are Dirichlet faces of the sub-box (held: its steps leave them as they are),
and after every step each rank sends its first owned plane to the left
neighbour and its last owned plane to the right one, which write them into
their ghost planes (``sbg_state_set_xplane``).  A 7-point step reads nothing
else, so every owned voxel gets exactly its whole-box update.  On check steps
the FP64 reduction scalars of the owned voxels are summed (or, for min and
max, reduced) over the ranks.

This module is the host logic of that scheme (which plane goes where, the
local physics of a sub-box, which scalars combine how); the per-rank compute
is any ``engine`` with get_plane/set_plane/step/checks (``LibraryEngine``
runs the library's kernels on the rank's GPU), and the transport is any
``comm`` with ``exchange(peer, send, recv)`` and ``allreduce(array, op)``
(``TorchComm`` uses torch.distributed: NCCL between GPUs, gloo on CPUs).
There is no arithmetic of the method here.
"""
from __future__ import annotations

import ctypes
import dataclasses
from dataclasses import dataclass

import numpy as np

from . import _abi
from ._abi import check, load


def partition(phi, nparts: int, block: int = 4, eps_mask: float = 0.0) -> np.ndarray:
    """x bounds of `nparts` slabs of the dense [Nz, Ny, Nx] phi (host array)."""
    arr = np.ascontiguousarray(phi, dtype=np.float32)
    nz, ny, nx = arr.shape
    dims = (ctypes.c_int64 * 3)(nx, ny, nz)
    out = np.zeros(nparts + 1, dtype=np.int64)
    check(load().sbg_slab_partition(arr.ctypes.data_as(ctypes.c_void_p), dims, int(block), float(eps_mask),
                                    int(nparts), out.ctypes.data_as(ctypes.c_void_p)))
    return out


@dataclass
class Slab:
    """Rank `rank` of `nranks`: owned planes [x_lo, x_hi) of a box of nx planes."""
    rank: int
    nranks: int
    x_lo: int
    x_hi: int
    nx: int

    @classmethod
    def of(cls, x_bounds, rank: int):
        return cls(rank, len(x_bounds) - 1, int(x_bounds[rank]), int(x_bounds[rank + 1]), int(x_bounds[-1]))

    @property
    def ghost_lo(self) -> int:
        return 1 if self.rank > 0 else 0

    @property
    def ghost_hi(self) -> int:
        return 1 if self.rank < self.nranks - 1 else 0

    @property
    def sub_x0(self) -> int:
        """First plane of the sub-box in box coordinates."""
        return self.x_lo - self.ghost_lo

    @property
    def sub_nx(self) -> int:
        return self.x_hi - self.x_lo + self.ghost_lo + self.ghost_hi

    @property
    def first_owned(self) -> int:
        """Local x of the first owned plane."""
        return self.ghost_lo

    @property
    def last_owned(self) -> int:
        return self.ghost_lo + (self.x_hi - self.x_lo) - 1

    def sub_field(self, field):
        """The sub-box part of a dense [..., Nz, Ny, Nx] field."""
        return field[..., self.sub_x0:self.sub_x0 + self.sub_nx]

    def owned_field(self, sub):
        """The owned planes of a dense [..., Nz, Ny, sub_nx] sub-box field."""
        return sub[..., self.first_owned:self.last_owned + 1]

    def local_physics(self, phys):
        """The physics of the sub-box: the same coefficients, the ghost faces held
        (Dirichlet), the box's own x faces where the slab reaches them."""
        d = list(phys.dirichlet)
        if self.ghost_lo:
            d[0] = True
        if self.ghost_hi:
            d[1] = True
        dims = (self.sub_nx,) + tuple(phys.dims[1:])
        return dataclasses.replace(phys, dims=dims, dirichlet=tuple(d))

    def exchange_plan(self):
        """(peer, local plane to send, local ghost plane to receive into) per neighbour."""
        plan = []
        if self.ghost_lo:
            plan.append((self.rank - 1, self.first_owned, 0))
        if self.ghost_hi:
            plan.append((self.rank + 1, self.last_owned, self.sub_nx - 1))
        return plan


def exchange_ghosts(slab: Slab, engine, comm, nspecies: int):
    """After a step: every neighbour's owned boundary plane into this rank's
    ghost plane on that side, for every species."""
    for s in range(nspecies):
        for peer, send_x, recv_x in slab.exchange_plan():
            send = engine.get_plane(s, send_x)
            recv = engine.empty_plane()
            comm.exchange(peer, send, recv)
            engine.set_plane(s, recv_x, recv)


def exchange_ghosts_local(slabs, engines, nspecies: int):
    """The same exchange between slabs held in one process (all planes are read
    before any is written)."""
    moves = []
    for slab, eng in zip(slabs, engines):
        for peer, send_x, _ in slab.exchange_plan():
            recv_x = 0 if peer > slab.rank else slabs[peer].sub_nx - 1
            for s in range(nspecies):
                moves.append((peer, s, recv_x, eng.get_plane(s, send_x)))
    for peer, s, recv_x, plane in moves:
        engines[peer].set_plane(s, recv_x, plane)


def run(slab: Slab, engine, comm, nspecies: int, nsteps: int):
    """nsteps steps with a ghost exchange after each."""
    for _ in range(int(nsteps)):
        engine.step(1)
        exchange_ghosts(slab, engine, comm, nspecies)


# combination of the per-rank check scalars (SBG_NRED layout per species)
_SUM, _MIN, _MAX = "sum", "min", "max"


def global_checks(slab: Slab, engine, comm, nspecies: int):
    """The FP64 check scalars of the whole box from the ranks' owned voxels:
    mass and active count summed over the ranks, the inlet flux from the rank
    that owns x = 0, the outlet flux from the one that owns x = Nx - 1, the
    residual norm from the summed squares, min and max reduced, non-finite
    voxels flagged (the largest count of any rank)."""
    out = []
    for s in range(nspecies):
        mass, count = engine.owned_sum(s, slab.first_owned, slab.last_owned + 1)
        r = engine.checks(s)
        j_in = r[_abi.RED_JIN] if slab.rank == 0 else 0.0
        j_out = r[_abi.RED_JOUT] if slab.rank == slab.nranks - 1 else 0.0
        summed = comm.allreduce(np.array([mass, j_in, j_out, r[_abi.RED_RESIDUAL] ** 2, count]), _SUM)
        lo = comm.allreduce(np.array([r[_abi.RED_MIN]]), _MIN)
        hi = comm.allreduce(np.array([r[_abi.RED_MAX], r[_abi.RED_NONFINITE]]), _MAX)
        g = np.zeros(_abi.NRED)
        g[_abi.RED_MASS], g[_abi.RED_JIN], g[_abi.RED_JOUT] = summed[0], summed[1], summed[2]
        g[_abi.RED_RESIDUAL] = np.sqrt(summed[3])
        g[_abi.RED_NACTIVE] = summed[4]
        g[_abi.RED_MIN], g[_abi.RED_MAX], g[_abi.RED_NONFINITE] = lo[0], hi[0], hi[1]
        out.append(g)
    return out


class TorchComm:
    """Transport over torch.distributed (NCCL for CUDA tensors, gloo on CPU)."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.device = device

    def exchange(self, peer: int, send, recv):
        reqs = [self.dist.isend(send, peer), self.dist.irecv(recv, peer)]
        for r in reqs:
            r.wait()

    def allreduce(self, arr, op):
        t = self.torch.tensor(arr, dtype=self.torch.float64, device=self.device)
        ops = {_SUM: self.dist.ReduceOp.SUM, _MIN: self.dist.ReduceOp.MIN, _MAX: self.dist.ReduceOp.MAX}
        self.dist.all_reduce(t, op=ops[op])
        return t.cpu().numpy()


class LibraryEngine:
    """A rank's compute on its GPU: one grid and state of the sub-box (SBG_F32
    or SBG_F64), planes as CUDA tensors."""

    def __init__(self, slab: Slab, phi, phys, u0, dtype: str = "f32", block: int = 4, order: str = "planes",
                 variant: str = "auto", stream=None):
        import torch
        from .api import Grid, State, make_params
        self.torch = torch
        self.slab = slab
        self.stream = stream
        sub_phi = np.ascontiguousarray(slab.sub_field(phi))
        self.phys = slab.local_physics(phys)
        self.params = make_params(self.phys)
        self.grid = Grid(sub_phi, block=block, order=order, stream=stream)
        self.state = State(self.grid, int(phys.nspecies), dtype).set_kernel(variant)
        self.state.set_all(np.ascontiguousarray(slab.sub_field(np.asarray(u0).reshape(
            (int(phys.nspecies),) + tuple(np.shape(phi))))), stream=stream)
        self.ny, self.nz = sub_phi.shape[1], sub_phi.shape[0]
        self.tdtype = torch.float64 if dtype == "f64" else torch.float32
        self.code = _abi.SBG_F64 if dtype == "f64" else _abi.SBG_F32

    def empty_plane(self):
        return self.torch.empty((self.nz, self.ny), dtype=self.tdtype, device="cuda")

    def get_plane(self, s: int, x: int):
        out = self.empty_plane()
        check(load().sbg_state_get_xplane(self.grid.handle, self.state.handle, 0, s, int(x),
                                          ctypes.c_void_p(out.data_ptr()), self.code, 1, self._stream()))
        return out

    def set_plane(self, s: int, x: int, plane):
        plane = plane.contiguous()
        check(load().sbg_state_set_xplane(self.grid.handle, self.state.handle, 0, s, int(x),
                                          ctypes.c_void_p(plane.data_ptr()), self.code, 1, self._stream()))

    def step(self, n: int):
        self.state.step(self.params, int(n), stream=self.stream)

    def checks(self, s: int):
        r = self.state.reduce(self.params, stream=self.stream)[s]
        return np.array([r[k] for k in self.state._RED_KEYS])

    def owned_sum(self, s: int, x0: int, x1: int):
        return self.state.box_sum((x0, 0, 0), (x1, self.ny, self.nz), species=s, stream=self.stream)

    def owned(self):
        """The owned planes of every species as a dense float64 [S, Nz, Ny, n_owned] array."""
        return self.slab.owned_field(self.state.get_all())

    def _stream(self):
        from .api import _stream_handle
        return _stream_handle(self.stream)
