"""Differentiable rollout: torch.autograd.Function over the library's
checkpointed adjoint (sbg_forward_record / sbg_adjoint).

The forward advances the state N steps and records a checkpoint every K
steps; the backward recomputes each K-step segment from its checkpoint and
runs the hand-written adjoint kernel backwards over it.  Gradients: the
initial field (0 on Dirichlet-held and inactive voxels, whose values are not
free), D per species and the surface rate k, the last three accumulated in
FP64.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _abi
from ._abi import check, load
from .api import Grid, State, _stream_handle, make_params


class Tape:
    def __init__(self, handle):
        self.handle = handle
        self._lib = load()

    def info(self):
        b, n = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.sbg_tape_info(self.handle, ctypes.byref(b), ctypes.byref(n)))
        return {"device_bytes": b.value, "checkpoints": n.value}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sbg_tape_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def forward_record(state: State, params, nsteps: int, checkpoint_every: int, stream=None) -> Tape:
    h = ctypes.c_void_p()
    check(load().sbg_forward_record(state.grid.handle, state.handle, ctypes.byref(params), int(nsteps),
                                    int(checkpoint_every), _stream_handle(stream), ctypes.byref(h)))
    return Tape(h)


def adjoint(tape: Tape, lam: State, stream=None):
    """lam: in dL/du^N, out dL/du^0.  Returns [dL/dD_0, dL/dD_1, dL/dk]."""
    g = np.zeros(3)
    check(load().sbg_adjoint(lam.grid.handle, tape.handle, lam.handle, g.ctypes.data_as(ctypes.c_void_p),
                             _stream_handle(stream)))
    return g


def _dense_get(state: State, like: torch.Tensor) -> torch.Tensor:
    out = torch.zeros_like(like)
    for s in range(state.nspecies):
        state.get(s, out=out[s])
    return out


class SbgRollout(torch.autograd.Function):
    """u^N = rollout(c0, D, k).

    c0: dense [S, Nz, Ny, Nx] CUDA tensor (float32 or float64; selects the
    state dtype); D: tensor [S]; k: 0-d tensor.  `grid`, `phys` (a
    workloads.Physics-like object), `nsteps` and `checkpoint_every` are not
    differentiated."""

    @staticmethod
    def forward(ctx, c0, D, k, grid: Grid, phys, nsteps: int, checkpoint_every: int):
        dtype = "f64" if c0.dtype == torch.float64 else "f32"
        ns = c0.shape[0]
        Dl = [float(v) for v in D.detach().cpu().reshape(-1).tolist()] + [0.0, 0.0]
        phys_k = dataclasses.replace(phys, D=(Dl[0], Dl[1]), k_surf=float(k.detach().cpu()))
        params = make_params(phys_k)
        st = State(grid, ns, dtype).set_all(c0.detach().contiguous())
        tape = forward_record(st, params, nsteps, checkpoint_every)
        uN = _dense_get(st, c0)
        ctx.tape, ctx.grid, ctx.ns, ctx.dtype, ctx.like = tape, grid, ns, dtype, c0
        return uN

    @staticmethod
    def backward(ctx, g_uN):
        lam = State(ctx.grid, ctx.ns, ctx.dtype).set_all(g_uN.detach().contiguous())
        grad = adjoint(ctx.tape, lam)
        dc0 = _dense_get(lam, ctx.like)
        dD = torch.tensor(grad[:ctx.ns], dtype=torch.float64)
        dk = torch.tensor(grad[2], dtype=torch.float64)
        return dc0, dD, dk, None, None, None, None


def rollout(c0, D, k, grid, phys, nsteps, checkpoint_every=64):
    return SbgRollout.apply(c0, D, k, grid, phys, nsteps, checkpoint_every)
