"""Simulated FRAP: effective diffusivity and tortuosity of a pore geometry
from the recovery of a bleached box (Sec. 3.3).

The pore run and a bulk-box run of the same edge lengths at the same D are
advanced by the step kernels, the box mass is recorded on the device between
steps (``sbg_frap_curve``), and the bulk curve is fitted to the pore curve
over a time scale s (``sbg_frap_fit``): the bulk curve at s D matches the
pore curve, so D_eff = s D and tau = D / D_eff (Eq. 2).

Each curve is normalised by its own equilibrium, F(t) = M_box(t) / (c n_box):
c is the mean of u over the active voxels (conserved in the closed box) and
n_box the number of active voxels in the box, so that both curves tend to 1
when the box's pores connect to the rest.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .api import Grid, State, frap_effective_D, make_params


@dataclass
class FrapResult:
    D_eff: float          # pore-space effective diffusivity s * D
    tau: float            # D / D_eff
    scale: float          # fitted time scale s
    rss: float            # residual sum of squares of the fit
    t: np.ndarray         # sample times of both curves
    F: np.ndarray         # normalised pore curve
    F_bulk: np.ndarray    # normalised bulk curve


def recovery(state: State, params, lo, hi, steps_per_sample: int, n_samples: int, geom: int = 0, stream=None):
    """(t, F) of the normalised recovery of the box lo <= (x, y, z) < hi,
    advancing ``state`` by ``steps_per_sample * n_samples`` steps
    (``sbg_frap_recovery``)."""
    t, F, _ = state.frap_recovery(params, lo, hi, steps_per_sample, n_samples, geom=geom, stream=stream)
    return t, F


def effective_D(phi, phys, u0, lo, hi, steps_per_sample: int, n_samples: int, dtype: str = "f32r",
                block: int = 4, s_lo: float = 1e-3, variant: str | None = None, stream=None) -> FrapResult:
    """FRAP estimate of D_eff for the pore space of ``phi`` (dense [Nz, Ny, Nx])
    under ``phys`` (closed box; species 0), bleaching lo <= (x, y, z) < hi of
    the initial field ``u0``; the bulk reference is the same box with every
    voxel in the pore space."""
    p = make_params(phys)
    curves = []
    for field in (phi, np.full(phi.shape, 1.0e3, np.float32)):
        g = Grid(field, block=block, stream=stream)
        st = State(g, 1, dtype)
        if variant is not None:
            st.set_kernel(variant)
        st.set(u0)
        curves.append(recovery(st, p, lo, hi, steps_per_sample, n_samples, stream=stream))
        st.close()
        g.close()
    (t, F), (_, Fb) = curves
    d_eff, tau, s, rss = frap_effective_D(t, F, t, Fb, float(phys.D[0]), s_lo, 1.0)
    return FrapResult(D_eff=d_eff, tau=tau, scale=s, rss=rss, t=t, F=F, F_bulk=Fb)
