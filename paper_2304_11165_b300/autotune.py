"""Autotuner for the step kernel: block edge, kernel variant and persistent
CTAs per SM.

For a set of geometries (one grid or a batch) it builds the grid at each
block edge, times a few steps of every candidate kernel configuration with
CUDA events on the current stream, and picks the fastest per active-voxel
update (the block edge trades block fill against per-block overhead; the
variant trades registers against latency hiding: the streaming kernel's rows
read through L1 (4^3 blocks; also over the batch solver's work lists), or the
ring kernels' halo loads when the group comes up, prefetched a group ahead in
registers, or copied a group ahead with cp.async).  Results are cached in a
JSON file keyed by GPU name, state dtype, species count and a fill bucket
(the fraction of 8^3-block slots that are pore voxels, in steps of 0.1), so
a second solve of a similar geometry skips the timing.

The knob of "blocks per CTA" is the persistent kernels' work unit here: a
CTA walks groups of 512 or 1024 voxels (one 8^3 block, eight or sixteen 4^3
blocks) and as many CTAs per SM as fit stay resident, so the tuned knobs are
the block edge, the kernel variant and the resident CTAs per SM (0 = all that
fit, or a fixed smaller number).

The cache path is $SBG_AUTOTUNE_CACHE, or ~/.cache/sbg/autotune.json.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from .api import Grid, State, make_params

DEFAULT_CANDIDATES = [(4, "stream", 0), (4, "pipelined", 0), (4, "prefetch", 0), (4, "async", 0), (8, "pipelined", 0),
                      (8, "prefetch", 0), (8, "async", 0), (4, "pipelined", 4), (8, "pipelined", 4)]


def cache_path() -> str:
    return os.environ.get("SBG_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sbg", "autotune.json"))


def _load_cache():
    try:
        return json.load(open(cache_path()))
    except (OSError, ValueError):
        return {}


def _save_cache(cache):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    except OSError:
        pass


def _grid(phis, block):
    return Grid.batch(phis, block=block) if len(phis) > 1 else Grid(phis[0], block=block)


def cache_key(device_name: str, dtype: str, nspecies: int, fill: float) -> str:
    """Key of a tuning result: the GPU, the state type, the species count and
    the fill of 8^3 blocks rounded to 0.1 (geometries of similar fill tune
    alike)."""
    return "%s|%s|%d|fill%.1f" % (device_name, dtype, int(nspecies), round(float(fill), 1))


def pick_best(table):
    """The candidate with the least time per active-voxel update (the first of equals)."""
    return min(table, key=lambda r: r["ns_per_voxel_update"])


def time_candidate(phis, grids, phys, dtype, candidate, steps, stream):
    """ns per active-voxel update of one (block, variant, ctas_per_sm) candidate:
    a zero field (which costs the same as any) stepped `steps` times after 8
    warm-up steps, timed with CUDA events on `stream`."""
    block, variant, ctas = candidate
    ns = int(phys.nspecies)
    params = make_params(phys)
    g = grids.get(block) or grids.setdefault(block, _grid(phis, block))
    st = State(g, ns, dtype).set_kernel(variant, ctas)
    for gi, phi in enumerate(phis):
        for s in range(ns):
            st.set(np.zeros(phi.shape, np.float32), species=s, geom=gi, stream=stream)
    st.step(params, 8, stream=stream)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    st.step(params, steps, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    st.close()
    return a.elapsed_time(b) * 1e6 / (steps * g.n_active * ns)


def tune(phis, phys, dtype: str = "f32x2", candidates=None, steps: int = 32, use_cache: bool = True,
         stream=None, timer=None):
    """Returns (best, table): best = dict(block, variant, ctas_per_sm, ns_per_voxel_update),
    table = every candidate's timing (None on a cache hit).  `phys` supplies the
    step parameters (dt, D, faces).  `timer(candidate)` -> ns per update
    replaces the GPU timing (time_candidate) when given."""
    phis = list(phis)
    candidates = candidates or DEFAULT_CANDIDATES
    ns = int(phys.nspecies)
    g8 = _grid(phis, 8)
    fill = g8.n_active / max(1, g8.n_blocks * 512)
    key = cache_key(torch.cuda.get_device_name(), dtype, ns, fill)
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True), None
    stream = stream or torch.cuda.current_stream()
    grids = {8: g8}
    if timer is None:
        def timer(c):
            return time_candidate(phis, grids, phys, dtype, c, steps, stream)
    table = [dict(block=c[0], variant=c[1], ctas_per_sm=c[2], ns_per_voxel_update=float(timer(c)))
             for c in candidates]
    best = pick_best(table)
    if use_cache:
        cache[key] = best
        _save_cache(cache)
    return dict(best, cached=False), table
