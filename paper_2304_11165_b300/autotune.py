"""Autotuner for the step kernel: block edge, kernel variant and persistent
CTAs per SM.

For a set of geometries (one grid or a batch) it builds the grid at each
block edge, times a few steps of every candidate kernel configuration with
CUDA events on the current stream, and picks the fastest per active-voxel
update (the block edge trades block fill against per-block overhead; the
variant trades registers against latency hiding: halo loads when the group
comes up, prefetched a group ahead in registers, or copied a group ahead with
cp.async).  Results are cached in a
JSON file keyed by GPU name, state dtype, species count and a fill bucket
(the fraction of 8^3-block slots that are pore voxels, in steps of 0.1), so
a second solve of a similar geometry skips the timing.

The cache path is $SBG_AUTOTUNE_CACHE, or ~/.cache/sbg/autotune.json.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from .api import Grid, State, make_params

DEFAULT_CANDIDATES = [(4, "pipelined", 0), (4, "prefetch", 0), (4, "async", 0), (8, "pipelined", 0),
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


def tune(phis, phys, dtype: str = "f32x2", candidates=None, steps: int = 32, use_cache: bool = True,
         stream=None):
    """Returns (best, table): best = dict(block, variant, ctas_per_sm, ns_per_voxel_update),
    table = every candidate's timing.  `phys` supplies the step parameters
    (dt, D, faces); the state is a zero field, which costs the same as any."""
    phis = list(phis)
    candidates = candidates or DEFAULT_CANDIDATES
    ns = int(phys.nspecies)
    g8 = _grid(phis, 8)
    fill = g8.n_active / max(1, g8.n_blocks * 512)
    key = "%s|%s|%d|fill%.1f" % (torch.cuda.get_device_name(), dtype, ns, round(fill, 1))
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True), None
    params = make_params(phys)
    stream = stream or torch.cuda.current_stream()
    grids = {8: g8}
    table = []
    for block, variant, ctas in candidates:
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
        ns_per = a.elapsed_time(b) * 1e6 / (steps * g.n_active * ns)
        table.append(dict(block=block, variant=variant, ctas_per_sm=ctas, ns_per_voxel_update=ns_per))
        st.close()
    best = min(table, key=lambda r: r["ns_per_voxel_update"])
    if use_cache:
        cache[key] = best
        _save_cache(cache)
    return dict(best, cached=False), table
