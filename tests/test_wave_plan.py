"""Work order of the wavefront step kernel (SBG_KERNEL_WAVE / WAVE4), checked
on the CPU through sbg_debug_wave_plan (host code, no device work).

A wavefront launch runs K steps: step s of a plane of blocks reads step s-1
of that plane and the planes beside it from a ring of R planes, and writes
its own ring slot, which held the plane R back.  Its CTAs take tickets (a
group of up to 16 blocks of one plane at one step) in the order listed, and a
ticket waits until the tickets it depends on are done.  The checks:

* the tickets cover every block of every plane once per step, in groups of at
  most 16 consecutive blocks of one plane;
* every ticket comes after every ticket it waits on, so the smallest
  unfinished ticket never waits (no deadlock, whatever the number of CTAs);
* the waits are enough: executing the tickets in random orders that respect
  only those waits, against a model of the rings, every read finds the plane
  it needs and every step's values come from the step before;
* parameters that cannot give such an order (R < L + 2, K < 1, L < 1) are
  rejected.
"""
import ctypes

import numpy as np
import pytest

from paper_2304_11165_b300 import _abi


def plan(counts, K, L, R, TB=16):
    lib = _abi.load()
    c = np.ascontiguousarray(counts, dtype=np.int32)
    n = ctypes.c_int64()
    rc = lib.sbg_debug_wave_plan(c.ctypes.data, len(c), K, L, R, TB, None, 0, ctypes.byref(n))
    if rc != _abi.SBG_OK:
        return rc, None
    out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    _abi.check(lib.sbg_debug_wave_plan(c.ctypes.data, len(c), K, L, R, TB, out.ctypes.data, n.value,
                                       ctypes.byref(n)))
    return rc, out[:n.value]


def deps(p, s, K, R, nplanes):
    """(step, plane) pairs a ticket at (s, p) waits on: step s-1 on the planes it
    reads, step s+1 on the planes that read the ring slot it overwrites."""
    out = []
    if s > 0:
        out += [(s - 1, q) for q in (p - 1, p, p + 1) if 0 <= q < nplanes]
    if s < K - 1:
        out += [(s + 1, q) for q in (p - R - 1, p - R, p - R + 1) if 0 <= q < nplanes]
    return out


CASES = [
    [5, 0, 17, 33, 16, 1, 0, 0, 40, 7],
    [1],
    [0, 0, 3],
    [16] * 12,
    list(np.random.default_rng(3).integers(0, 70, size=40)),
]


@pytest.mark.parametrize("counts", CASES)
@pytest.mark.parametrize("K,L,R,TB", [(2, 4, 7, 32), (4, 4, 7, 32), (2, 2, 5, 16), (2, 1, 3, 7), (3, 1, 4, 16),
                                      (4, 3, 5, 64), (1, 1, 3, 32)])
def test_tickets_cover_every_block_once_per_step(counts, K, L, R, TB):
    rc, t = plan(counts, K, L, R, TB)
    assert rc == _abi.SBG_OK
    starts = np.concatenate([[0], np.cumsum(counts)])
    for s in range(K):
        for p, n in enumerate(counts):
            mine = t[(t[:, 3] == s) & (t[:, 2] == p)]
            assert np.all((mine[:, 1] >= 1) & (mine[:, 1] <= TB))
            covered = np.concatenate([np.arange(a, a + b) for a, b in mine[:, :2]]) if len(mine) else np.array([])
            np.testing.assert_array_equal(np.sort(covered), np.arange(starts[p], starts[p + 1]))
    assert len(t) == K * sum((n + TB - 1) // TB for n in counts)


@pytest.mark.parametrize("counts", CASES)
@pytest.mark.parametrize("K,L,R", [(2, 4, 7), (4, 4, 7), (2, 2, 5), (2, 1, 3), (4, 3, 5)])
def test_every_ticket_comes_after_what_it_waits_on(counts, K, L, R):
    rc, t = plan(counts, K, L, R, 32)
    assert rc == _abi.SBG_OK
    nplanes = len(counts)
    last = {}
    for i, (_, _, p, s) in enumerate(t):
        last[(s, p)] = i
    for i, (_, _, p, s) in enumerate(t):
        for d in deps(p, s, K, R, nplanes):
            if counts[d[1]] == 0:
                continue
            assert last[d] < i, (i, (s, p), d)


@pytest.mark.parametrize("counts", [CASES[0], CASES[3]])
@pytest.mark.parametrize("K,L,R", [(2, 4, 7), (4, 2, 5), (3, 1, 3)])
def test_waits_suffice_for_the_rings(counts, K, L, R):
    """Random executions that respect only the waits: each ticket, when it runs,
    must find in the ring every group of the planes p-1..p+1 at step s-1 (the
    input buffer for s = 0), and writes its own groups into ring slot p mod R."""
    rc, t = plan(counts, K, L, R)
    assert rc == _abi.SBG_OK
    nplanes = len(counts)
    groups = {}
    for i, (b0, n, p, s) in enumerate(t):
        groups.setdefault((s, p), []).append(i)
    rng = np.random.default_rng(0)
    for trial in range(6):
        done = np.zeros(len(t), bool)
        ring = [dict() for _ in range(K - 1)]  # (slot, first block) -> plane written there
        pending = set(range(len(t)))
        while pending:
            ready = [i for i in pending
                     if all(done[j] for d in deps(t[i, 2], t[i, 3], K, R, nplanes) for j in groups.get(d, []))]
            assert ready, "no ticket can run"
            i = ready[rng.integers(len(ready))]
            b0, n, p, s = t[i]
            if s > 0:
                for q in (p - 1, p, p + 1):
                    if 0 <= q < nplanes:
                        for j in groups.get((s - 1, q), []):
                            assert ring[s - 1].get((q % R, t[j, 0])) == q, (trial, (s, p), q)
            if s < K - 1:
                ring[s][(p % R, b0)] = p
            done[i] = True
            pending.remove(i)


@pytest.mark.parametrize("K,L,R,TB", [(2, 2, 3, 16), (2, 1, 2, 16), (0, 1, 3, 16), (2, 0, 3, 16), (4, 3, 4, 16),
                                      (2, 4, 7, 0)])
def test_orders_that_could_deadlock_are_rejected(K, L, R, TB):
    rc, _ = plan([4, 9, 20, 1], K, L, R, TB)
    assert rc == _abi.SBG_ERR_INVALID_ARG
