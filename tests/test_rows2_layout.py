"""Host-side checks of the two-row step kernel's thread layout (the mapping
of `k_step_rows2` restated): every voxel of a 1024-voxel group belongs to
exactly one thread's row pair, every halo slot is written and read by one
thread only and lies inside the halo buffer, a quarter-warp's 16-byte row
loads touch each shared-memory bank once, and the shared memory per CTA
gives the CTA counts per SM the launcher asks for."""
import pytest

THREADS = 128
GROUP = 1024
SMEM_SM = 228 * 1024  # bytes of shared memory per SM the launcher plans with, 1 KB of it reserved per CTA


def layout(B):
    B3 = B ** 3
    G = GROUP // B3          # blocks per group
    TPB = B3 // 8            # threads per block
    ZB = (B // 2) * B * B    # row b = row a + ZB
    HB = (B // 2) * B        # row b's halo slot = row a's + HB
    face = lambda j, f: (j * 6 + f) * B * B  # noqa: E731
    rows = []
    for tid in range(THREADS):
        j, r = divmod(tid, TPB)
        x0 = 0 if B == 4 else (r & 1) * 4
        rr = r if B == 4 else r >> 1
        y, z0 = rr % B, rr // B
        la = (z0 * B + y) * B + x0
        hxm, hxp = x0 == 0, x0 + 3 == B - 1
        hym, hyp = y == 0, y == B - 1
        hzm, hzp = z0 == 0, z0 + B // 2 == B - 1
        slots = []
        if hxm:
            slots += [face(j, 0) + z0 * B + y + q * HB for q in (0, 1)]
        if hxp:
            slots += [face(j, 1) + z0 * B + y + q * HB for q in (0, 1)]
        for hit, f in ((hym, 2), (hyp, 3)):
            if hit:
                slots += [face(j, f) + z0 * B + x0 + q * HB + e for q in (0, 1) for e in range(4)]
        if hzm:
            slots += [face(j, 4) + y * B + x0 + e for e in range(4)]
        if hzp:
            slots += [face(j, 5) + y * B + x0 + e for e in range(4)]
        rows.append(dict(j=j, la=la, va=j * B3 + la, x0=x0, y=y, z0=z0, slots=slots))
    return dict(B3=B3, G=G, ZB=ZB, HB=HB, kHalo=G * 6 * B * B, rows=rows)


@pytest.mark.parametrize("B", [4, 8])
def test_each_voxel_of_a_group_has_one_owner(B):
    L = layout(B)
    owned = []
    for t in L["rows"]:
        for q in (0, 1):
            owned += [t["va"] + q * L["ZB"] + e for e in range(4)]
    assert sorted(owned) == list(range(GROUP))


@pytest.mark.parametrize("B", [4, 8])
def test_halo_slots_are_private_and_in_bounds(B):
    """Each thread writes (by cp.async or a plain store) and later reads only
    its own slots, so the halo needs no CTA barrier; together the slots fill
    the six B x B faces of every block of the group exactly once."""
    L = layout(B)
    slots = [s for t in L["rows"] for s in t["slots"]]
    assert len(slots) == len(set(slots))
    assert min(slots) >= 0 and max(slots) < L["kHalo"]
    assert sorted(slots) == list(range(L["kHalo"]))


@pytest.mark.parametrize("B", [4, 8])
def test_quarter_warp_row_loads_are_conflict_free(B):
    """A 16-byte shared load is served per quarter-warp (8 threads, 128
    bytes): the eight rows must start in eight different 16-byte bank
    groups, for row a and for row b."""
    L = layout(B)
    for base in range(0, THREADS, 8):
        for q in (0, 1):
            starts = [(4 * (t["va"] + q * L["ZB"])) % 128 for t in L["rows"][base:base + 8]]
            assert sorted(starts) == list(range(0, 128, 16)), (B, base, q, starts)


@pytest.mark.parametrize("B", [4, 8])
def test_tile_neighbours_stay_in_the_block(B):
    """Neighbours not taken from the halo are inside the thread's own block of
    the stage tile: x within the row, y within the block, row a's z+ and row
    b's z- between the two rows."""
    L = layout(B)
    for t in L["rows"]:
        for q in (0, 1):
            z = t["z0"] + q * (B // 2)
            if t["x0"] > 0:
                assert t["x0"] - 1 >= 0
            if t["x0"] + 3 < B - 1:
                assert t["x0"] + 4 <= B - 1
            if q == 0:
                assert z + 1 <= B - 1       # row a's z+ neighbour is in the tile
            else:
                assert z - 1 >= 0           # row b's z- neighbour is in the tile


@pytest.mark.parametrize("B,NH,AH,wsm,want,expect", [
    (4, 1, True, False, 10, 10), (4, 1, True, True, 10, 7), (8, 1, True, False, 10, 10),
    (4, 2, True, False, 5, 5), (8, 2, True, False, 5, 5), (4, 1, False, False, 7, 7),
])
def test_shared_memory_fits_the_planned_ctas(B, NH, AH, wsm, want, expect):
    """Two ring stages of NH arrays, one or two halo buffers per array, the
    optional row-weight buffer and the stage barriers: the CTAs per SM that
    fit, capped at the launcher's register-based wish."""
    L = layout(B)
    S = 2
    floats = S * NH * GROUP + (2 if AH else 1) * NH * L["kHalo"] + (2 * GROUP if wsm else 0)
    smem = floats * 4 + S * 8
    fit = SMEM_SM // (smem + 1024)
    assert min(want, fit) == expect
    if NH == 2 and B == 4:
        assert smem <= 41 * 1024 and fit == 5
