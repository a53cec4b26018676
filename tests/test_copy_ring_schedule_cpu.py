"""The copy schedule of the copy-fed smoother (k_smooth_tma.cu), checked on the
host.

The kernel brings the planes of a, x_in, b and d into rings of shared-memory
slots by bulk-tensor copies, grouped per plane step under one mbarrier each,
and its stages read those slots.  A slot overwritten while a stage still reads
it, a read of a plane whose copy was not waited for, or an mbarrier re-armed
before every thread has waited for its previous phase would give wrong results
or a wait that runs out.  This test replays the schedule the kernel follows,
with the ring sizes and the copy lead read from its source, for every segment
of small grids and every step kind, and checks those three properties.

Schedule (per segment [k0, k1) of a tile column, steps t = k0 - 3 .. k1 + 2):
- the group consumed at step c holds a and x_in of plane c + 1, b of plane
  c - 1 and d of plane c - 3 (only the planes some step reads); it is issued
  before the first step for c < k0 - 3 + PF - 1 (the group of step k0 - 4
  holds a and x_in of plane k0 - 3 only), else right after the block barrier
  of step c - PF + 1;
- every thread waits for the group of step t after the barrier of step t;
- step t reads a and x_in of plane t + 1 (the thread's own values for the next
  step), and the residual stage (plane t - 1: a, x_in, b), the black stage
  (plane t - 2: a) and the final stage (plane t - 3: a, d) when their plane is
  in the segment's range.
"""
import os
import re
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "paper_1812_08606_gb300", "csrc", "k_smooth_tma.cu")


def _constants():
    text = open(SRC).read()
    vals = {}
    for m in re.finditer(r"constexpr int ([^;]+);", text):
        for part in m.group(1).split(","):
            name, _, expr = part.partition("=")
            name, expr = name.strip(), expr.strip()
            if re.fullmatch(r"-?\d+", expr):
                vals[name] = int(expr)
    return vals


C = _constants()
PF, NMB = C["PF"], C["NMB"]
SLOTS = {"a": C["SA"], "x": C["SX"], "b": C["SB"], "d": C["SD"]}


def _group(c, k0, k1, nz, xzero, first, ax_only):
    """Planes the group consumed at step c copies, as (array, plane)."""
    rlo, rhi = max(0, k0 - 2), min(nz, k1 + 2)
    out = []
    pa, pb, pd = c + 1, c - 1, c - 3
    if 0 <= pa < nz and pa <= k1 + 2:
        out.append(("a", pa))
        if not xzero:
            out.append(("x", pa))
    if not ax_only and rlo <= pb < rhi:
        out.append(("b", pb))
    if not ax_only and not first and k0 <= pd < k1:
        out.append(("d", pd))
    return out


def _reads(t, k0, k1, nz, xzero, first):
    """Planes step t reads and uses, as (array, plane)."""
    rlo, rhi = max(0, k0 - 2), min(nz, k1 + 2)
    blo, bhi = max(0, k0 - 1), min(nz, k1 + 1)
    tend = k1 + 2
    out = []
    own = t + 1
    if 0 <= own < nz and own <= tend:     # committed at step t + 1 <= tend
        out.append(("a", own))
        if not xzero:
            out.append(("x", own))
    kr, kb, kf = t - 1, t - 2, t - 3
    if rlo <= kr < rhi:
        out += [("a", kr), ("b", kr)]
        if not xzero:
            out.append(("x", kr))
    if blo <= kb < bhi:
        out.append(("a", kb))
    if k0 <= kf < k1:
        out.append(("a", kf))
        if not first:
            out.append(("d", kf))
    return out


def _replay(k0, k1, nz, xzero, first):
    tstart, tend = k0 - 3, k1 + 2
    # issue times: a group issued "before the first step" gets time tstart - 0.5
    groups = {}
    for c in range(tstart - 1, tstart + PF - 1):
        groups[c] = (tstart - 0.5, _group(c, k0, k1, nz, xzero, first, c == tstart - 1))
    for t in range(tstart, tend + 1):
        c = t + PF - 1
        if c <= tend:
            groups[c] = (t, _group(c, k0, k1, nz, xzero, first, False))
    # every group from tstart - 1 to tend is issued once and waited once
    assert sorted(groups) == list(range(tstart - 1, tend + 1))
    # slot contents over time: list of (issue time, group, array, plane) per (array, slot)
    writes = {}
    for c, (when, planes) in groups.items():
        for arr, p in planes:
            writes.setdefault((arr, p % SLOTS[arr]), []).append((when, c, p))
    # mbarrier reuse: the group issued into mbarrier slot c % NMB must come after
    # the wait for the previous group there (waits of step u finish before the
    # barrier of step u + 1; the groups issued before the first step use
    # distinct mbarriers)
    for c, (when, _) in groups.items():
        prev = c - NMB
        if prev in groups:
            assert when >= prev + 1, ("mbarrier re-armed before its previous phase was waited", c, prev)
    waited = set()

    def check_read(t, arr, p):
        s = p % SLOTS[arr]
        hist = [w for w in writes.get((arr, s), []) if w[0] <= t]
        assert hist, ("read of a slot never written", arr, p, t)
        when, c, plane = max(hist)
        assert plane == p, ("slot holds another plane", arr, p, plane, t)
        assert when < t, ("slot written in the step that reads it", arr, p, t)
        assert c in waited, ("plane read before its group was waited for", arr, p, c, t)

    waited.add(tstart - 1)               # waited before the first step
    for arr, p in (("a", tstart), ("x", tstart)):
        if (arr == "x" and xzero) or not 0 <= p < nz:
            continue
        check_read(tstart - 0.25, arr, p)
    for t in range(tstart, tend + 1):
        waited.add(t)
        for arr, p in _reads(t, k0, k1, nz, xzero, first):
            check_read(t, arr, p)


@pytest.mark.parametrize("xzero,first", [(True, True), (False, False), (False, True)])
def test_copy_rings_hold_every_plane_a_step_reads(xzero, first):
    for nz in (8, 9, 12, 17, 24):
        for k0 in range(nz):
            for k1 in range(k0 + 1, nz + 1):
                _replay(k0, k1, nz, xzero, first)


def test_ring_sizes_read_from_the_kernel_source():
    assert PF >= 2 and NMB >= PF
    assert all(s & (s - 1) == 0 for s in SLOTS.values())   # slot = plane & (S - 1)


def test_a_smaller_ring_fails_the_replay(monkeypatch):
    """The replay catches an undersized ring: with one slot fewer for a (or
    mbarriers fewer than the copy lead) some read finds another plane."""
    monkeypatch.setitem(SLOTS, "a", PF + 3)
    with pytest.raises(AssertionError):
        for k1 in range(1, 17):
            _replay(0, k1, 16, False, False)
    monkeypatch.setitem(SLOTS, "a", C["SA"])
    monkeypatch.setattr(sys.modules[__name__], "NMB", PF - 1)
    with pytest.raises(AssertionError):
        _replay(0, 16, 16, False, False)


def test_copy_boxes_keep_the_16_byte_rule():
    """Every copy starts at an x coordinate whose byte offset is a multiple of
    16 (a and x_in, b: bx FTX - HX; d: bx FTX), every box row is a multiple of
    16 bytes, and every box dimension is at most 256 elements: the conditions a
    tiled bulk-tensor copy needs (an unaligned x origin is an illegal
    instruction on the GPU, which no check catches before the copy runs)."""
    rp, hx, tr = C["RP"], C["HX"], C["TR"]
    rw, dr = 2 * rp, tr + 2
    ftx, fty = rw - 2 * hx, tr - 4
    elem = 4   # FP32
    for bx in range(0, 64):
        assert ((bx * ftx - hx) * elem) % 16 == 0
        assert (bx * ftx * elem) % 16 == 0
    for width in (rw, ftx):
        assert (width * elem) % 16 == 0
    for dim in (rw, dr, tr, ftx, fty):
        assert 0 < dim <= 256
    # the slots the copies land in start on 128-byte boundaries
    assert (rp * dr * 8) % 128 == 0 and (rp * tr * 8) % 128 == 0 and ((ftx // 2) * fty * 8) % 128 == 0
