"""The single-pass kernel's row schedule (csrc/lbm_step.cuh), emulated on the
CPU: one barrier per iteration is enough only if every stage reads rows that
an earlier iteration wrote and that no stage overwrote since, and no ring slot
read in an iteration is written in the same iteration.  Checked for the rows
per iteration the kernel is built with (2) and the alternative (4), with the
ring depths parsed from the kernel source, over row segments of every kind
the grids produce (fixed chunks and the balanced grid's arbitrary ranges),
with a wall top (mirror rows) and a periodic one."""
import os
import random
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _depths(rr):
    src = open(os.path.join(ROOT, "paper_1512_01977_gb300", "csrc", "lbm_step.cuh")).read()
    line = re.search(r"static constexpr int DP = [^;]*;", src).group(0)
    out = {}
    for name, expr in re.findall(r"(D[PDJU]) = (RR <= 2 \? \d+ : \d+|\d+)", line):
        m = re.match(r"RR <= 2 \? (\d+) : (\d+)", expr)
        out[name] = (int(m.group(1)) if rr <= 2 else int(m.group(2))) if m else int(expr)
    return out


def _mirror_top(j, nr):
    # rows beyond the top wall: nr + m <-> nr - 1 - m (single reflection)
    return 2 * nr - 1 - j


def _check_segment(nr, j0, jend, periodic, rr, d):
    lag = rr + 2
    depth = {"psi": d["DP"], "psd": d["DD"], "rj": d["DJ"], "uf": d["DU"]}
    rings = {k: {} for k in depth}
    pb, it = j0 - 6, 0
    while pb - 3 * lag < jend:
        reads, writes = [], []
        for k in range(rr):  # stage L
            row = pb + k
            if j0 - 6 <= row < jend + 6:
                writes += [("psi", row), ("rj", row)]
        for k in range(rr):  # stage D
            row = pb - lag + k
            if j0 - 4 <= row < jend + 4:
                er = _mirror_top(row, nr) if (not periodic and row >= nr) else row
                reads += [("psi", er + q) for q in range(-2, 3)]
                writes.append(("psd", row))
        for k in range(rr):  # stage U
            row = pb - 2 * lag + k
            if j0 - 2 <= row < jend + 2:
                er = _mirror_top(row, nr) if (not periodic and row >= nr) else row
                reads += [("rj", er)] + [("psi", er + q) for q in (-1, 0, 1)]
                reads += [("psd", er + q) for q in range(-2, 3)]
                writes.append(("uf", row))
        for k in range(rr):  # stage C
            row = pb - 3 * lag + k
            if j0 <= row < jend:
                reads += [("rj", row)] + [("uf", row + q) for q in range(-2, 3)]
        for name, row in reads:
            got = rings[name].get(row % depth[name])
            assert got is not None and got[0] == row and got[1] < it, (name, row, got, nr, j0, jend, rr)
        written = {(name, row % depth[name]) for name, row in writes}
        for name, row in reads:
            assert (name, row % depth[name]) not in written, ("same-iteration clobber", name, row, nr, j0, jend, rr)
        for name, row in writes:
            rings[name][row % depth[name]] = (row, it)
        pb += rr
        it += 1


@pytest.mark.parametrize("rr", [2, 4])
def test_ring_schedule(rr):
    d = _depths(rr)
    assert 11 + 2 * rr <= d["DP"] and 4 + 2 * rr <= d["DD"] and 6 + 4 * rr <= d["DJ"] and 4 + 2 * rr <= d["DU"]
    for nr in (16, 17, 20, 31, 33, 64, 100, 257):
        for periodic in (False, True):
            for chunk in (1, 2, 3, 7, 16, 23, 64, 144):
                for j0 in range(0, nr, chunk):
                    _check_segment(nr, j0, min(j0 + chunk, nr), periodic, rr, d)
    rng = random.Random(1512)
    for _ in range(1500):
        nr = rng.choice([16, 18, 40, 129, 2048])
        j0 = rng.randrange(0, nr)
        _check_segment(nr, j0, rng.randrange(j0 + 1, nr + 1), rng.random() < 0.3, rr, d)


@pytest.mark.parametrize("ring,depth", [("DJ", 8), ("DD", 4), ("DP", 8), ("DU", 4)])
def test_too_shallow_rings_are_caught(ring, depth):
    """The emulation has teeth: the next smaller power-of-two depth of any
    ring (the kernel masks ring indices) breaks it."""
    d = _depths(2)
    shallow = dict(d, **{ring: depth})
    with pytest.raises(AssertionError):
        for nr in (16, 40, 129):
            for periodic in (False, True):
                for j0 in range(0, nr, 16):
                    _check_segment(nr, j0, min(j0 + 16, nr), periodic, 2, shallow)



def _items(tz, rr, mapping):
    """Per stage, the (thread, row offset, first column) of every active item of
    the two-column march for strip width tz, as the kernel maps thread ids."""
    widths = {"L": tz + 12, "D": tz + 8, "U": tz + 4, "C": tz}
    nt = (rr * (tz + 12) // 2 + 31) // 32 * 32
    out = {}
    for st, w in widths.items():
        h = w // 2
        got = []
        for tid in range(nt):
            if mapping == "rows":
                row, col, on = tid >> 6, 2 * (tid & 63), (tid & 63) < h
            else:
                row, col, on = tid // h, 2 * (tid % h), tid < rr * h
            if on:
                got.append((tid, row, col))
        out[st] = (got, h)
    return out, nt


@pytest.mark.parametrize("tz,mapping", [(112, "rows"), (112, "packed"), (64, "packed"), (96, "packed")])
def test_item_mapping_covers_each_pair_once(tz, mapping):
    """Every (row, column pair) of every stage has exactly one thread, for the
    warp-row mapping the kernel uses with 112-column strips (128 threads, rows of
    at most 64 pairs on two whole warps each) and the packed mapping otherwise;
    with the warp-row mapping no warp holds items of two rows."""
    rr = 2
    src = open(os.path.join(ROOT, "paper_1512_01977_gb300", "csrc", "lbm_step.cuh")).read()
    assert "kWarpRows = S::NT == 128 && RR == 2 && HL <= 64;" in src  # the condition restated here
    items, nt = _items(tz, rr, mapping)
    if mapping == "rows":
        assert nt == 128 and (tz + 12) // 2 <= 64
    for st, (got, h) in items.items():
        assert sorted((r, c) for _, r, c in got) == [(r, 2 * c) for r in range(rr) for c in range(h)], st
        if mapping == "rows":
            for w in range(nt // 32):
                assert len({r for tid, r, _ in got if tid // 32 == w}) <= 1, (st, w)
