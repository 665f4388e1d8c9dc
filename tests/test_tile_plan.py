"""CPU checks of the batched kernel's work plan (lbm_axi_tile_plan): every row
of every z-strip of every solve belongs to exactly one tile, tiles are grouped
by CTA, and the largest CTA load is within one tile of the average (the
guarantee of dealing the largest tiles first to the least-loaded CTA)."""
import numpy as np
import pytest

from paper_1512_01977_gb300 import inputs as I

FILL = 18  # rows of pipeline fill a tile costs beyond its own rows


@pytest.fixture(scope="module")
def lbm():
    from paper_1512_01977_gb300 import build, lbm as L

    build.build()
    L.lib()
    return L


def _check(lbm, sizes, strip, slots):
    tiles, first, makespan = lbm.lbm_axi_tile_plan(sizes, strip, slots)
    ncta = len(first) - 1
    assert 1 <= ncta <= slots and first[0] == 0 and first[-1] == len(tiles)
    assert np.all(np.diff(first) >= 1)
    seen = {}
    for s, t, j0, j1 in tiles:
        nz, nr = sizes[s]
        assert 0 <= t < -(-nz // strip) and 0 <= j0 < j1 <= nr
        seen.setdefault((s, t), []).append((j0, j1))
    for s, (nz, nr) in enumerate(sizes):
        for t in range(-(-nz // strip)):
            ranges = sorted(seen.pop((s, t)))
            assert ranges[0][0] == 0 and ranges[-1][1] == nr
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    assert not seen
    cost = tiles[:, 3] - tiles[:, 2] + FILL
    loads = np.add.reduceat(cost, first[:-1])
    assert makespan == loads.max()
    assert loads.max() <= cost.sum() / ncta + cost.max()
    return tiles, first, makespan


def test_single_large_solve_one_tile_per_cta(lbm):
    """The 4096 x 2048 bench grid on 608 slots (4 CTAs x 152 SMs): 43 strips of
    14 chunks, one tile of 146-147 rows per CTA -- no CTA marches two strips."""
    tiles, first, makespan = _check(lbm, [(4096, 2048)], 96, 608)
    assert len(tiles) == 602 and len(first) == 603
    assert makespan == 147 + FILL


@pytest.mark.parametrize("strip", [64, 96])
def test_batched_droplet_mix(lbm, strip):
    specs = I.batch_droplets(n=256, seed=4)
    _check(lbm, [(sp["nz"], sp["nr"]) for sp in specs], strip, 608)


@pytest.mark.parametrize("sizes,slots", [([(16, 16)], 608), ([(1, 16), (5, 17), (200, 40)], 3),
                                         ([(300, 2048)] * 3, 10), ([(70, 44)] * 50, 1)])
def test_small_and_skewed_cases(lbm, sizes, slots):
    _check(lbm, sizes, 96, slots)


def test_invalid_arguments(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.lbm_axi_tile_plan([(0, 16)], 96, 8)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_axi_tile_plan([(16, 16)], 96, 0)
