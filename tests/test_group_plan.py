"""The grouped call's static tile schedule, computed on the host through
ftgemm_group_plan (no GPU): tile grids and k-blocks per problem, every tile
scheduled once, the longest-processing-time greedy's balance bound,
longest-K-first order, the raster inside a problem, and argument errors."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def ft():
    import paper_2305_01024_gb300.build as b
    b.build()
    import paper_2305_01024_gb300 as ft
    return ft


EPILOGUE_KB = 6  # a tile costs at least this many k-blocks in the schedule


def _grid(ft, m, n, k, dtype, level):
    # the data tile of C (ftgemm_tc_tile): 3 (bf16) or 5 (e4m3) rows and
    # columns of the 128 x 256 MMA tile carry checksums at level TILE, the
    # data columns rounded down to a multiple of 4
    dm, dn = ((125, 252) if dtype == ft.BF16 else (123, 248)) if level == ft.FT_TILE else (128, 256)
    kblk = 64 if dtype == ft.BF16 else 128
    return -(-m // dm), -(-n // dn), -(-k // kblk)


@pytest.mark.parametrize("dtype_name,level_name", [("BF16", "FT_TILE"), ("BF16", "FT_OFF"),
                                                   ("E4M3", "FT_TILE")])
def test_every_tile_once_with_its_k_blocks(ft, dtype_name, level_name):
    dtype, level = getattr(ft, dtype_name), getattr(ft, level_name)
    shapes = [(300, 500, 256), (2048, 96, 1024), (64, 64, 64), (777, 1531, 2049), (125, 252, 128),
              (123, 248, 128), (126, 253, 64)]
    tiles, start = ft.group_plan(shapes, dtype, level, ncta=7)
    want = set()
    for p, (m, n, k) in enumerate(shapes):
        tm, tn, kb = _grid(ft, m, n, k, dtype, level)
        want |= {(p, i, j, kb) for i in range(tm) for j in range(tn)}
    assert len(tiles) == len(want) and set(tiles) == want
    assert start[0] == 0 and start[-1] == len(tiles) and len(start) == 8
    assert all(a <= b for a, b in zip(start, start[1:]))


def _loads(tiles, start):
    cost = [max(t[3], EPILOGUE_KB) for t in tiles]
    return [sum(cost[start[c]:start[c + 1]]) for c in range(len(start) - 1)], max(cost)


def test_balance_bound_on_a_mixed_group(ft):
    # 512 problems with the mixed shapes of the grouped benchmark: greedy list
    # scheduling leaves no CTA more than one tile's cost above the least loaded
    u = synth.unit(synth.workload_seed("group512", 90), 3 * 512)
    m = 64 + 16 * np.floor(u[0::3] * 253).astype(int)
    n = 64 + 16 * np.floor(u[1::3] * 253).astype(int)
    k = 64 + 16 * np.floor(u[2::3] * 125).astype(int)
    shapes = list(zip(m.tolist(), n.tolist(), k.tolist()))
    tiles, start = ft.group_plan(shapes, ft.BF16, ft.FT_TILE, ncta=152)
    loads, cmax = _loads(tiles, start)
    assert max(loads) - min(loads) <= cmax
    assert max(loads) <= sum(loads) / len(loads) + cmax


def test_longest_k_first_and_stable(ft):
    shapes = [(500, 500, 128), (500, 500, 1024), (500, 500, 128), (500, 500, 512)]
    tiles, start = ft.group_plan(shapes, ft.BF16, ft.FT_TILE, ncta=5)
    ks = [shapes[t[0]][2] for t in tiles]
    for c in range(5):
        run = ks[start[c]:start[c + 1]]
        assert all(a >= b for a, b in zip(run, run[1:]))  # each CTA: longer K first
    # on one CTA the problem order is K descending, ties in the caller's order
    tiles1, _ = ft.group_plan(shapes, ft.BF16, ft.FT_TILE, ncta=1)
    order = []
    for t in tiles1:
        if t[0] not in order:
            order.append(t[0])
    assert order == [1, 3, 0, 2]


def test_raster_inside_a_problem(ft):
    # one CTA runs the whole problem in the kernel's raster: bands of 16 tile
    # rows, each band column by column, rows in order inside a column
    m, n = 40 * 125, 3 * 252
    tiles, _ = ft.group_plan([(m, n, 256)], ft.BF16, ft.FT_TILE, ncta=1)
    seq = [(t[1], t[2]) for t in tiles]
    want = []
    for first in range(0, 40, 16):
        rows = range(first, min(40, first + 16))
        want += [(r, c) for c in range(3) for r in rows]
    assert seq == want


def test_more_ctas_than_tiles(ft):
    tiles, start = ft.group_plan([(100, 100, 64)], ft.E4M3, ft.FT_OFF, ncta=4)
    assert tiles == [(0, 0, 0, 1)]
    assert sorted(start[c + 1] - start[c] for c in range(4)) == [0, 0, 0, 1]


def test_argument_errors(ft):
    with pytest.raises(ft.FtgemmError) as e:
        ft.group_plan([(64, 64, 64)], ft.F32, ft.FT_TILE)
    assert e.value.status == ft.ERR_UNSUPPORTED
    with pytest.raises(ft.FtgemmError) as e:
        ft.group_plan([(64, 64, 64)], ft.BF16, ft.FT_BLOCK)
    assert e.value.status == ft.ERR_UNSUPPORTED
    for bad in ([], [(0, 64, 64)], [(64, 64, -1)]):
        with pytest.raises(ft.FtgemmError) as e:
            ft.group_plan(bad, ft.BF16, ft.FT_TILE)
        assert e.value.status == ft.ERR_ARG
    with pytest.raises(ft.FtgemmError) as e:
        ft.group_plan([(64, 64, 64)], ft.BF16, ft.FT_TILE, ncta=0)
    assert e.value.status == ft.ERR_ARG
