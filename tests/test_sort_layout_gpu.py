"""The tile sort's order inside each tile, cell by cell.

Within a tile of C cells whose smallest cell count is R, the sorted slots
hold, in order:
  - R full layers: layer r lists every cell once, in the tile's cell order;
  - L depth layers of the tail: layer d lists, in cell order, the cells with
    more than R + d particles (2D3V: L = 3; 3D3V: L = 0);
  - the rest: each cell's particles beyond R + L, cell by cell, dealt into S
    interleaved runs when there are at least 64 S of them (2D3V: S = 8;
    3D3V: S = 4): the i-th goes to run i mod S, runs in order, each holding
    T / S or T / S + 1 of them (the first T mod S runs one more).
The cell order of a tile is row-major with x fastest; 3D3V tiles 16 cells
wide take their rows in the order 0, 2, 1, 3 of each group of four.

The particles of one cell are interchangeable (their ranks come from atomics),
so the cells of the sorted slots are fixed by the counts alone: the test
rebuilds that sequence from the sorted particles' cells and compares it with
the GPU's, slot by slot, after the first sort of an upload (global scatter)
and after sorts of a layout still in its last sort's slots (tile by tile,
meshes of 608 tiles or more), before and after hot particles move.
"""
import numpy as np
import pytest

import workloads as W
from pichelp import make_pair

pytestmark = pytest.mark.gpu

NO_SORT = 1 << 30  # steps between automatic sorts: none in these runs


def expected_local_cells(counts, layers, runs):
    """Local cell of each slot of one tile, from its per-cell counts."""
    C = len(counts)
    R = int(counts.min())
    ex = counts - R
    parts = [np.arange(C)] * R
    parts += [np.nonzero(ex > d)[0] for d in range(layers)]
    rest = np.repeat(np.arange(C), np.maximum(ex - layers, 0))
    T = len(rest)
    if T >= 64 * runs:
        i = np.arange(T)
        m, q = i % runs, i // runs
        pos = m * (T // runs) + np.minimum(m, T % runs) + q
        dealt = np.empty(T, np.int64)
        dealt[pos] = rest
        rest = dealt
    parts.append(rest)
    return np.concatenate(parts).astype(np.int64)


def tile_and_local(p, tile):
    ix, iy = p["ix"].astype(np.int64), p["iy"].astype(np.int64)
    tx, ty = tile[0], tile[1]
    if len(tile) == 2:
        return (iy // ty, ix // tx), (iy % ty) * tx + ix % tx
    tz = tile[2]
    iz = p["iz"].astype(np.int64)
    ly = iy % ty
    if tx == 16 and ty >= 4:
        ly = (ly & ~3) | ((ly & 1) << 1) | ((ly >> 1) & 1)
    return (iz // tz, iy // ty, ix // tx), ((iz % tz) * ty + ly) * tx + ix % tx


def check_layout(sim, s, tile, dims, layers, runs):
    p = sim.get_particles(s)
    assert np.all(p["ix"] >= 0), "a sort drops removed particles"
    coords, local = tile_and_local(p, tile)
    nt = [(d + t - 1) // t for d, t in zip(dims, tile)]
    if len(tile) == 2:
        key = coords[0] * nt[0] + coords[1]
    else:
        key = (coords[0] * nt[1] + coords[1]) * nt[0] + coords[2]
    assert np.all(np.diff(key) >= 0), "slots grouped by tile, tiles in order"
    C = int(np.prod(tile))
    bounds = np.flatnonzero(np.diff(key)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [len(key)]])
    checked = 0
    for a, b in zip(starts, ends):
        got = local[a:b]
        counts = np.bincount(got, minlength=C)
        want = expected_local_cells(counts, layers, runs)
        assert np.array_equal(got, want), (int(key[a]), got[:40], want[:40])
        checked += 1
    return checked


def test_sort_layout_2d_global_and_tiled():
    wl = W.small_case(nx=512, ny=256, ppc=8, u_th=0.3, a0=3.0)
    tile = (16, 8)
    sim, _, _ = make_pair(wl, sort_every=NO_SORT, tile=tile)
    try:
        assert (512 // 16) * (256 // 8) >= 4 * 152
        sim.sort()                                   # after the upload: global scatter
        n = check_layout(sim, 0, tile, (wl.nx, wl.ny), 3, 8)
        assert n == 1024
        sim.sort()                                   # in its last sort's slots: tile by tile
        check_layout(sim, 0, tile, (wl.nx, wl.ny), 3, 8)
        sim.step(6)                                  # hot particles leave their cells and tiles
        sim.sort()
        check_layout(sim, 0, tile, (wl.nx, wl.ny), 3, 8)
    finally:
        sim.close()


def test_sort_layout_2d_dealt_rest():
    # 32 tiles of 32 x 16 (the global scatter); 24 per cell, mixed by hot
    # motion, leave more than 64 S particles per tile after the depth layers
    wl = W.small_case(nx=256, ny=64, ppc=24, u_th=0.3, a0=3.0)
    tile = (32, 16)
    sim, _, _ = make_pair(wl, sort_every=NO_SORT, tile=tile)
    try:
        sim.step(10)
        sim.sort()
        p = sim.get_particles(0)
        _, local = tile_and_local(p, tile)
        check_layout(sim, 0, tile, (wl.nx, wl.ny), 3, 8)
        # at least one tile's rest was dealt (the case this test is for)
        key = (p["iy"] // 16) * (256 // 32) + p["ix"] // 32
        dealt = 0
        for t in np.unique(key):
            c = np.bincount(local[key == t], minlength=512)
            dealt += int(np.maximum(c - c.min() - 3, 0).sum() >= 64 * 8)
        assert dealt > 0
    finally:
        sim.close()


def test_sort_layout_3d_global_and_tiled():
    wl = W.small_case3(nx=256, ny=32, nz=32, ppc=2, u_th=0.3, a0=3.0)
    tile = (16, 4, 4)
    sim, _, _ = make_pair(wl, sort_every=NO_SORT, tile=tile)
    try:
        assert (256 // 16) * (32 // 4) * (32 // 4) >= 4 * 152
        sim.sort()
        n = check_layout(sim, 0, tile, (wl.nx, wl.ny, wl.nz), 0, 4)
        assert n == 1024
        sim.sort()
        check_layout(sim, 0, tile, (wl.nx, wl.ny, wl.nz), 0, 4)
        sim.step(5)
        sim.sort()
        check_layout(sim, 0, tile, (wl.nx, wl.ny, wl.nz), 0, 4)
    finally:
        sim.close()
