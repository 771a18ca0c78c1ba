"""The tile-by-tile sort (meshes of 608 tiles or more, four per SM): a
source in its last sort's slots is gathered one tile per CTA through shared
memory.  Runs that sort often, against the oracle:

  - 3D3V binned layout, 1024 tiles, re-binned every 8 steps while the
    co-moving window relabels the tile columns (the re-bins read ranges
    relabelled by txo, and the overflow range after the tiles);
  - 2D3V compact layout, 2048 tiles of 8 x 4 (the default for this mesh),
    sorted every 8 steps, hot particles drifting out of their tiles between
    sorts (written directly).

After 30 steps every particle (u, s, x), E and B agree with the oracle within
the tolerances of the many-step parity tests.
"""
import numpy as np
import pytest

import workloads as W
from pichelp import (compare_fields, compare_particles, make_pair, window_oracle_run, window_plasmas,
                     window_schedule)

pytestmark = pytest.mark.gpu

STEPS = 30


def test_tiled_rebin_3d_with_window():
    wl = W.small_case3(nx=256, ny=32, nz=32, ppc=1, a0=3.0, u_th=0.2)
    ncells, start, speed = 16, 4, 2.0
    sim, orc, parts = make_pair(wl, sort_every=8, bins=(25, 16), window_cells=ncells)
    try:
        nt = (256 // 16) * (32 // 4) * (32 // 4)
        assert nt >= 4 * 152
        dt, dx = sim.grid()[:2]
        moves = window_schedule(start, STEPS, 0, dt, dx, speed, ncells)
        assert len(moves) >= 2
        plasmas = window_plasmas(wl, ncells, len(moves), [len(parts[0]["ix"])])
        for pl in plasmas:
            sim.stage_injection(pl)
        sim.set_window(ncells, start, speed)
        sim.step(STEPS)
        assert sim.binned(0)
        window_oracle_run(orc, STEPS, start, dt, dx, speed, ncells, plasmas)
        compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
        compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)
    finally:
        sim.close()


def test_tiled_sort_2d_compact():
    wl = W.small_case(nx=256, ny=256, ppc=2, a0=3.0, u_th=0.5)
    sim, orc, _ = make_pair(wl, sort_every=8)
    try:
        sim.step(STEPS)
        orc.step(STEPS)
        compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
        compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)
    finally:
        sim.close()
