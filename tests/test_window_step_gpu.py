"""The co-moving window on the stepping path (pic_set_window,
pic_stage_injection) against the oracle's window (Sec. 2: the box follows the
laser through the plasma).

pic_step moves the box before the step from index n whenever
n >= start and moved + ncells <= floor((n - start) dt speed / dx); the oracle
run (pichelp.window_oracle_run) applies the same rule, written out there, with
orc.shift_window and the same staged plasma in the same order.  Cases:
  - 3D3V binned layout, moves of one tile column (16-wide and 8-wide tiles):
    the ranges are relabelled, no sort; the launch count of a step with a
    move shows that path (seven kernels more than a step without), and the
    layout is still binned at the end;
  - 3D3V binned layout with moves that are not tile multiples, and the
    compact layout: the compact path (append, sort);
  - 2D3V with CUDA graphs (stretches end where a move is due), FP32 and FP64
    with two co-located species;
  - fewer plasmas staged than moves: the last moves let vacuum in;
  - argument checks.
After several moves, every particle (u, s, x), E, B and the Gauss residual
agree with the oracle within the window tests' tolerances.
"""
import math

import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import compare_fields, compare_particles, make_pair, window_oracle_run, window_plasmas, window_schedule

pytestmark = pytest.mark.gpu


def _run(wl, steps, ncells, speed, start, *, tile=None, bins=None, sort_every=64, precision=32,
         staged_short=0, graphs=None):
    sim, orc, parts = make_pair(wl, sort_every=sort_every, tile=tile, bins=bins, precision=precision,
                                window_cells=ncells)
    if graphs is not None:
        sim.set_graphs(graphs)
    dt, dx = sim.grid()[0], sim.grid()[1]
    moves = window_schedule(start, steps, 0, dt, dx, speed, ncells)
    assert len(moves) >= 3, moves
    ids = [len(p["ix"]) for p in parts]
    slabs = window_plasmas(wl, ncells, len(moves) - staged_short, ids)
    for sl in slabs:
        sim.stage_injection(sl)
    assert sim.staged_injections() == len(slabs)
    sim.set_window(ncells, start, speed)
    return sim, orc, slabs, moves, (dt, dx)


def _finish(sim, orc, steps, start, grid, speed, ncells, slabs, moves, tol=1e-4, f64=False):
    moved = window_oracle_run(orc, steps, start, grid[0], grid[1], speed, ncells, slabs)
    assert moved == len(moves) * ncells
    assert sim.window() == moved
    assert sim.get_step() == orc.step_index
    assert sim.staged_injections() == 0
    for s in range(len(orc.p)):
        compare_particles(sim, orc, s, tol, tol, tol, f64=f64)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), tol, f64=f64)
    r_max, _ = sim.gauss_residual()
    r_orc = np.abs(orc.gauss_residual()).max()
    assert abs(r_max - r_orc) < 1e-4 + 1e-3 * r_orc, (r_max, r_orc)


CASES3 = {
    # name: tile, bins, ncells, speed
    "binned-rotate-16": ((16, 4, 4), (25, 16), 16, 2.0),
    "binned-rotate-8": ((8, 4, 4), (25, 16), 8, 1.0),
    "binned-unaligned": ((16, 4, 4), (25, 16), 6, 1.0),
    "compact": ((16, 4, 4), None, 5, 1.0),
}


@pytest.mark.parametrize("case", list(CASES3))
def test_window_in_pic_step_3d(case):
    tile, bins, ncells, speed = CASES3[case]
    wl = W.small_case3(nx=64, ny=8, nz=8, ppc=2, a0=3.0, u_th=0.05)
    steps, start = 60, 4
    sim, orc, slabs, moves, grid = _run(wl, steps, ncells, speed, start, tile=tile, bins=bins)
    try:
        if case == "binned-rotate-16":
            # up to the first move, then one step with a move and one without
            k0 = moves[0]
            sim.step(k0)
            l0 = sim.launch_count()
            sim.step(1)
            l1 = sim.launch_count()
            assert moves[1] > k0 + 1
            sim.step(1)
            l2 = sim.launch_count()
            # the move: rows, cells, vacate, inject, counters, live count, background
            assert (l1 - l0) - (l2 - l1) == 7, (l0, l1, l2)
            sim.step(steps - k0 - 2)
        else:
            sim.step(steps)
        if bins and ncells % tile[0] == 0:
            assert sim.binned(0), "the moves relabel ranges: the layout stays binned"
        _finish(sim, orc, steps, start, grid, speed, ncells, slabs, moves)
        assert (~orc.p[0]["alive"].astype(bool)).sum() > 0, "the moves should have removed particles"
    finally:
        sim.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_window_in_pic_step_2d_graphs(precision):
    two = precision == 64
    wl = W.small_case(nx=64, ny=16, ppc=2, a0=3.0, u_th=0.05, two_species=two)
    steps, start, ncells = 50, 3, 4
    sim, orc, slabs, moves, grid = _run(wl, steps, ncells, 1.0, start, sort_every=16, precision=precision,
                                        graphs=32)
    try:
        sim.step(steps)
        caps, reps = sim.graph_stats()
        assert caps + reps > 0
        tol = 1e-10 if precision == 64 else 1e-4
        _finish(sim, orc, steps, start, grid, 1.0, ncells, slabs, moves, tol=tol, f64=precision == 64)
    finally:
        sim.close()


def test_window_vacuum_when_nothing_staged():
    wl = W.small_case3(nx=64, ny=8, nz=8, ppc=2, a0=3.0, u_th=0.05)
    steps, start, ncells = 60, 4, 16
    sim, orc, slabs, moves, grid = _run(wl, steps, ncells, 2.0, start, tile=(16, 4, 4), bins=(25, 16),
                                        staged_short=2)
    try:
        sim.step(steps)
        _finish(sim, orc, steps, start, grid, 2.0, ncells, slabs, moves)
    finally:
        sim.close()


def test_window_argument_checks():
    wl = W.small_case3(nx=32, ny=8, nz=8, ppc=1)
    sim, _, parts = make_pair(wl)
    try:
        for bad in ((-1, 0, 1.0), (wl.nx - 7, 0, 1.0), (4, 0, 0.0), (4, 0, float("nan"))):
            with pytest.raises(pic.PicError) as e:
                sim.set_window(*bad)
            assert e.value.status == -1
        sim.set_window(0)  # off
        # a cell outside the particle region: nothing staged
        inj = W.injection_particles(wl, 4, seed=1, id_base=len(parts[0]["ix"]))
        inj[0]["ix"][0] = wl.nx - 1
        with pytest.raises(pic.PicError) as e:
            sim.stage_injection(inj)
        assert e.value.status == -1
        assert sim.staged_injections() == 0
    finally:
        sim.close()
    wlp = W.small_case3(nx=32, ny=8, nz=8, ppc=1, bc_x="periodic")
    simp, _, _ = make_pair(wlp)
    try:
        with pytest.raises(pic.PicError):
            simp.set_window(4, 0, 1.0)
    finally:
        simp.close()
