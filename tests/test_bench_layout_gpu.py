"""The 3D3V benchmark's own layout at scale, with the laser inside the plasma.

A cut of the 512 x 256 x 256 laser-wakefield workload (512 x 32 x 8 cells,
260,096 electrons at 2 per cell, a0 = 3) runs in the layout the benchmark
times: binned ranges with 25 % headroom and 16 spare slots, the default
16 x 4 x 4 tiles (512 CTAs), a re-bin every 64 steps.  The run starts at the
step where the envelope of the pulse is near its peak at x = 0, so within a
few steps the laser drives the plasma: particles cross cells and tiles in
every direction and arrive in other tiles' ranges.

Three checks, the tolerances of the parity tests:
  - per step: at three points of the run the oracle's state is loaded into a
    second context, and one step of each is compared: every particle's u
    (relative, floor 1e-3), s and x at 1e-5, and J, E, B and the left
    boundary values element by element at 1e-5 of the largest magnitude;
  - over the run: a context started from the same seeded state as the oracle
    runs 120 steps beside it, and the Eq. (4) polarization, the mean and the
    variance of the kinetic energy agree within 1 %, the live counts within
    0.1 %;
  - the same with the co-moving window on (moves of one 16-cell tile column
    from 10 steps into the run, the plasma of each move staged): the ranges
    are relabelled in place across several moves and a re-bin, and the run
    still follows the oracle's window within those bounds.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import (compare_fields, compare_particles, make_pair, window_oracle_run, window_plasmas,
                     window_schedule)

pytestmark = pytest.mark.gpu

BINS = (25, 16)
SORT_EVERY = 64
STEPS = 120
CHECK_AT = (30, 75, 118)


def _cut():
    return W.scaled(W.CONFIG2, name="3d3v-512x32x8-cut-ppc2-lp-a0_3", ny=32, nz=8)


def _load_oracle_state(sim, orc):
    """The oracle's particles (float64, removed ones left out), E, B, the left
    boundary values and the step index, loaded into a library context."""
    for s, p in enumerate(orc.p):
        live = p["alive"].astype(bool)
        d = {"id": np.flatnonzero(live).astype(np.int32)}
        for a in ("x", "y", "z"):
            v = p[a][live]
            i = np.floor(v)
            d["i" + a] = i.astype(np.int32)
            d["o" + a] = v - i
        for k in ("ux", "uy", "uz", "sx", "sy", "sz", "w"):
            d[k] = p[k][live]
        sim.set_particles_f64(s, d)
    f = {k: orc.f[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    f["by_left"] = orc.f["byL"]
    f["bz_left"] = orc.f["bzL"]
    sim.set_fields(f)
    sim.set_step(orc.step_index)


def _one_step_compared(chk, orc):
    chk.push_deposit()          # the layout was compacted by the upload: this re-bins first
    orc.zero_current()
    saved = [orc.push(s) for s in range(len(orc.p))]
    for s, old in enumerate(saved):
        orc.deposit(s, *old)
    compare_fields(chk, orc, ("jx", "jy", "jz"), 1e-5)
    chk.field_update()
    orc.field_update()
    compare_fields(chk, orc, ("ex", "ey", "ez", "bx", "by", "bz", "by_left", "bz_left"), 1e-5)
    for s in range(len(orc.p)):
        compare_particles(chk, orc, s, 1e-5, 1e-5, 1e-5)


def test_binned_layout_at_scale_with_the_laser_in_the_plasma():
    wl = _cut()
    dt = 0.95 / math.sqrt(sum((1 / (d * 2 * math.pi)) ** 2 for d in (wl.dx_lambda, wl.dy_lambda, wl.dz_lambda)))
    start = int(round(wl.t_peak_periods * 2 * math.pi / dt)) - 30
    sim, orc, _ = make_pair(wl, step=start, sort_every=SORT_EVERY, bins=BINS)
    assert sim.grid()[0] == pytest.approx(dt, rel=1e-12)
    chk = pic.Simulation(pic.config_from_workload(wl, sort_every=SORT_EVERY, bins=BINS))
    try:
        k = 0
        hot = 0.0
        while k < STEPS:
            if k in CHECK_AT:
                _load_oracle_state(chk, orc)
                _one_step_compared(chk, orc)       # advances the oracle by one step
                sim.step(1)
                k += 1
                continue
            sim.step(1)
            orc.step(1)
            k += 1
        assert orc.step_index == start + STEPS
        assert sim.get_step() == start + STEPS
        # the laser is in the plasma: fields of order a0, particles driven to |u| ~ 1
        assert np.abs(orc.f["ey"]).max() > 1.0
        u = np.sqrt(orc.p[0]["ux"] ** 2 + orc.p[0]["uy"] ** 2 + orc.p[0]["uz"] ** 2)
        hot = float((u > 0.5).mean())
        assert hot > 0.02, hot
        g = sim.polarization(0)
        om = orc.moments(0)
        assert abs(g["count"] - om[4]) <= 1e-3 * om[4]
        np.testing.assert_allclose(g["P"], om[:3], atol=1e-2)
        assert g["ekin_mean"] == pytest.approx(om[5], rel=1e-2)
        assert g["ekin_var"] == pytest.approx(om[6], rel=1e-2)
    finally:
        chk.close()
        sim.close()


def test_binned_layout_at_scale_co_moving():
    wl = _cut()
    dt = 0.95 / math.sqrt(sum((1 / (d * 2 * math.pi)) ** 2 for d in (wl.dx_lambda, wl.dy_lambda, wl.dz_lambda)))
    start = int(round(wl.t_peak_periods * 2 * math.pi / dt)) - 30
    sim, orc, parts = make_pair(wl, step=start, sort_every=SORT_EVERY, bins=BINS, window_cells=16)
    try:
        dt, dx = sim.grid()[:2]
        ncells, w0 = 16, start + 10
        moves = window_schedule(w0, STEPS, start, dt, dx, 1.0, ncells)
        assert len(moves) >= 5, moves
        plasmas = window_plasmas(wl, ncells, len(moves), [len(parts[0]["ix"])])
        for pl in plasmas:
            sim.stage_injection(pl)
        sim.set_window(ncells, w0, 1.0)
        for k in range(STEPS):
            sim.step(1)
            # the moves and the re-bin keep the binned layout (no fallback to the compact one)
            assert sim.binned(0), k
        sim.sync()
        with oracle.parallel():
            moved = window_oracle_run(orc, STEPS, w0, dt, dx, 1.0, ncells, plasmas)
        assert moved == sim.window() == len(moves) * ncells
        assert sim.staged_injections() == 0
        assert np.abs(orc.f["ey"]).max() > 1.0
        g = sim.polarization(0)
        om = orc.moments(0)
        assert abs(g["count"] - om[4]) <= 1e-3 * om[4]
        np.testing.assert_allclose(g["P"], om[:3], atol=1e-2)
        assert g["ekin_mean"] == pytest.approx(om[5], rel=1e-2)
        assert g["ekin_var"] == pytest.approx(om[6], rel=1e-2)
        compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-2)
    finally:
        sim.close()
