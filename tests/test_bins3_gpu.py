"""GPU parity of the binned 3D3V layout against the FP64 3D oracle.

In the binned layout every tile owns a slot range with spare room and each
fused step stores every surviving particle into the range of the tile its new
cell lies in (in the other particle buffer), with one overflow range for
particles whose tile range is full.  The physics is that of the compact
layout, so the tolerances are those of the compact-layout tests; the cases
drive particles across tile boundaries every step, fill ranges to overflow,
and mix binned steps with read-backs, window shifts, in-step diagnostics and
the FP64 instantiation.
"""
import numpy as np
import pytest

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import compare_fields, compare_particles, make_pair

pytestmark = pytest.mark.gpu


def _tiles_of(ix, iy, iz, wl, tile=(16, 4, 4)):
    ntx, nty = -(-wl.nx // tile[0]), -(-wl.ny // tile[1])
    return ((iz // tile[2]) * nty + iy // tile[1]) * ntx + ix // tile[0]


def _cells(orc, s):
    p = orc.p[s]
    alive = p["alive"].astype(bool)
    return (np.floor(p["x"][alive]).astype(int), np.floor(p["y"][alive]).astype(int),
            np.floor(p["z"][alive]).astype(int))


@pytest.mark.parametrize("tile", [None, (8, 4, 4), (32, 4, 4)], ids=["16x4x4", "8x4x4", "32x4x4"])
def test_binned_many_steps_laser_removal_two_species(tile):
    # hot particles cross tile boundaries every step, leave at the open x ends,
    # and the laser enters at x_min; re-binned every 5 steps
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, u_th=2.0, a0=6.0, two_species=True)
    sim, orc, _ = make_pair(wl, sort_every=5, tile=tile, bins=(25, 16))
    for _ in range(3):
        sim.step(4)
        orc.step(4)
    assert (~orc.p[0]["alive"].astype(bool)).sum() > 0, "case should remove particles"
    assert np.abs(orc.f["ey"]).max() > 0.5, "laser should be in the box"
    for s in range(len(wl.species)):
        compare_particles(sim, orc, s, 1e-4, 1e-4, 1e-4)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)


def test_binned_overflow_range_carries_the_excess():
    # 10% headroom, no extra slots: tiles that gain more than that spill
    # into the overflow range, whose particles take the global path and are
    # binned again on the next step
    wl = W.small_case3(nx=34, ny=16, nz=12, ppc=3, u_th=1.5, bc_x="periodic", pol="none")
    sim, orc, parts = make_pair(wl, sort_every=100, bins=(10, 0))
    # the ranges are sized on the initial tile counts, and arrivals take the
    # spare slots after them: the oracle says which tiles receive more
    # arrivals than that after one step
    t0 = _tiles_of(parts[0]["ix"], parts[0]["iy"], parts[0]["iz"], wl)
    c0 = np.bincount(t0)
    spare = (c0 + c0 * 10 // 100 + 7) // 8 * 8 - c0
    sim.step(1)
    orc.step(1)
    p = orc.p[0]
    t1 = _tiles_of(np.floor(p["x"]).astype(int), np.floor(p["y"]).astype(int), np.floor(p["z"]).astype(int), wl)
    moved = (t1 != t0) & p["alive"].astype(bool)
    arrivals = np.bincount(t1[moved], minlength=len(c0))
    assert np.maximum(arrivals - spare, 0).sum() > 0, "case should spill arrivals into the overflow range"
    compare_particles(sim, orc, 0, 1e-5, 1e-5, 1e-5)
    for _ in range(4):
        sim.step(2)
        orc.step(2)
    compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)


def test_binned_matches_compact_layout_state():
    # binned and compact contexts from one state: the same particles after
    # every step (up to float summation order in J)
    wl = W.small_case3(nx=26, ny=18, nz=13, ppc=2, u_th=0.8, bc_x="open", two_species=True)
    f = W.random_fields(wl, seed=23)
    a, orc, _ = make_pair(wl, fields=f, step=3, sort_every=4, bins=(25, 16))
    b, _, _ = make_pair(wl, fields=f, step=3, sort_every=4)
    for _ in range(6):
        a.step(1)
        b.step(1)
        orc.step(1)
    for s in range(2):
        compare_particles(a, orc, s, 1e-4, 1e-4, 1e-4)
        compare_particles(b, orc, s, 1e-4, 1e-4, 1e-4)
    fa, fb = a.get_fields(), b.get_fields()
    for k in ("ex", "ey", "ez", "bx", "by", "bz"):
        np.testing.assert_allclose(fa[k], fb[k], atol=1e-5 * max(1.0, np.abs(fb[k]).max()))


def test_binned_in_step_diagnostics_match_oracle():
    # the Eq. (4) sums of the fused step include the overflow range's CTAs
    wl = W.small_case3(nx=34, ny=16, nz=12, ppc=3, u_th=1.0, bc_x="periodic", pol="none")
    sim, orc, _ = make_pair(wl, sort_every=100, bins=(10, 0))
    emin, emax = 0.0, 50.0
    sim.set_diagnostics(3, [emin], [emax])
    sim.step(6)
    orc.step(6)
    step, diag = sim.get_diagnostics()
    assert step == 6
    om = orc.moments(0, emin, emax)
    assert diag[0]["count"] == om[4]
    np.testing.assert_allclose(diag[0]["P"], om[:3], atol=1e-5)
    assert diag[0]["ekin_mean"] == pytest.approx(om[5], rel=1e-4)


def test_binned_read_back_then_resume():
    # a read-back returns the compact layout; stepping on re-bins
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, u_th=1.0, a0=5.0)
    sim, orc, _ = make_pair(wl, sort_every=6, bins=(25, 16))
    for _ in range(4):
        sim.step(3)
        orc.step(3)
        compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)


def test_binned_fp64_matches_oracle():
    wl = W.small_case3(nx=26, ny=18, nz=13, ppc=2, bc_x="open", two_species=True, u_th=0.6)
    f = W.random_fields(wl, seed=29)
    sim, orc, _ = make_pair(wl, fields=f, step=1, precision=64, sort_every=3, bins=(10, 4))
    for _ in range(5):
        sim.step(1)
        orc.step(1)
    for s in range(2):
        compare_particles(sim, orc, s, 1e-11, 1e-11, 1e-11, f64=True)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-11, f64=True)


def test_binned_falls_back_to_compact_when_capacity_is_short():
    # capacity for the particles but not for the ranges: the compact layout
    # carries on, with the same results
    wl = W.small_case3(nx=26, ny=18, nz=13, ppc=2, u_th=0.5)
    parts = W.generate_particles(wl)
    cfg = pic.config_from_workload(wl, capacity_factor=1.05, sort_every=3)
    cfg.bin_headroom_pct, cfg.bin_min_extra = 25, 16
    sim = pic.Simulation(cfg)
    sim.set_particles(0, parts[0])
    orc = oracle.OracleSim(wl, parts)
    sim.step(6)
    orc.step(6)
    compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    sim.close()


def test_binned_window_shift():
    # a window shift compacts, appends the injected plasma, and re-bins
    wl = W.small_case3(nx=48, ny=10, nz=8, ppc=2, a0=3.0, u_th=0.05)
    sim, orc, parts = make_pair(wl, sort_every=4, bins=(25, 16))
    next_id = len(parts[0]["ix"])
    for steps, n in ((8, 6), (8, 10)):
        sim.step(steps)
        orc.step(steps)
        inj = W.injection_particles(wl, n, seed=50 + n, id_base=next_id)
        next_id += len(inj[0]["ix"])
        sim.shift_window(n, inj)
        orc.shift_window(n, inj)
    sim.step(6)
    orc.step(6)
    compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)


def test_binned_layout_feeds_the_slot_wise_reductions():
    # pic_polarization, pic_energy_histogram and pic_gauss_residual read every
    # slot of the binned ranges (holes hold PIC_DEAD) between binned steps
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, u_th=1.5, a0=5.0, two_species=True)
    sim, orc, _ = make_pair(wl, sort_every=100, bins=(10, 4))
    sim.step(7)
    orc.step(7)
    for s in range(2):
        gm = sim.polarization(s)
        om = orc.moments(s)
        assert gm["count"] == om[4]
        np.testing.assert_allclose(gm["P"], om[:3], atol=1e-5)
        assert gm["ekin_mean"] == pytest.approx(om[5], rel=1e-4)
        # counts exact but for a particle at a bin edge (decided in float)
        g = sim.energy_histogram(s, 0.0, 40.0, 16)
        o = orc.histogram(s, 0.0, 40.0, 16)
        diff = np.abs(g[:, 0] - o[:, 0])
        assert diff.sum() <= 2, (g[:, 0], o[:, 0])
        ok = diff == 0
        np.testing.assert_allclose(g[ok, 1:], o[ok, 1:], rtol=1e-4, atol=1e-6 * np.abs(o[:, 1]).max())
    r_max, _ = sim.gauss_residual()
    r_orc = np.abs(orc.gauss_residual()).max()
    assert abs(r_max - r_orc) < 1e-4 + 1e-3 * r_orc, (r_max, r_orc)


def test_binned_steps_then_split_path_and_fresh_upload():
    # the split kernels read every slot: the stale slots the binned steps
    # leave are sealed first; a fresh upload replaces the layout
    wl = W.small_case3(nx=34, ny=16, nz=12, ppc=2, u_th=1.2, bc_x="periodic", pol="none", two_species=True)
    sim, orc, parts = make_pair(wl, sort_every=4, bins=(25, 16))
    sim.step(3)
    orc.step(3)
    sim.gather_push_spin()
    sim.deposit()
    sim.field_update()
    orc.step(1)
    sim.step(2)
    orc.step(2)
    for s in range(2):
        compare_particles(sim, orc, s, 1e-4, 1e-4, 1e-4)
    # upload the oracle's state over the binned layout and step on
    sim.step(2)
    for s, d in enumerate(parts):
        sim.set_particles(s, d)
    orc2 = oracle.OracleSim(wl, parts, fields=None)
    sim.set_fields({k: orc2.f[k].astype(np.float32) for k in ("ex", "ey", "ez", "bx", "by", "bz")})
    sim.set_step(0)
    sim.step(2)
    orc2.step(2)
    for s in range(2):
        compare_particles(sim, orc2, s, 1e-4, 1e-4, 1e-4)
    sim.sync()  # no device error flag left (no particle dropped)


def test_binned_overflow_alert_rebins_before_particles_are_lost():
    # little headroom, a hot plasma and no periodic sort: tile ranges keep
    # spilling into the overflow range, whose alert past half full makes the
    # next step re-bin instead of letting the range fill and drop particles
    wl = W.small_case3(nx=34, ny=16, nz=12, ppc=3, u_th=3.0, bc_x="periodic", pol="none", two_species=True)
    sim, orc, _ = make_pair(wl, sort_every=1000, bins=(1, 0))
    launches = []
    for _ in range(12):
        l0 = sim.launch_count()
        sim.step(1)
        sim.sync()  # the host reads the alert of each step before the next
        launches.append(sim.launch_count() - l0)
        orc.step(1)
    assert max(launches) > min(launches), "a step should have re-binned (its sort's launches)"
    for s in range(2):
        compare_particles(sim, orc, s, 1e-4, 1e-4, 1e-4)
