"""pic_step replayed from CUDA graphs against pic_step launching every kernel.

  - vacuum with the laser entering (2D3V and 3D3V): no atomics anywhere, so
    the replayed steps must give the launched steps' fields bit for bit
    (this pins the laser table the captured boundary kernels read);
  - plasma with in-step Eq. (4) diagnostics: the same kernels in the same
    order, so everything but the float current sums (whose atomics add in
    any order) agrees exactly: step index, diagnostic step, kernel count;
    particles and fields agree to float rounding, and both runs follow the
    oracle;
  - stretches with the same length, diagnostic phase and buffer parity are
    replayed, not captured again.
"""
import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import compare_fields, compare_particles, make_pair, rel_max

pytestmark = pytest.mark.gpu

FIELDS = ("ex", "ey", "ez", "bx", "by", "bz", "by_left", "bz_left")


def _vacuum_pair(wl, sort_every):
    out = []
    for graphs in (0, 32):
        sim = pic.Simulation(pic.config_from_workload(wl, sort_every=sort_every))
        sim.set_graphs(graphs)
        out.append(sim)
    return out


@pytest.mark.parametrize("three", [False, True], ids=["2d3v", "3d3v"])
def test_vacuum_laser_replayed_steps_are_bit_exact(three):
    wl = W.small_case3(nx=40, ny=16, nz=12) if three else W.small_case(nx=64, ny=32)
    launched, replayed = _vacuum_pair(wl, sort_every=16)
    try:
        for sim in (launched, replayed):
            sim.set_step(3)
            sim.step(45)          # stretches of 16, 16, 13 steps
            sim.sync()
        fa, fb = launched.get_fields(), replayed.get_fields()
        assert np.abs(fa["ey"]).max() > 0.1, "the laser should be in the box"
        for k in FIELDS:
            assert np.array_equal(fa[k], fb[k]), k
        assert launched.get_step() == replayed.get_step() == 48
        assert launched.graph_stats() == (0, 0)
        caps, reps = replayed.graph_stats()
        assert caps >= 2 and caps + reps == 3, (caps, reps)
    finally:
        launched.close()
        replayed.close()


def test_plasma_with_diagnostics_replayed_like_launched():
    wl = W.small_case(nx=64, ny=32, ppc=4, u_th=0.3, two_species=True, a0=3.0)
    sims, orcs = [], []
    for graphs in (0, 32):
        sim, orc, _ = make_pair(wl, sort_every=8)
        sim.set_graphs(graphs)
        sim.set_diagnostics(4)
        sims.append(sim)
        orcs.append(orc)
    launched, replayed = sims
    try:
        for sim in sims:
            sim.step(40)          # stretches of 8 after each sort: two parities, one diagnostic phase
            sim.sync()
        orc = orcs[0]
        orc.step(40)
        assert launched.get_step() == replayed.get_step() == 40
        da, ma = launched.get_diagnostics()
        db, mb = replayed.get_diagnostics()
        assert da == db == 40
        assert launched.launch_count() == replayed.launch_count()
        caps, reps = replayed.graph_stats()
        assert caps == 2 and reps >= 2, (caps, reps)
        for s in range(2):
            np.testing.assert_allclose(ma[s]["P"], mb[s]["P"], atol=1e-6)
            ga, gb = launched.get_particles_f64(s), replayed.get_particles_f64(s)
            oa, ob = np.argsort(ga["id"]), np.argsort(gb["id"])
            assert np.array_equal(ga["id"][oa], gb["id"][ob])
            for k in ("ux", "uy", "uz", "sx", "sy", "sz"):
                assert np.abs(ga[k][oa] - gb[k][ob]).max() <= 1e-4 * max(1.0, np.abs(ga[k]).max()), k
            compare_particles(replayed, orc, s, 1e-4, 1e-4, 1e-4)
        fa, fb = launched.get_fields(), replayed.get_fields()
        for k in FIELDS:
            assert rel_max(fb[k].astype(float), fa[k].astype(float)) <= 1e-4, k
        compare_fields(replayed, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)
    finally:
        for sim in sims:
            sim.close()


def test_graphs_off_and_on_again_and_binned_layout_launches():
    # the binned 3D3V layout takes no graph (its re-bin decision is made
    # between steps); switching graphs off drops them
    wl = W.small_case3(nx=32, ny=16, nz=12, ppc=2, u_th=0.3)
    sim, orc, _ = make_pair(wl, sort_every=8, bins=(25, 16))
    try:
        sim.step(10)
        orc.step(10)
        assert sim.graph_stats() == (0, 0)
        compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    finally:
        sim.close()
    with pytest.raises(pic.PicError):
        s2 = pic.Simulation(pic.config_from_workload(W.small_case()))
        try:
            s2.set_graphs(-1)
        finally:
            s2.close()
