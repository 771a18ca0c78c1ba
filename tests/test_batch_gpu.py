"""GPU tests of the batch of independent 2D3V runs (pic_batch_*): against the
same runs stepped one by one through the single-run calls, against the
oracle, the per-run step counts, and the autotuner."""
import numpy as np
import pytest

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import compare_fields, compare_particles, rel_l2

pytestmark = pytest.mark.gpu


def _scan(nruns=5, seed=7):
    runs = W.batch_scan(nruns, seed=seed, size_scale=0.06, step_scale=0.012)
    # one run longer than the others, one with no steps at all
    runs[0] = (runs[0][0], 14)
    runs[-1] = (runs[-1][0], 0)
    return runs


def _load(sim, wl):
    parts = W.generate_particles(wl)
    for s, d in enumerate(parts):
        sim.set_particles(s, d)
    sim.capture_background()
    return parts


def test_batch_matches_single_runs_and_stops_each_run_at_its_length():
    runs = _scan()
    cfgs = [pic.config_from_workload(wl, sort_every=4) for wl, _ in runs]
    with pic.Batch(cfgs, [n for _, n in runs]) as b:
        for r, (wl, _) in enumerate(runs):
            _load(b.run(r), wl)
        b.step(6)
        b.step(100)
        assert b.steps_done() == [n for _, n in runs]
        for r, (wl, n) in enumerate(runs):
            with pic.Simulation(pic.config_from_workload(wl, sort_every=4)) as one:
                _load(one, wl)
                one.step(n)
                a, c = b.run(r), one
                assert a.get_step() == c.get_step() == n
                # the batch sorts (and so compacts removed particles) at the end
                # of a sort-free stretch, pic_step at the start of the next step:
                # compare the live particles
                pa, pc = a.get_particles(0), c.get_particles(0)
                pa = {k: v[pa["ix"] >= 0] for k, v in pa.items()}
                pc = {k: v[pc["ix"] >= 0] for k, v in pc.items()}
                assert len(pa["id"]) == len(pc["id"])
                oa, oc = np.argsort(pa["id"]), np.argsort(pc["id"])
                for k in ("ix", "iy", "id"):
                    assert np.array_equal(pa[k][oa], pc[k][oc]), (r, k)
                for k in ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz"):
                    np.testing.assert_allclose(pa[k][oa], pc[k][oc], rtol=1e-5, atol=1e-6, err_msg=f"{r} {k}")
                fa, fc = a.get_fields(), c.get_fields()
                for k in ("ex", "ey", "ez", "bx", "by", "bz"):
                    assert rel_l2(fa[k].astype(float), fc[k].astype(float)) < 1e-5, (r, k)


def test_batch_matches_oracle():
    runs = _scan(nruns=3, seed=8)
    runs = [(wl, 10) for wl, _ in runs]
    cfgs = [pic.config_from_workload(wl, sort_every=3) for wl, _ in runs]
    with pic.Batch(cfgs, [n for _, n in runs]) as b:
        orcs = []
        for r, (wl, _) in enumerate(runs):
            parts = _load(b.run(r), wl)
            orcs.append(oracle.OracleSim(wl, parts))
        b.step(10)
        for r, o in enumerate(orcs):
            o.step(10)
            sim = b.run(r)
            compare_particles(sim, o, 0, 1e-4, 1e-4, 1e-4)
            compare_fields(sim, o, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)
            om, gm = o.moments(0), sim.polarization(0)
            np.testing.assert_allclose(gm["P"], om[:3], atol=1e-5)


def test_batch_tune_picks_a_candidate_and_keeps_the_state():
    runs = [(wl, 40) for wl, _ in _scan(nruns=3, seed=9)]
    cfgs = [pic.config_from_workload(wl) for wl, _ in runs]
    with pic.Batch(cfgs, [n for _, n in runs]) as b:
        orcs = []
        for r, (wl, _) in enumerate(runs):
            parts = _load(b.run(r), wl)
            orcs.append(oracle.OracleSim(wl, parts))
        tx, ty, se = b.tune(2, tiles=((16, 8), (8, 4)), sorts=(2, 3))
        assert (tx, ty) in ((16, 8), (8, 4)) and se in (2, 3)
        done = b.steps_done()
        assert len(set(done)) == 1 and done[0] > 0
        b.step(3)
        for r, o in enumerate(orcs):
            o.step(done[r] + 3)
            compare_particles(b.run(r), o, 0, 1e-4, 1e-4, 1e-4)
            compare_fields(b.run(r), o, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)


def test_batch_rejects_3d_and_fp64():
    wl = W.small_case3(nx=16, ny=8, nz=6)
    with pytest.raises(pic.PicError):
        pic.Batch([pic.config_from_workload(wl)], [1])
    wl2 = W.small_case(nx=32, ny=16)
    with pytest.raises(pic.PicError):
        pic.Batch([pic.config_from_workload(wl2, precision=64)], [1])
