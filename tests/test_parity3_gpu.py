"""GPU parity of the 3D3V path through the C ABI against the FP64 3D oracle,
with the tolerances of the 2D3V parity tests (per step: momentum relative
1e-5 with a floor of 1e-3 on |u|, spin absolute 1e-5, position 1e-5 cells,
relative L2 of J, E, B 1e-5; removal and sort permutation exact)."""
import math

import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import compare_fields, compare_particles, make_pair

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    dict(nx=26, ny=18, nz=13, ppc=2, bc_x="open", two_species=True),    # ragged against every tile shape
    dict(nx=24, ny=16, nz=12, ppc=2, bc_x="periodic", two_species=False),
    dict(nx=20, ny=12, nz=9, ppc=3, bc_x="open", two_species=False, pol="cp"),
]
IDS = ["open-2sp-ragged", "periodic", "open-cp"]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_split_path_one_step_3d(case):
    wl = W.small_case3(u_th=0.3, **case)
    f = W.random_fields(wl, seed=17)
    sim, orc, _ = make_pair(wl, fields=f, step=4)
    sim.gather_push_spin()
    sim.deposit()
    orc.zero_current()
    saved = [orc.push(s) for s in range(len(orc.p))]
    for s, old in enumerate(saved):
        orc.deposit(s, *old)
    for s in range(len(wl.species)):
        compare_particles(sim, orc, s, TOL, TOL, TOL)
    compare_fields(sim, orc, ("jx", "jy", "jz"), TOL)
    sim.field_update()
    orc.field_update()
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz", "by_left", "bz_left"), TOL)
    f = sim.get_fields()
    np.testing.assert_allclose(f["by_left"], orc.f["byL"], atol=1e-5 * max(1.0, np.abs(orc.f["byL"]).max()))
    np.testing.assert_allclose(f["bz_left"], orc.f["bzL"], atol=1e-5 * max(1.0, np.abs(orc.f["bzL"]).max()))


@pytest.mark.parametrize("tile", [None, (8, 8, 4), (8, 4, 4)], ids=["16x4x4", "8x8x4", "8x4x4"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fused_step_one_step_3d(case, tile):
    wl = W.small_case3(u_th=0.3, **case)
    f = W.random_fields(wl, seed=18)
    sim, orc, _ = make_pair(wl, fields=f, step=2, tile=tile)
    sim.push_deposit()
    orc.zero_current()
    saved = [orc.push(s) for s in range(len(orc.p))]
    for s, old in enumerate(saved):
        orc.deposit(s, *old)
    for s in range(len(wl.species)):
        compare_particles(sim, orc, s, TOL, TOL, TOL)
    compare_fields(sim, orc, ("jx", "jy", "jz"), TOL)
    sim.field_update()
    orc.field_update()
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz", "by_left", "bz_left"), TOL)


def test_fused_many_steps_3d_with_laser_sorting_and_removal():
    # fast particles leave their tiles (sorted every 3 steps) and the box; the
    # laser enters at x_min
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, u_th=2.0, a0=6.0)
    sim, orc, _ = make_pair(wl, sort_every=3, tile=(8, 4, 4))
    for _ in range(12):
        sim.step(1)
        orc.step(1)
    assert (~orc.p[0]["alive"].astype(bool)).sum() > 0, "case should remove particles"
    assert np.abs(orc.f["ey"]).max() > 0.5, "laser should be in the box"
    compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-4)


def test_sort_3d_is_a_grouping_permutation():
    wl = W.small_case3(nx=32, ny=16, nz=12, ppc=3, u_th=1.0, two_species=True)
    sim, orc, parts = make_pair(wl)
    sim.step(4)
    before = [sim.get_particles(s) for s in range(2)]
    sim.sort()
    for s in range(2):
        b, a = before[s], sim.get_particles(s)
        live = b["ix"] >= 0
        assert len(a["id"]) == live.sum()
        ob, oa = np.argsort(b["id"]), np.argsort(a["id"])
        bl = {k: v[ob][live[ob]] for k, v in b.items()}
        for k in a:
            assert np.array_equal(a[k][oa], bl[k]), k
        ntx, nty = (32 + 15) // 16, (16 + 3) // 4     # default 16x4x4 tiles
        tile = ((a["iz"] // 4) * nty + a["iy"] // 4) * ntx + a["ix"] // 16
        assert np.all(np.diff(tile) >= 0)


def test_gauss_law_and_polarization_3d():
    # neutral start with the laser entering: the GPU's Gauss residual stays at
    # FP32 round-off and its Eq. (4) moments follow the oracle
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, a0=6.0, u_th=0.05)
    sim, orc, _ = make_pair(wl)
    for _ in range(3):
        sim.step(10)
        orc.step(10)
        r_max, r_rms = sim.gauss_residual()
        f = sim.get_fields()
        emax = max(np.abs(f[k]).max() for k in ("ex", "ey", "ez"))
        _, dx, dy, dz = sim.grid()
        bound = 4 * np.finfo(np.float32).eps * (emax * (1 / dx + 1 / dy + 1 / dz) + 0.05) * math.sqrt(orc.step_index)
        assert r_max < bound, (r_max, bound)
    om = orc.moments(0)
    gm = sim.polarization(0)
    assert gm["count"] == om[4]
    np.testing.assert_allclose(gm["P"], om[:3], atol=1e-5)
    assert gm["ekin_mean"] == pytest.approx(om[5], rel=1e-4)


def test_3d_fp64_instantiation_matches_oracle():
    wl = W.small_case3(nx=26, ny=18, nz=13, ppc=2, bc_x="open", two_species=True, u_th=0.3)
    f = W.random_fields(wl, seed=19)
    sim, orc, _ = make_pair(wl, fields=f, step=1, precision=64)
    for _ in range(3):
        sim.step(1)
        orc.step(1)
    for s in range(2):
        compare_particles(sim, orc, s, 1e-11, 1e-11, 1e-11, f64=True)
    compare_fields(sim, orc, ("ex", "ey", "ez", "bx", "by", "bz"), 1e-11, f64=True)
