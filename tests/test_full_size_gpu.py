"""The 3D3V laser-wakefield workload at its full size (512 x 256 x 256 cells,
66.6 million electrons) in the launch configuration the benchmark times
(binned layout, 25 % headroom, 16 spare slots, 16 x 4 x 4 tiles, re-binned
every 64 steps), checked on outputs the oracle can compute piece by piece.

The run is advanced through pic_step to the interaction phase (40 steps
after the envelope peak reaches x = 0); then one step is taken with
pic_push_deposit and pic_field_update, and its state before and after is
read back:
  - a1-a4: 200,000 particles drawn at random, plus every particle of a
    32 x 16 x 16-cell box on the axis where the particles move fastest,
    pushed by the oracle in the read-back fields; u (relative to the larger
    of |u| before and after the step, floor 1e-3), s and x (cells) within
    1e-5 of the GPU's, and the same particles removed through x_min;
  - a5: the oracle's current of that box's particles (and of a 3-cell margin
    around it) on the box's nodes, element by element within 1e-5 of the
    largest |J| there;
  - a6: the oracle's Yee update of the whole mesh from the read-back E, B
    and the GPU's current: every E, B and left-boundary value within 1e-5
    of its vector's largest magnitude;
  - a property that holds at any size: the Gauss residual of the whole mesh
    stays within the FP32 round-off bound of the smaller tests.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
BOX_CELLS = (32, 16, 16)   # the checked box, centred on the axis in y and z
MARGIN = 3
SAMPLE = 200_000
VEC = {"e": ("ex", "ey", "ez"), "b": ("bx", "by", "bz")}


def _live(p):
    keep = p["ix"] >= 0
    return {k: v[keep] for k, v in p.items()}


def _subset(p, mask):
    return {k: v[mask] for k, v in p.items()}


def _pos(p):
    return (p["ix"] + p["ox"].astype(np.float64), p["iy"] + p["oy"].astype(np.float64),
            p["iz"] + p["oz"].astype(np.float64))


def test_full_size_step_against_oracle_samples():
    wl = W.CONFIG2
    parts = W.generate_particles(wl)
    cfg = pic.config_from_workload(wl, sort_every=64, bins=(25, 16))
    sim = pic.Simulation(cfg)
    try:
        sim.set_particles(0, parts[0])
        sim.capture_background()
        del parts
        dt = sim.grid()[0]
        start = int(math.ceil(wl.t_peak_periods * 2 * math.pi / dt)) + 40
        sim.step(start)
        assert sim.binned(0)
        fa = sim.get_fields()
        pa = _live(sim.get_particles(0))
        sim.push_deposit()           # re-bins (the read-back compacted), then the binned fused kernel
        fj = sim.get_fields()
        sim.field_update()
        fb = sim.get_fields()
        pb = _live(sim.get_particles(0))
        r_max, _ = sim.gauss_residual()
        _, dx, dy, dz = sim.grid()
    finally:
        sim.close()
    n = len(pa["ix"])
    assert n > 60_000_000
    assert np.abs(fa["ey"]).max() > 1.0, "the pulse should be in the box"

    # a1-a5 on a sample and on the box: along x, the 32-cell stretch of the
    # axis whose particles move fastest (where the pulse drives them)
    rng = np.random.default_rng(7)
    x, y, z = _pos(pa)
    bx, by, bz = BOX_CELLS
    y0, z0 = wl.ny // 2 - by // 2, wl.nz // 2 - bz // 2
    y1, z1 = y0 + by, z0 + bz
    axis = (y >= y0 - MARGIN) & (y < y1 + MARGIN) & (z >= z0 - MARGIN) & (z < z1 + MARGIN)
    speed = np.sqrt(pa["ux"].astype(np.float64) ** 2 + pa["uy"] ** 2 + pa["uz"] ** 2)
    best, x0 = -1.0, None
    for xs in range(MARGIN + 2, wl.nx - bx - MARGIN - 2, bx // 2):
        m = axis & (x >= xs - MARGIN) & (x < xs + bx + MARGIN)
        if m.sum() > 1000 and speed[m].mean() > best:
            best, x0 = float(speed[m].mean()), xs
    assert x0 is not None, "no populated stretch on the axis"
    x1 = x0 + bx
    near = axis & (x >= x0 - MARGIN) & (x < x1 + MARGIN)
    pick = np.zeros(n, bool)
    pick[rng.choice(n, SAMPLE, replace=False)] = True
    sub = _subset(pa, pick | near)
    box_only = _subset(pa, near)
    fields = {k: fa[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    fields["byL"], fields["bzL"] = fa["by_left"], fa["bz_left"]

    with oracle.parallel():
        orc = oracle.OracleSim(wl, [sub], fields=fields, step=start)
        old = orc.push(0)
        orc.deposit(0, *old)     # a5 also removes the particles that left the region
    op = orc.p[0]
    order_b = np.argsort(pb["id"])
    ids_b = pb["id"][order_b]
    pos = np.minimum(np.searchsorted(ids_b, op["id"]), len(ids_b) - 1)
    found = ids_b[pos] == op["id"]
    alive = op["alive"].astype(bool)
    assert np.array_equal(found, alive), "removed sets differ"
    gb = _subset(pb, order_b[pos[alive]])
    gx, gy, gz = _pos(gb)
    for a, g in (("x", gx), ("y", gy), ("z", gz)):
        assert np.abs(g - op[a][alive]).max() <= TOL, a
    # u relative to the larger of |u| before and after the step (floor 1e-3):
    # where the step's impulse cancels most of u, FP32 rounds at the scale of
    # the terms, not of their small sum
    u_old = np.sqrt(sub["ux"][alive].astype(np.float64) ** 2 + sub["uy"][alive] ** 2 + sub["uz"][alive] ** 2)
    u_new = np.sqrt(op["ux"][alive] ** 2 + op["uy"][alive] ** 2 + op["uz"][alive] ** 2)
    scale = np.maximum(np.maximum(u_old, u_new), 1e-3)
    for k in ("ux", "uy", "uz"):
        d = np.abs(gb[k] - op[k][alive]) / scale
        assert d.max() <= TOL, (k, float(d.max()))
    for k in ("sx", "sy", "sz"):
        assert np.abs(gb[k] - op[k][alive]).max() <= TOL, k
    hot = np.sqrt(op["ux"] ** 2 + op["uy"] ** 2 + op["uz"] ** 2)
    assert (hot > 0.1).sum() > 1000, "the sample should hold driven particles"
    del orc

    with oracle.parallel():
        orc = oracle.OracleSim(wl, [box_only], fields=fields, step=start)
        orc.zero_current()
        old = orc.push(0)
        orc.deposit(0, *old)
    sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
    jmax = max(np.abs(orc.f[k][sl]).max() for k in ("jx", "jy", "jz"))
    assert jmax > 0
    for k in ("jx", "jy", "jz"):
        assert np.abs(fj[k][sl] - orc.f[k][sl]).max() <= TOL * jmax, k
    del orc

    # a6 on the whole mesh
    empty = {k: np.zeros(0, np.int32 if k in ("ix", "iy", "iz", "id") else np.float32) for k in pa}
    mesh = dict(fields)
    for k in ("jx", "jy", "jz"):
        mesh[k] = fj[k]
    with oracle.parallel():
        orc = oracle.OracleSim(wl, [empty], fields=mesh, step=start)
        orc.field_update()
    for kind, keys in VEC.items():
        vmax = max(np.abs(orc.f[k]).max() for k in keys)
        for k in keys:
            assert np.abs(fb[k] - orc.f[k]).max() <= TOL * vmax, k
    bmax = max(np.abs(orc.f[k]).max() for k in ("byL", "bzL"))
    assert np.abs(fb["by_left"] - orc.f["byL"]).max() <= TOL * max(bmax, 1e-30)
    assert np.abs(fb["bz_left"] - orc.f["bzL"]).max() <= TOL * max(bmax, 1e-30)

    # Gauss's law at full size
    emax = max(np.abs(fb[k]).max() for k in ("ex", "ey", "ez"))
    n0 = wl.species[0].n0
    bound = 4 * np.finfo(np.float32).eps * (emax * (1 / dx + 1 / dy + 1 / dz) + n0) * math.sqrt(start + 1)
    assert r_max < bound, (r_max, bound)
