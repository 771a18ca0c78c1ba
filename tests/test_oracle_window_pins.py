"""Pins of the oracle's co-moving window (Sec. 2: the box follows the laser).

A shift of the box by n cells is a change of coordinates: with nothing near
the edges it must commute with the update (a run shifted half way equals the
unshifted run read n cells further on), particles move by exactly -n cells,
and a neutral plasma that enters through the right end keeps Gauss's law.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W

E_B = ("ex", "ey", "ez", "bx", "by", "bz")


def _pulse_case(dim):
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.0, ppc=0, u_th=0.0, s0=(1, 0, 0))
    wl = W.Workload(name="pulse", nx=160, ny=8, dx_lambda=1 / 16, dy_lambda=1 / 8, cfl=0.9, steps=1,
                    species=(sp,), bc_x="open", pol="none")
    if dim == 3:
        wl = dataclasses.replace(wl, dim=3, nz=6, dz_lambda=1 / 8)
    return wl


def _empty(dim):
    keys = ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w") + (("oz",) if dim == 3 else ())
    d = {k: np.zeros(0, np.float32) for k in keys}
    d.update(ix=np.zeros(0, np.int32), iy=np.zeros(0, np.int32), id=np.zeros(0, np.int32))
    if dim == 3:
        d["iz"] = np.zeros(0, np.int32)
    return [d]


@pytest.mark.parametrize("dim", [2, 3])
def test_shift_commutes_with_vacuum_update(oracle_mod, dim):
    # a right-moving pulse with a transverse structure, far from both ends
    wl = _pulse_case(dim)
    sims = [oracle_mod.OracleSim(wl, _empty(dim)) for _ in range(2)]
    g = sims[0].grid
    xn = np.arange(wl.nx) * g.dx
    xh = (np.arange(wl.nx) + 0.5) * g.dx
    yn = np.arange(wl.ny) * g.dy
    tr = (1 + 0.3 * np.cos(2 * np.pi * yn / (wl.ny * g.dy)))[:, None]
    for s in sims:
        s.f["ey"][...] = np.exp(-((xn - 60 * g.dx) / (8 * g.dx)) ** 2)[None, :] * tr
        s.f["bz"][...] = np.exp(-((xh - 60 * g.dx) / (8 * g.dx)) ** 2)[None, :] * tr
    a, b = sims
    n = 12
    a.step(20)
    b.step(20)
    b.shift_window(n)
    a.step(25)
    b.step(25)
    # B's new x_min is a Silver-Mueller boundary where A has interior: the weak
    # left-moving part the transverse structure sheds differs there and spreads
    # at most one cell a step (courant number < 1); beyond that reach the runs agree
    lo = 26
    for k in E_B:
        np.testing.assert_allclose(b.f[k][..., lo:wl.nx - n - 4], a.f[k][..., lo + n:wl.nx - 4], atol=1e-14,
                                   err_msg=k)
    assert np.abs(a.f["ey"][..., lo + n:]).max() > 0.5


@pytest.mark.parametrize("dim", [2, 3])
def test_shift_moves_particles_by_n_cells_and_removes_the_left_ones(oracle_mod, dim):
    wl = W.small_case(nx=40, ny=12, ppc=2, u_th=0.01) if dim == 2 else \
        W.small_case3(nx=40, ny=8, nz=6, ppc=2, u_th=0.01)
    f = W.random_fields(wl, seed=3)
    sim = oracle_mod.OracleSim(wl, W.generate_particles(wl), fields=f)
    x0 = sim.p[0]["x"].copy()
    rest = {k: sim.p[0][k].copy() for k in ("y", "ux", "sz", "id")}
    sim.shift_window(5)
    # the mesh slides 5 columns toward x_min; the uncovered columns are the
    # unperturbed plasma ahead of the box (zero field)
    for k in E_B:
        np.testing.assert_array_equal(sim.f[k][..., :-5], f[k][..., 5:])
        assert np.all(sim.f[k][..., -5:] == 0.0)
    np.testing.assert_array_equal(sim.p[0]["x"], x0 - 5)
    np.testing.assert_array_equal(sim.p[0]["alive"], (x0 - 5 >= 2).astype(np.int32))
    for k, v in rest.items():
        np.testing.assert_array_equal(sim.p[0][k], v)


@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_law_across_shifts_with_injected_plasma(oracle_mod, dim):
    # cold neutral plasma (no particle reaches the open x_max) with the laser
    # entering; the box moves twice and fresh plasma with its immobile ions
    # fills the uncovered columns
    if dim == 2:
        wl = W.small_case(nx=64, ny=16, ppc=2, a0=3.0, u_th=0.0)
    else:
        wl = W.small_case3(nx=48, ny=10, nz=8, ppc=2, a0=3.0, u_th=0.0)
    sim = oracle_mod.OracleSim(wl, W.generate_particles(wl))
    n0 = sum(len(p["x"]) for p in sim.p)
    idb = n0
    for shift in (6, 10):
        sim.step(12)
        inj = W.injection_particles(wl, shift, seed=100 + shift, id_base=idb)
        idb += len(inj[0]["ix"])
        sim.shift_window(shift, inj)
        assert np.abs(sim.gauss_residual()).max() < 1e-12
    sim.step(12)
    assert np.abs(sim.f["ey"]).max() > 0.3
    assert np.abs(sim.gauss_residual()).max() < 1e-11
    assert len(sim.p[0]["x"]) == idb


@pytest.mark.parametrize("dim", [2, 3])
def test_shift_relabels_columns_and_keeps_injected_ids(oracle_mod, dim):
    # with every mesh value equal to its column index, a shift by n leaves
    # column i holding i + n (the uncovered n columns at zero), and the left
    # boundary values By(-1/2), Bz(-1/2) are those of the column that now sits
    # at x = -1/2: old column n - 1.  Injected plasma keeps the ids it was
    # given.
    wl = _pulse_case(dim)
    sim = oracle_mod.OracleSim(wl, _empty(dim))
    n = 10
    col = np.arange(wl.nx, dtype=float)
    for k in sim.FIELD_KEYS:
        sim.f[k][...] = col
    inj = W.injection_particles(dataclasses.replace(wl, species=(dataclasses.replace(wl.species[0], ppc=1),)),
                                n, seed=3, id_base=5000)
    sim.shift_window(n, inj)
    for k in sim.FIELD_KEYS:
        np.testing.assert_array_equal(sim.f[k][..., :-n], np.broadcast_to(col[n:], sim.f[k][..., :-n].shape))
        assert np.all(sim.f[k][..., -n:] == 0.0)
    assert np.all(sim.f["byL"] == n - 1) and np.all(sim.f["bzL"] == n - 1)
    ids = np.sort(sim.p[0]["id"])
    np.testing.assert_array_equal(ids, 5000 + np.arange(len(inj[0]["id"])))
    # and sit where they were given, cell plus offset, in the moved box
    o = np.argsort(sim.p[0]["id"])
    np.testing.assert_array_equal(sim.p[0]["x"][o], inj[0]["ix"] + inj[0]["ox"].astype(np.float64))
    np.testing.assert_array_equal(sim.p[0]["y"][o], inj[0]["iy"] + inj[0]["oy"].astype(np.float64))
