"""GPU parity at the edges of the accepted inputs, against the FP64 oracle.

- The smallest meshes the library accepts (2D3V 8 x 4, 3D3V 8 x 4 x 4).
  There the tile and its field window are wider than the mesh, so window
  rows wrap onto the mesh more than once (periodic axes) or lie outside it
  (open x). Covered: both layouts, both boundary kinds, and tiles wider than
  the mesh.
- A species with no particles beside one with particles.
- A single particle that crosses a cell face on every axis in every step.
- A species whose particles all leave the box, stepped on once they are gone.

Tolerances as in the parity tests. After one step from a common state: u
relative 1e-5 (floor 1e-3 on |u|), s absolute 1e-5, x 1e-5 cells, and J, E, B
element-wise against their vector's magnitude. After further steps: 1e-4.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from pichelp import compare_fields, compare_particles, make_pair

pytestmark = pytest.mark.gpu

EB = ("ex", "ey", "ez", "bx", "by", "bz")


def _step_compared(sim, orc):
    """One step of the library (fused push and deposit, then the Yee update)
    and of the oracle from the same state, compared after each half."""
    sim.push_deposit()
    orc.zero_current()
    saved = [orc.push(s) for s in range(len(orc.p))]
    for s, old in enumerate(saved):
        orc.deposit(s, *old)
    for s in range(len(orc.p)):
        compare_particles(sim, orc, s, 1e-5, 1e-5, 1e-5)
    compare_fields(sim, orc, ("jx", "jy", "jz"), 1e-5)
    sim.field_update()
    orc.field_update()
    keys = EB + (("by_left", "bz_left") if orc.wl.bc_x == "open" else ())
    compare_fields(sim, orc, keys, 1e-5)


def _more_steps_compared(sim, orc, n):
    sim.step(n)
    orc.step(n)
    for s in range(len(orc.p)):
        compare_particles(sim, orc, s, 1e-4, 1e-4, 1e-4)
    compare_fields(sim, orc, EB, 1e-4)


MIN2 = [
    ("open-8x4tile", dict(bc_x="open"), None),
    ("open-32x8tile", dict(bc_x="open"), (32, 8)),
    ("periodic-16x8tile", dict(bc_x="periodic", pol="none"), (16, 8)),
]


@pytest.mark.parametrize("kw,tile", [(k, t) for _, k, t in MIN2], ids=[i for i, _, _ in MIN2])
def test_smallest_2d_mesh(kw, tile):
    wl = W.small_case(nx=8, ny=4, ppc=3, u_th=0.3, **kw)
    f = W.random_fields(wl, seed=41)
    sim, orc, _ = make_pair(wl, fields=f, step=3, tile=tile, sort_every=2)
    _step_compared(sim, orc)
    _more_steps_compared(sim, orc, 5)


MIN3 = [
    ("open-compact", dict(bc_x="open"), None, None),
    ("periodic-compact", dict(bc_x="periodic", pol="none"), None, None),
    ("open-binned", dict(bc_x="open"), None, (25, 16)),
    ("periodic-binned", dict(bc_x="periodic", pol="none"), None, (25, 16)),
    ("periodic-binned-8x8x4", dict(bc_x="periodic", pol="none"), (8, 8, 4), (25, 16)),
]


@pytest.mark.parametrize("kw,tile,bins", [(k, t, b) for _, k, t, b in MIN3], ids=[i for i, *_ in MIN3])
def test_smallest_3d_mesh(kw, tile, bins):
    wl = W.small_case3(nx=8, ny=4, nz=4, ppc=2, u_th=0.3, **kw)
    f = W.random_fields(wl, seed=42)
    sim, orc, _ = make_pair(wl, fields=f, step=3, tile=tile, bins=bins, sort_every=2)
    _step_compared(sim, orc)
    _more_steps_compared(sim, orc, 5)


def _with_empty_second_species(wl):
    """The workload's two species, the second with no particles (ppc 0)."""
    e, p = wl.species
    return dataclasses.replace(wl, species=(e, dataclasses.replace(p, ppc=0, colocate_with=-1)))


@pytest.mark.parametrize("dim,bins", [(2, None), (3, None), (3, (25, 16))], ids=["2d", "3d-compact", "3d-binned"])
def test_empty_species_beside_a_populated_one(dim, bins):
    base = (W.small_case(nx=40, ny=24, ppc=2, u_th=0.3, two_species=True) if dim == 2 else
            W.small_case3(nx=26, ny=18, nz=13, ppc=2, u_th=0.3, two_species=True))
    wl = _with_empty_second_species(base)       # capacity 0 for the second species
    parts = W.generate_particles(base)
    parts[1] = {k: v[:0].copy() for k, v in parts[1].items()}
    f = W.random_fields(wl, seed=43)
    sim, orc, _ = make_pair(wl, fields=f, step=2, bins=bins, sort_every=3, parts=parts)
    assert len(parts[0]["ix"]) > 0
    _step_compared(sim, orc)
    _more_steps_compared(sim, orc, 6)
    assert len(sim.get_particles(1)["id"]) == 0
    m = sim.polarization(1)
    assert m["count"] == 0 and m["sum_w"] == 0
    assert list(m["P"]) == [0.0, 0.0, 0.0]


def _single(wl, cell, offs, u):
    """One electron at cell + offs with momentum u, spin +y."""
    three = wl.dim == 3
    d = dict(ix=np.array([cell[0]], np.int32), iy=np.array([cell[1]], np.int32),
             ox=np.array([offs[0]], np.float32), oy=np.array([offs[1]], np.float32),
             ux=np.array([u[0]], np.float32), uy=np.array([u[1]], np.float32),
             uz=np.array([u[2]], np.float32), sx=np.zeros(1, np.float32), sy=np.ones(1, np.float32),
             sz=np.zeros(1, np.float32), w=np.array([0.05], np.float32), id=np.zeros(1, np.int32))
    if three:
        d["iz"] = np.array([cell[2]], np.int32)
        d["oz"] = np.array([offs[2]], np.float32)
    return [d]


SINGLE = [
    ("2d", 2, None),
    ("3d-compact", 3, None),
    ("3d-binned", 3, (25, 16)),
]


@pytest.mark.parametrize("dim,bins", [(d, b) for _, d, b in SINGLE], ids=[i for i, _, _ in SINGLE])
def test_single_particle_crossing_every_axis(dim, bins):
    # u = (3, -2, 1.5): about 0.5 cell along +x, 0.25 along -y and 0.15 along
    # +z a step on these meshes; starting near the (+x, -y, +z) corner of its
    # cell it crosses a face on every axis in the first step
    if dim == 2:
        wl = W.small_case(nx=12, ny=8, ppc=1, bc_x="periodic", pol="none")
        parts = _single(wl, (10, 0), (0.8, 0.1), (3.0, -2.0, 1.5))
    else:
        wl = W.small_case3(nx=12, ny=8, nz=4, ppc=1, bc_x="periodic", pol="none")
        parts = _single(wl, (10, 0, 3), (0.8, 0.1, 0.9), (3.0, -2.0, 1.5))
    f = W.random_fields(wl, seed=44, e_amp=0.05, b_amp=0.2)
    sim, orc, _ = make_pair(wl, fields=f, parts=parts, bins=bins, sort_every=2)
    pos = ("x", "y", "z") if dim == 3 else ("x", "y")
    x0 = [orc.p[0][a][0] for a in pos]
    _step_compared(sim, orc)
    x1 = [orc.p[0][a][0] for a in pos]
    assert all(np.floor(a) != np.floor(b) for a, b in zip(x0, x1)), "case should cross a face on every axis"
    _more_steps_compared(sim, orc, 9)


@pytest.mark.parametrize("dim,bins", [(2, None), (3, None), (3, (25, 16))], ids=["2d", "3d-compact", "3d-binned"])
def test_species_that_leaves_the_box_entirely(dim, bins):
    # every particle drifts along -x at about 0.7 cells a step and leaves at
    # the open x_min; the steps after the last removal run on an empty species
    wl = (W.small_case(nx=12, ny=4, ppc=2, u_th=0.0, pol="none") if dim == 2 else
          W.small_case3(nx=12, ny=4, nz=4, ppc=2, u_th=0.0, pol="none"))
    parts = W.generate_particles(wl)
    parts[0]["ux"][:] = np.float32(-5.0)
    sim, orc, _ = make_pair(wl, parts=parts, bins=bins, sort_every=4)
    _step_compared(sim, orc)
    _more_steps_compared(sim, orc, 13)
    assert not orc.p[0]["alive"].any(), "case should remove every particle"
    assert sim.polarization(0)["count"] == 0
    _more_steps_compared(sim, orc, 4)


@pytest.mark.parametrize("dim,bins", [(2, None), (3, (25, 16))], ids=["2d", "3d-binned"])
def test_smallest_meshes_fp64(dim, bins):
    # the FP64 instantiation at the smallest meshes, periodic on every axis,
    # agrees with the oracle to FP64 rounding
    wl = (W.small_case(nx=8, ny=4, ppc=3, u_th=0.3, bc_x="periodic", pol="none") if dim == 2 else
          W.small_case3(nx=8, ny=4, nz=4, ppc=2, u_th=0.3, bc_x="periodic", pol="none"))
    f = W.random_fields(wl, seed=45)
    sim, orc, _ = make_pair(wl, fields=f, step=1, bins=bins, sort_every=2, precision=64)
    for _ in range(3):
        sim.step(1)
        orc.step(1)
    compare_particles(sim, orc, 0, 1e-11, 1e-11, 1e-11, f64=True)
    compare_fields(sim, orc, EB, 1e-11, f64=True)
