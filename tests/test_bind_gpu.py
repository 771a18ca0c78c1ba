"""pic_bind_buffers: torch tensors as the context's state.

  - bound at creation (2D3V, compact layout with sorts) and in the middle of
    a run (3D3V, binned layout): the run goes on as an unbound twin's does
    (particles and fields to float rounding of the current sums) and follows
    the oracle;
  - the tensors are the state: the current buffer's tensors, ordered by id,
    equal pic_get_particles bit for bit, and the mesh tensors pic_get_fields;
  - pointers that are not device memory of the context's device, or not
    16-byte aligned, are refused and nothing changes.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import compare_fields, compare_particles, make_pair, rel_max

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FIELDS = ("ex", "ey", "ez", "bx", "by", "bz")


def _twins(wl, **kw):
    a, orc, parts = make_pair(wl, **kw)
    b, _, _ = make_pair(wl, parts=parts, **kw)
    return a, b, orc


def _same_run(a, b, orc, nsp):
    fa, fb = a.get_fields(), b.get_fields()
    for k in FIELDS:
        assert rel_max(fb[k].astype(float), fa[k].astype(float)) <= 1e-4, k
    for s in range(nsp):
        compare_particles(b, orc, s, 1e-4, 1e-4, 1e-4)
    compare_fields(b, orc, FIELDS, 1e-4)


def _views_are_state(sim):
    views = sim.particle_views(0)
    g = sim.get_particles(0)
    g = {k: v[g["ix"] >= 0] for k, v in g.items()}
    order = np.argsort(g["id"])
    ids = views["id"].cpu().numpy()
    live = views["cell"].cpu().numpy() != -1
    vo = np.argsort(ids[live])
    assert np.array_equal(ids[live][vo], g["id"][order])
    for k in ("ux", "uy", "uz", "sx", "sy", "sz", "w"):
        assert np.array_equal(views[k].cpu().numpy()[live][vo], g[k][order]), k
    f = sim.get_fields()
    eb = sim._bound["eb"].cpu().numpy()[..., :sim.nx]
    for c, k in enumerate(FIELDS):
        assert np.array_equal(eb[c].reshape(f[k].shape), f[k]), k


def test_bound_at_creation_2d():
    wl = W.small_case(nx=64, ny=32, ppc=3, u_th=0.2, a0=3.0)
    a, orc, parts = make_pair(wl, sort_every=5)
    b = pic.Simulation(pic.config_from_workload(wl, sort_every=5))
    try:
        b.bind_torch()
        b.set_particles(0, parts[0])
        b.capture_background()
        for sim in (a, b):
            sim.step(16)
        orc.step(16)
        _same_run(a, b, orc, 1)
        _views_are_state(b)
    finally:
        a.close()
        b.close()


def test_bound_mid_run_3d_binned():
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, u_th=0.3, a0=3.0)
    a, b, orc = _twins(wl, sort_every=8, bins=(25, 16))
    try:
        for sim in (a, b):
            sim.step(7)
        b.bind_torch()
        for sim in (a, b):
            sim.step(9)
        orc.step(16)
        assert b.binned(0)
        _same_run(a, b, orc, 1)
        _views_are_state(b)
    finally:
        a.close()
        b.close()


def test_bind_refuses_foreign_misaligned_or_overlapping_memory():
    wl = W.small_case(nx=32, ny=16, ppc=1)
    sim, orc, _ = make_pair(wl)
    try:
        ld, plane, rb, caps = sim.buffer_sizes()
        assert ld >= wl.nx and plane == ld * wl.ny and rb == 4 and caps[0] > 0
        before = sim.get_fields()
        host = np.zeros(6 * plane + 4, np.float32)
        bad = torch.zeros(6 * plane + 8, dtype=torch.float32, device="cuda")
        for ptr in (host.ctypes.data, bad.data_ptr() + 4):
            b = pic.pic_buffers_t()
            b.eb = ptr
            with pytest.raises(pic.PicError) as e:
                sim._c(pic.load().pic_bind_buffers(sim.h, C.byref(b), sim._s))
            assert e.value.status == -1
        # arrays that would share bytes once bound: E/B and J from one
        # tensor 16 bytes apart, and E/B over a species array
        big = torch.zeros(9 * plane + 64, dtype=torch.float32, device="cuda")
        rec = torch.zeros(caps[0] + 64, dtype=torch.float32, device="cuda")
        b = pic.pic_buffers_t()
        b.eb, b.j = big.data_ptr(), big.data_ptr() + 16
        with pytest.raises(pic.PicError) as e:
            sim._c(pic.load().pic_bind_buffers(sim.h, C.byref(b), sim._s))
        assert e.value.status == -1 and "overlap" in str(e.value)
        b = pic.pic_buffers_t()
        b.eb = big.data_ptr()
        b.sp[0][1].ux = big.data_ptr() + 4 * plane
        b.sp[0][1].uy = rec.data_ptr()
        with pytest.raises(pic.PicError) as e:
            sim._c(pic.load().pic_bind_buffers(sim.h, C.byref(b), sim._s))
        assert e.value.status == -1 and "overlap" in str(e.value)
        after = sim.get_fields()
        for k in FIELDS:
            assert np.array_equal(before[k], after[k])
        sim.step(3)
        orc.step(3)
        compare_particles(sim, orc, 0, 1e-4, 1e-4, 1e-4)
    finally:
        sim.close()
