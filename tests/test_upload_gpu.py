"""pic_set_particles from pinned host arrays (read in place by the upload
kernel) against the same particles from pageable arrays (copied, then packed):
the same state bit for bit in 2D3V and 3D3V, FP32 and FP64 contexts, from
float32 and float64 host arrays; a cell outside the particle region is
rejected by both paths."""
import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

INT = ("ix", "iy", "iz", "id")


def _pinned(d, dtype):
    keep, ptrs = [], {}
    for k, v in d.items():
        a = np.ascontiguousarray(v, dtype=np.int32 if k in INT else dtype)
        t = torch.from_numpy(a).pin_memory()
        keep.append(t)
        ptrs[k] = t.data_ptr()
    return keep, ptrs


def _state(sim, f64):
    g = sim.get_particles_f64(0) if f64 else sim.get_particles(0)
    o = np.argsort(g["id"])
    return {k: v[o] for k, v in g.items()}


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("three", [False, True], ids=["2d3v", "3d3v"])
def test_pinned_upload_equals_copied_upload(three, precision):
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2, u_th=0.3) if three else W.small_case(nx=64, ny=32, ppc=3,
                                                                                          u_th=0.3)
    d = W.generate_particles(wl)[0]
    keys = ("ix", "iy", "ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w", "id") + (("iz", "oz") if three else ())
    d = {k: d[k] for k in keys}
    for host in (np.float32, np.float64):
        sims = []
        for pinned in (False, True):
            sim = pic.Simulation(pic.config_from_workload(wl, precision=precision))
            if pinned:
                keep, ptrs = _pinned(d, host)
                if host is np.float32:
                    sim.set_particles_raw(0, len(d["ix"]), ptrs)
                else:
                    sim.set_particles_f64_raw(0, len(d["ix"]), ptrs)
                del keep
            elif host is np.float32:
                sim.set_particles(0, d)
            else:
                sim.set_particles_f64(0, d)
            sims.append(sim)
        try:
            a, b = (_state(s, True) for s in sims)
            for k in a:
                assert np.array_equal(a[k], b[k]), (k, host)
        finally:
            for s in sims:
                s.close()


def test_pinned_upload_rejects_a_cell_outside_the_region():
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=1)
    d = dict(W.generate_particles(wl)[0])
    d["iz"] = d["iz"].copy()
    d["iz"][5] = wl.nz
    sim = pic.Simulation(pic.config_from_workload(wl))
    try:
        keep, ptrs = _pinned(d, np.float32)
        with pytest.raises(pic.PicError) as e:
            sim.set_particles_raw(0, len(d["ix"]), ptrs)
        assert e.value.status == -1
        assert sim.count(0) == 0
    finally:
        sim.close()
