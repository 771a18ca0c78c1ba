"""pic_moments_noalloc against pic_polarization.

pic_moments_noalloc is the variant of the Eq. (4) moments reduction for
callers that cannot have the library allocate device memory (graph capture,
caller-owned memory pools, loops that cannot take cudaMalloc's device-wide
synchronisation).  It keeps its partial sums in a fixed file-scope device
array.  This file is collected last so that a failure here cannot hide any
other test's result; it builds all of its own state, so it also passes when
run alone in a fresh process.
"""
import math

import numpy as np
import pytest

import paper_2002_02211_gb300 as pic
import workloads as W

pytestmark = pytest.mark.gpu


def _device_arrays(torch, g):
    cell = np.where(g["ix"] >= 0,
                    (g["iy"].astype(np.uint32) << np.uint32(16)) | g["ix"].astype(np.uint32),
                    np.uint32(0xFFFFFFFF)).astype(np.uint32)
    dev = {"cell": torch.from_numpy(cell.view(np.int32)).cuda()}
    for k in ("ux", "uy", "uz", "sx", "sy", "sz", "w"):
        dev[k] = torch.from_numpy(np.ascontiguousarray(g[k])).cuda()
    return dev


def test_moments_noalloc_matches_polarization_on_two_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    wl = W.small_case(nx=48, ny=32, ppc=4, u_th=0.5, two_species=True)
    parts = W.generate_particles(wl)
    fields = W.random_fields(wl, seed=9, e_amp=0.2, b_amp=0.8)
    with pic.Simulation(pic.config_from_workload(wl)) as sim:
        for s, d in enumerate(parts):
            sim.set_particles(s, d)
        sim.set_fields(fields)
        sim.step(3)          # some particles leave: removed slots are in the arrays
        out = torch.zeros(7, dtype=torch.float64, device="cuda")
        for s, sp in enumerate(wl.species):
            g = sim.get_particles(s)
            dev = _device_arrays(torch, g)
            n = len(g["ix"])
            for emin, emax in [(-math.inf, math.inf), (0.01, 0.2)]:
                ref = sim.polarization(s, emin, emax)
                for call in range(2):       # two calls in a row share the scratch array
                    out.fill_(float("nan"))
                    torch.cuda.synchronize()
                    pic.moments_noalloc(n, dev["cell"].data_ptr(), dev["ux"].data_ptr(),
                                        dev["uy"].data_ptr(), dev["uz"].data_ptr(),
                                        dev["sx"].data_ptr(), dev["sy"].data_ptr(),
                                        dev["sz"].data_ptr(), dev["w"].data_ptr(), sp.m, emin, emax,
                                        out.data_ptr(), stream=None)
                    torch.cuda.synchronize()
                    m = out.cpu().numpy()
                    np.testing.assert_allclose(m[:3], ref["P"], atol=1e-6)
                    assert m[3] == pytest.approx(ref["sum_w"], rel=1e-6)
                    assert m[4] == ref["count"]
                    assert m[5] == pytest.approx(ref["ekin_mean"], rel=1e-5)
                    assert m[6] == pytest.approx(ref["ekin_var"], rel=1e-4, abs=1e-300)


def test_moments_noalloc_rejects_sizes_beyond_the_maximum():
    with pytest.raises(pic.PicError) as e:
        pic.moments_noalloc(2 ** 31, 1, 1, 1, 1, 1, 1, 1, 1, 1.0, 0.0, 1.0, 1)
    assert e.value.status == -1 and "2^31" in str(e.value)


def test_moments_noalloc_count_slot_for_tiny_inputs():
    # the particle count the entry point stores on the device before the
    # reduction: an empty call must give zero moments, one live particle its own
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    dev = {k: torch.zeros(4, dtype=torch.float32, device="cuda") for k in ("ux", "uy", "uz", "sx", "sy", "sz", "w")}
    dev["cell"] = torch.zeros(4, dtype=torch.int32, device="cuda")
    ptrs = [dev[k].data_ptr() for k in ("cell", "ux", "uy", "uz", "sx", "sy", "sz", "w")]
    pic.moments_noalloc(0, *ptrs, 1.0, -math.inf, math.inf, out.data_ptr())
    torch.cuda.synchronize()
    assert out.cpu().numpy().tolist() == [0.0] * 7
    dev["sy"][0] = 1.0
    dev["w"][0] = 0.25
    pic.moments_noalloc(1, *ptrs, 1.0, -math.inf, math.inf, out.data_ptr())
    torch.cuda.synchronize()
    m = out.cpu().numpy()
    assert m[:3].tolist() == [0.0, 1.0, 0.0] and m[3] == 0.25 and m[4] == 1.0
