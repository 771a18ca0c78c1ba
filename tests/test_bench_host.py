"""Host-side arithmetic of bench.py's roofline line, against the algorithmic
bytes the method fixes for the fused a1-a5 kernel: per particle read cell,
offsets, u (3), s (3), w and write cell, offsets, u, s; per cell the E, B
window and the current added to J.  Also: the DRAM traffic record is used
only for the kernel source it was measured on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def _count(dim, real):
    """Algorithmic bytes per particle and per cell, counted field by field."""
    offsets = dim                   # ox, oy (, oz)
    read = 4 + real * (offsets + 3 + 3 + 1)
    write = 4 + real * (offsets + 3 + 3)
    cell = real * (6 + 3)           # E, B read (6 components), J added (3)
    return read + write, cell


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", [32, 64])
def test_fused_bytes_follow_the_field_count(dim, precision):
    per_p, per_c = _count(dim, precision // 8)
    alg, lay = bench.fused_bytes(dim, 1000, 10, precision, False)
    assert alg == per_p * 1000 + per_c * 10
    assert lay == 0


def test_fused_bytes_fp32_values():
    # 76 B (2D3V) and 84 B (3D3V) a particle, 36 B a cell; the binned layout's
    # id read and w, id writes (12 B) reported apart
    assert bench.fused_bytes(2, 1, 0, 32, False) == (76, 0)
    assert bench.fused_bytes(3, 1, 0, 32, False) == (84, 0)
    assert bench.fused_bytes(3, 0, 1, 32, False) == (36, 0)
    assert bench.fused_bytes(3, 1, 0, 32, True) == (84, 12)
    assert bench.fused_bytes(3, 1, 0, 64, True) == (160, 16)


def test_config2_launch_bytes():
    # 66,584,576 electrons on 512 x 256 x 256 cells: 6.80 GB a launch
    n = 2 * (512 - 4) * 256 * 256
    alg, _ = bench.fused_bytes(3, n, 512 * 256 * 256, 32, True)
    assert n == 66_584_576
    assert alg == 84 * n + 36 * 33_554_432
    assert alg / 1e9 == pytest.approx(6.80, abs=0.005)


def test_traffic_record_only_for_its_source(tmp_path, monkeypatch):
    wl = W.CONFIG2
    rec = {"kernel": "k_step_fused3", "workload": wl.name, "dram_bytes_per_launch": 123,
           "source_sha256": bench.kernel_source_hash(3)}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_step_fused3_binned.traffic.json").write_text(json.dumps(rec))
    # the hash covers the sources under the repository; only the record moves
    real_hash = bench.kernel_source_hash(3)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda dim: real_hash)
    assert bench.traffic_record(3, wl, True)["dram_bytes_per_launch"] == 123
    assert bench.traffic_record(3, W.CONFIG3, True) is None          # another workload
    monkeypatch.setattr(bench, "kernel_source_hash", lambda dim: "0" * 64)
    assert bench.traffic_record(3, wl, True) is None                  # another kernel source


def _dt(wl):
    import math
    d = [wl.dx_lambda, wl.dy_lambda] + ([wl.dz_lambda] if wl.dim == 3 else [])
    return wl.cfl / math.sqrt(sum((1.0 / (2 * math.pi * v)) ** 2 for v in d))


def test_timed_region_starts_in_the_interaction_phase():
    # 40 steps after the envelope peak reaches x = 0: t_peak = 15 periods,
    # config 2 dt = 0.2597/omega0 -> step 363 + 40; config 3 dt = 0.1319 -> 715 + 40
    assert _dt(W.CONFIG2) == pytest.approx(0.2598, abs=1e-4)
    assert bench.interaction_start(W.CONFIG2, _dt(W.CONFIG2)) == 403
    assert bench.interaction_start(W.CONFIG3, _dt(W.CONFIG3)) == 755
    # no laser, no interaction phase to wait for
    import dataclasses
    assert bench.interaction_start(dataclasses.replace(W.CONFIG2, pol="none"), 0.26) == 0


def test_window_follows_the_envelope_peak():
    # the co-moving leg starts when the envelope peak reaches 3/4 of the box
    # (x = 384 cells of dx = lambda/20 in config 2): step 828
    assert bench.window_start(W.CONFIG2, _dt(W.CONFIG2), 0.75) == 828


def test_workload_particle_counts():
    # every cell but the two vacuum columns at each open x end, ppc per cell
    # and species: config 1 (256 x 128, 4 ppc) 129,024 electrons; config 2
    # (512 x 256 x 256, 2 ppc) 66,584,576; config 3 (4096 x 1024, 8 + 8 ppc)
    # 67,043,328 particles
    def count(wl):
        cols = wl.nx if wl.bc_x == "periodic" else wl.nx - 4
        return sum(sp.ppc * cols * wl.ny * (wl.nz if wl.dim == 3 else 1) for sp in wl.species)

    assert count(W.CONFIG1) == 129_024
    assert count(W.CONFIG2) == 66_584_576
    assert count(W.CONFIG3) == 67_043_328
    # and the generator draws exactly that many on a small cut of each
    for wl in (W.CONFIG1, W.scaled(W.CONFIG2, ny=8, nz=4), W.scaled(W.CONFIG3, nx=64, ny=8)):
        assert sum(len(d["ix"]) for d in W.generate_particles(wl)) == count(wl)
