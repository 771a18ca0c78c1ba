"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/pic.h declares, and validates configurations on
the host (no CUDA call is made here)."""
import ctypes as C
import os
import re

import pytest

import paper_2002_02211_gb300 as pic
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:pic_status_t|void|const char\s*\*)\s*\*?\s*(pic_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pic_create", "pic_gather_push_spin", "pic_deposit", "pic_field_update",
                     "pic_step", "pic_polarization", "pic_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = pic.load()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header():
    for n in _declared():
        if n in ("pic_destroy", "pic_last_error", "pic_batch_destroy", "pic_batch_last_error"):
            continue
        assert n in pic._SIGS, n


def _status(cfg):
    return pic.load().pic_validate_config(C.byref(cfg))


def test_validate_config_accepts_the_workloads():
    for wl in (W.CONFIG1, W.CONFIG2, W.CONFIG3, W.small_case(), W.small_case(bc_x="periodic", two_species=True),
               W.small_case3()):
        assert _status(pic.config_from_workload(wl)) == 0


@pytest.mark.parametrize("field,value", [
    ("nx", 4), ("ny", 2), ("nx", 40000), ("cfl", 1.0), ("cfl", 0.0), ("dx_lambda", 0.0),
    ("bc_x", 7), ("pol", 9), ("nspecies", 0), ("nspecies", 5), ("sort_every", -1),
])
def test_validate_config_rejects(field, value):
    cfg = pic.config_from_workload(W.small_case())
    setattr(cfg, field, value)
    assert _status(cfg) == -1
    assert pic.load().pic_last_error(None)


def test_validate_config_rejects_bad_tiles_and_species():
    cfg = pic.config_from_workload(W.small_case())
    cfg.tile_x, cfg.tile_y = 6, 4        # not a compiled tile shape
    assert _status(cfg) == -1
    cfg.tile_x, cfg.tile_y = 32, 16
    assert _status(cfg) == 0
    cfg = pic.config_from_workload(W.small_case())
    cfg.sp[0].m = 0.0
    assert _status(cfg) == -1
    cfg = pic.config_from_workload(W.small_case())
    cfg.sp[0].capacity = -5
    assert _status(cfg) == -1


def test_validate_config_mesh_size_limits():
    # smallest accepted meshes, the largest per-axis sizes, and the 3D3V
    # bound on the mesh padded to whole tiles (the tile sort indexes its
    # cells with 32-bit signed keys)
    def cfg2(nx, ny):
        return pic.config_from_workload(W.small_case(nx=nx, ny=ny, ppc=1))

    def cfg3(nx, ny, nz, tile=None):
        return pic.config_from_workload(W.small_case3(nx=nx, ny=ny, nz=nz, ppc=1), tile=tile)

    assert _status(cfg2(8, 4)) == 0
    assert _status(cfg2(32767, 32767)) == 0
    for nx, ny in ((7, 4), (8, 3), (32768, 4), (8, 32768)):
        assert _status(cfg2(nx, ny)) == -1, (nx, ny)
    assert _status(cfg3(8, 4, 4)) == 0
    for dims in ((7, 4, 4), (8, 3, 4), (8, 4, 3), (2045, 4, 4), (8, 2045, 4), (8, 4, 1021)):
        assert _status(cfg3(*dims)) == -1, dims
    # default 16x4x4 tiles: 2044 x 1028 x 1020 pads to 2048 x 1028 x 1020 =
    # 2,147,450,880 cells (accepted), 2044 x 1029 x 1020 to 2048 x 1032 x 1020
    # = 2,155,806,720 > 2^31 - 1 (refused)
    assert _status(cfg3(2044, 1028, 1020)) == 0
    assert _status(cfg3(2044, 1029, 1020)) == -1
    assert "2^31" in pic.load().pic_last_error(None).decode()
    assert _status(cfg3(2044, 2044, 1020)) == -1
    # the padding follows the tile: 2020 columns pad to 2032 with 16-wide
    # tiles (2,138,964,480 cells with 1032 x 1020) and to 2048 with 32-wide ones
    assert _status(cfg3(2020, 1032, 1020)) == 0
    assert _status(cfg3(2020, 1032, 1020, tile=(32, 4, 4))) == -1


def test_validate_config_binned_layout():
    # binned layout: 3D3V only, headroom in [0, 400] %, spare slots in [0, 4096]
    cfg = pic.config_from_workload(W.small_case3(), bins=(25, 16))
    assert _status(cfg) == 0
    for field, value in (("bin_headroom_pct", -1), ("bin_headroom_pct", 401), ("bin_min_extra", -1),
                         ("bin_min_extra", 5000)):
        bad = pic.config_from_workload(W.small_case3(), bins=(25, 16))
        setattr(bad, field, value)
        assert _status(bad) == -1, field
    cfg2 = pic.config_from_workload(W.small_case())
    cfg2.bin_headroom_pct = 25
    assert _status(cfg2) == -1


def test_bin_capacity_covers_the_range_bound():
    # the binding's capacity for the binned layout holds the library's bound:
    # every tile range at count * (1 + pct/100) + extra + 7, plus the overflow range
    wl = W.small_case3(nx=40, ny=16, nz=12, ppc=2)
    cfg = pic.config_from_workload(wl, bins=(25, 16))
    n = 2 * (wl.nx - 4) * wl.ny * wl.nz
    ntiles = -(-wl.nx // 16) * -(-wl.ny // 4) * -(-wl.nz // 4)
    bound = n + n * 25 // 100 + ntiles * (16 + 7) + ((max(1024, n // 4) + 7) // 8) * 8
    assert cfg.sp[0].capacity >= bound


def test_moments_noalloc_checks_its_arguments_on_the_host():
    # the size limit is checked before any CUDA call: the largest accepted
    # count is 2^31 - 1 (the device loops index with 64 bits), one more is
    # refused, and so are a negative count and null pointers
    L = pic.load()
    args = [C.c_void_p(1)] * 8 + [C.c_double(1.0), C.c_double(0.0), C.c_double(1.0), C.c_void_p(1), None]
    for n in (2 ** 31, -1):
        assert L.pic_moments_noalloc(n, *args) == -1
        assert b"2^31" in L.pic_last_error(None)
    nulls = [None] * 8 + args[8:]
    assert L.pic_moments_noalloc(10, *nulls) == -1
    assert b"null" in L.pic_last_error(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # without libpic.so the binding raises; there is no other implementation
    # to fall back to
    missing = str(tmp_path / "libpic.so")
    monkeypatch.setattr(pic, "_lib", None)
    monkeypatch.setattr(pic, "LIB_PATH", missing)
    with pytest.raises(OSError, match="CUDA library not built"):
        pic.load(build=False)
    with pytest.raises(OSError):
        pic._check(-1)                      # any status lookup needs the library too
