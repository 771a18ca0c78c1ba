"""Python binding of libpic.so, the GB300 (sm_103a) 2D3V / 3D3V PIC + Thomas-BMT step.

Argument marshalling only: every function below calls the C entry point of
the same name declared in include/pic.h, and all arithmetic runs in the CUDA
kernels.  Device memory is owned by the library; CUDA streams come from
PyTorch (pass ``torch.cuda.current_stream()`` or any ``torch.cuda.Stream``)
or are None for the legacy default stream.

There is no CPU fallback: loading fails loudly if the library cannot be built
or opened.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

__all__ = ["PicError", "pic_config_t", "pic_species_t", "config_from_workload", "Simulation", "Batch",
           "load", "LIB_PATH"]

LIB_PATH = _build.LIB
MAX_SPECIES = 4
BC = {"open": 0, "periodic": 1}
POL = {"none": 0, "lp-y": 1, "cp": 2}
STATUS = {0: "PIC_OK", -1: "PIC_ERR_ARG", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_NAN", -4: "PIC_ERR_CFL",
          -5: "PIC_ERR_OVERFLOW", -6: "PIC_ERR_TIMEOUT", -7: "PIC_ERR_STATE"}


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class pic_species_t(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("a", C.c_double), ("mobile", C.c_int),
                ("capacity", C.c_int64)]


class pic_config_t(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx_lambda", C.c_double), ("dy_lambda", C.c_double),
                ("cfl", C.c_double), ("bc_x", C.c_int), ("pol", C.c_int), ("a0", C.c_double),
                ("waist_lambda", C.c_double), ("fwhm_periods", C.c_double),
                ("t_peak_periods", C.c_double), ("nspecies", C.c_int),
                ("sp", pic_species_t * MAX_SPECIES), ("sort_every", C.c_int), ("tile_x", C.c_int),
                ("tile_y", C.c_int), ("precision", C.c_int), ("dim", C.c_int), ("nz", C.c_int),
                ("dz_lambda", C.c_double), ("tile_z", C.c_int),
                ("bin_headroom_pct", C.c_int), ("bin_min_extra", C.c_int)]


_I32P = C.POINTER(C.c_int32)
_F32P = C.POINTER(C.c_float)


class pic_particles_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("ix", _I32P), ("iy", _I32P), ("ox", _F32P), ("oy", _F32P),
                ("ux", _F32P), ("uy", _F32P), ("uz", _F32P), ("sx", _F32P), ("sy", _F32P),
                ("sz", _F32P), ("w", _F32P), ("id", _I32P), ("iz", _I32P), ("oz", _F32P)]


_F64P = C.POINTER(C.c_double)

# record arrays of one particle buffer, in pic_particle_buffer_t order
_BUF_REALS = ("ox", "oy", "oz", "ux", "uy", "uz", "sx", "sy", "sz", "w")


class pic_particle_buffer_t(C.Structure):
    _fields_ = [("cell", C.c_void_p)] + [(k, C.c_void_p) for k in _BUF_REALS] + [("id", C.c_void_p)]


class pic_buffers_t(C.Structure):
    _fields_ = [("sp", (pic_particle_buffer_t * 2) * 4), ("eb", C.c_void_p), ("j", C.c_void_p)]


class pic_particles_f64_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("ix", _I32P), ("iy", _I32P)] + \
        [(k, _F64P) for k in ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w")] + \
        [("id", _I32P), ("iz", _I32P), ("oz", _F64P)]


class pic_fields_f64_t(C.Structure):
    _fields_ = [(k, _F64P) for k in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz",
                                     "by_left", "bz_left")]


class pic_fields_t(C.Structure):
    _fields_ = [(k, _F32P) for k in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz",
                                     "by_left", "bz_left")]


class pic_loss_t(C.Structure):
    _fields_ = [("species", C.c_int), ("axis", C.c_int), ("e_cut_mev", C.c_double), ("e_width_mev", C.c_double)]


class pic_moments_t(C.Structure):
    _fields_ = [("P", C.c_double * 3), ("sum_w", C.c_double), ("count", C.c_double),
                ("ekin_mean", C.c_double), ("ekin_var", C.c_double)]


_lib = None

_SIGS = {
    "pic_validate_config": [C.POINTER(pic_config_t)],
    "pic_create": [C.POINTER(pic_config_t), C.c_void_p, C.POINTER(C.c_void_p)],
    "pic_get_grid": [C.c_void_p] + [C.POINTER(C.c_double)] * 4,
    "pic_set_particles": [C.c_void_p, C.c_int, C.POINTER(pic_particles_t), C.c_void_p],
    "pic_get_count": [C.c_void_p, C.c_int, C.POINTER(C.c_int64)],
    "pic_set_particles_f64": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pic_get_particles": [C.c_void_p, C.c_int, C.POINTER(pic_particles_t), C.c_void_p],
    "pic_get_particles_f64": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pic_get_fields_f64": [C.c_void_p, C.c_void_p, C.c_void_p],
    "pic_set_fields": [C.c_void_p, C.POINTER(pic_fields_t), C.c_void_p],
    "pic_get_fields": [C.c_void_p, C.POINTER(pic_fields_t), C.c_void_p],
    "pic_set_step": [C.c_void_p, C.c_int64],
    "pic_get_step": [C.c_void_p, C.POINTER(C.c_int64)],
    "pic_gather_push_spin": [C.c_void_p, C.c_void_p],
    "pic_deposit": [C.c_void_p, C.c_void_p],
    "pic_field_update": [C.c_void_p, C.c_void_p],
    "pic_sort": [C.c_void_p, C.c_void_p],
    "pic_push_deposit": [C.c_void_p, C.c_void_p],
    "pic_step": [C.c_void_p, C.c_int, C.c_void_p],
    "pic_set_graphs": [C.c_void_p, C.c_int],
    "pic_graph_stats": [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "pic_launch_count": [C.c_void_p, C.POINTER(C.c_int64)],
    "pic_polarization": [C.c_void_p, C.c_int, C.c_double, C.c_double, C.POINTER(pic_moments_t),
                         C.c_void_p],
    "pic_capture_background": [C.c_void_p, C.c_void_p],
    "pic_energy_histogram": [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                             C.POINTER(C.c_double), C.c_void_p],
    "pic_gauss_residual": [C.c_void_p, C.POINTER(C.c_double), C.c_void_p],
    "pic_sync": [C.c_void_p, C.c_void_p],
    "pic_shift_window": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pic_loss": [C.c_void_p, C.POINTER(pic_loss_t), C.POINTER(C.c_double), C.c_void_p],
    "pic_adjoint": [C.c_void_p, C.c_int, C.c_int, C.POINTER(pic_loss_t), C.POINTER(C.c_double),
                    C.POINTER(C.c_double), C.c_void_p],
    "pic_adjoint_particle_grads": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pic_batch_create": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)],
    "pic_batch_run": [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)],
    "pic_batch_step": [C.c_void_p, C.c_int64, C.c_void_p],
    "pic_batch_steps_done": [C.c_void_p, C.c_void_p],
    "pic_batch_launch_count": [C.c_void_p, C.POINTER(C.c_int64)],
    "pic_batch_tune": [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pic_get_window": [C.c_void_p, C.POINTER(C.c_int64)],
    "pic_set_window": [C.c_void_p, C.c_int, C.c_int64, C.c_double],
    "pic_stage_injection": [C.c_void_p, C.c_void_p, C.c_void_p],
    "pic_staged_injections": [C.c_void_p, C.POINTER(C.c_int64)],
    "pic_get_layout": [C.c_void_p, C.c_int, C.POINTER(C.c_int)],
    "pic_buffer_sizes": [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                         C.POINTER(C.c_int64)],
    "pic_bind_buffers": [C.c_void_p, C.c_void_p, C.c_void_p],
    "pic_current_buffer": [C.c_void_p, C.c_int, C.POINTER(C.c_int)],
    "pic_set_diagnostics": [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
    "pic_get_diagnostics": [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p],
    "pic_moments_noalloc": [C.c_int64] + [C.c_void_p] * 8 + [C.c_double, C.c_double, C.c_double,
                                                              C.c_void_p, C.c_void_p],
}


def load(build: bool = True):
    """Opens libpic.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build:
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise OSError(f"CUDA library not built: {LIB_PATH}")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.pic_destroy.argtypes = [C.c_void_p]
        L.pic_destroy.restype = None
        L.pic_last_error.argtypes = [C.c_void_p]
        L.pic_last_error.restype = C.c_char_p
        L.pic_batch_destroy.argtypes = [C.c_void_p]
        L.pic_batch_destroy.restype = None
        L.pic_batch_last_error.argtypes = [C.c_void_p]
        L.pic_batch_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != 0:
        msg = load().pic_last_error(ctx)
        raise PicError(status, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        return None
    h = getattr(stream, "cuda_stream", stream)
    return C.c_void_p(int(h))


def moments_noalloc(n, cell, ux, uy, uz, sx, sy, sz, w, mass_me, emin, emax, out_dev, stream=None):
    """pic_moments_noalloc: every array argument is a device address (int)."""
    ptrs = [C.c_void_p(int(a)) for a in (cell, ux, uy, uz, sx, sy, sz, w)]
    _check(load().pic_moments_noalloc(int(n), *ptrs, float(mass_me), float(emin), float(emax),
                                      C.c_void_p(int(out_dev)), _stream(stream)))


def bin_capacity(n: int, ntiles: int, headroom_pct: int, min_extra: int) -> int:
    """Slots a mobile species of n particles needs for the binned 3D3V layout:
    every tile range grown by its headroom and rounded up to 8, plus the
    overflow range."""
    return int(n + n * headroom_pct // 100 + ntiles * (min_extra + 7) + max(1024, n // 4) + 8)


def config_from_workload(wl, capacity_factor: float = 1.0, sort_every: int = 0, tile=None,
                         precision: int = 32, bins=None, window_cells: int = 0):
    """pic_config_t for a workload description (nx, ny, dx_lambda, ..., species;
    dim, nz, dz_lambda for 3D3V).  tile: (tx, ty) in 2D3V, (tx, ty, tz) in
    3D3V, None for the library's choice.  bins: (headroom_pct, min_extra)
    turns on the binned 3D3V layout, with the mobile species' capacities
    grown to fit it.  window_cells: cells a move of the co-moving window
    takes in; the capacities then hold two moves' plasma more (the particle
    count may exceed the initial one between moves, and the live-count bound
    runs ahead of it until the device's count arrives)."""
    three = getattr(wl, "dim", 2) == 3
    cfg = pic_config_t()
    cfg.nx, cfg.ny = wl.nx, wl.ny
    cfg.dx_lambda, cfg.dy_lambda = wl.dx_lambda, wl.dy_lambda
    cfg.cfl = wl.cfl
    cfg.bc_x = BC[wl.bc_x]
    cfg.pol = POL[wl.pol]
    cfg.a0 = wl.a0
    cfg.waist_lambda = wl.waist_lambda
    cfg.fwhm_periods = wl.fwhm_periods
    cfg.t_peak_periods = wl.t_peak_periods
    cfg.nspecies = len(wl.species)
    ncx = wl.nx if wl.bc_x == "periodic" else wl.nx - 4
    for s, sp in enumerate(wl.species):
        cfg.sp[s].q, cfg.sp[s].m, cfg.sp[s].a = sp.q, sp.m, sp.a
        cfg.sp[s].mobile = 1 if sp.mobile else 0
        cross = wl.ny * (wl.nz if three else 1)
        cfg.sp[s].capacity = int(math.ceil(sp.ppc * (ncx * capacity_factor + 2 * window_cells) * cross))
    cfg.sort_every = sort_every
    tile = tuple(tile) if tile else (0, 0, 0)
    cfg.tile_x, cfg.tile_y = tile[0], tile[1]
    cfg.precision = precision
    if three:
        cfg.dim, cfg.nz, cfg.dz_lambda = 3, wl.nz, wl.dz_lambda
        cfg.tile_z = tile[2] if len(tile) > 2 else 0
        if bins:
            pct, extra = int(bins[0]), int(bins[1])
            cfg.bin_headroom_pct, cfg.bin_min_extra = pct, extra
            tx, ty, tz = (tile if tile[0] else (16, 4, 4))
            ntiles = -(-wl.nx // tx) * -(-wl.ny // ty) * -(-wl.nz // tz)
            for s, sp in enumerate(wl.species):
                if sp.mobile:
                    cfg.sp[s].capacity = bin_capacity(cfg.sp[s].capacity, ntiles, pct, extra)
    return cfg


def _ptr(a, t):
    return a.ctypes.data_as(t)


_INT_KEYS = ("ix", "iy", "iz", "id")


class Simulation:
    """One library context (pic_create ... pic_destroy) with numpy-facing calls."""

    FIELD_KEYS = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")

    def __init__(self, cfg: pic_config_t, stream=None, handle=None):
        """A new context (pic_create), or with ``handle`` a view of a context
        owned elsewhere (a batch run), which close() leaves alone."""
        L = load()
        self.cfg = cfg
        self.nx, self.ny = cfg.nx, cfg.ny
        self.dim = 3 if cfg.dim == 3 else 2
        self.nz = cfg.nz if self.dim == 3 else 1
        self.nspecies = cfg.nspecies
        self.owner = handle is None
        if handle is None:
            h = C.c_void_p()
            _check(L.pic_create(C.byref(cfg), _stream(stream), C.byref(h)))
        else:
            h = handle
        self.h = h
        self.stream = stream

    def close(self):
        if getattr(self, "h", None):
            if self.owner:
                load().pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, status):
        _check(status, self.h)

    @property
    def _s(self):
        return _stream(self.stream)

    def grid(self):
        """(dt, dx, dy) in 2D3V, (dt, dx, dy, dz) in 3D3V."""
        v = [C.c_double() for _ in range(4)]
        self._c(load().pic_get_grid(self.h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v[:4 if self.dim == 3 else 3])

    @property
    def _pkeys(self):
        base = ("ix", "iy", "ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w", "id")
        return base + (("iz", "oz") if self.dim == 3 else ())

    @property
    def _mesh_shape(self):
        return (self.nz, self.ny, self.nx) if self.dim == 3 else (self.ny, self.nx)

    @property
    def _bnd_shape(self):
        return (self.nz, self.ny) if self.dim == 3 else (self.ny,)

    # state ----------------------------------------------------------------
    def set_particles(self, s, d):
        n = len(d["ix"])
        arr = {k: np.ascontiguousarray(d[k], dtype=np.int32 if k in _INT_KEYS else np.float32)
               for k in self._pkeys}
        p = pic_particles_t(n=n, **{k: _ptr(v, _I32P if v.dtype == np.int32 else _F32P)
                                    for k, v in arr.items()})
        self._c(load().pic_set_particles(self.h, s, C.byref(p), self._s))

    def set_particles_f64(self, s, d):
        """set_particles from float64 arrays (exact in a precision-64 context)."""
        n = len(d["ix"])
        arr = {k: np.ascontiguousarray(d[k], dtype=np.int32 if k in _INT_KEYS else np.float64)
               for k in self._pkeys}
        p = pic_particles_f64_t(n=n, **{k: _ptr(v, _I32P if v.dtype == np.int32 else _F64P)
                                        for k, v in arr.items()})
        self._c(load().pic_set_particles_f64(self.h, s, C.byref(p), self._s))

    def set_particles_raw(self, s, n, ptrs):
        """Like set_particles, from raw host addresses (e.g. pinned buffers):
        ptrs maps every pic_particles_t array name to an integer address."""
        kw = {k: C.cast(C.c_void_p(int(v)), _I32P if k in _INT_KEYS else _F32P)
              for k, v in ptrs.items()}
        p = pic_particles_t(n=int(n), **kw)
        self._c(load().pic_set_particles(self.h, s, C.byref(p), self._s))

    def set_particles_f64_raw(self, s, n, ptrs):
        """set_particles_f64 from raw host addresses (float64 record arrays)."""
        kw = {k: C.cast(C.c_void_p(int(v)), _I32P if k in _INT_KEYS else _F64P)
              for k, v in ptrs.items()}
        p = pic_particles_f64_t(n=int(n), **kw)
        self._c(load().pic_set_particles_f64(self.h, s, C.byref(p), self._s))

    def count(self, s):
        n = C.c_int64()
        self._c(load().pic_get_count(self.h, s, C.byref(n)))
        return n.value

    def get_particles(self, s):
        n = self.count(s)
        out = {k: np.empty(n, np.int32 if k in _INT_KEYS else np.float32) for k in self._pkeys}
        p = pic_particles_t(n=n, **{k: _ptr(v, _I32P if v.dtype == np.int32 else _F32P)
                                    for k, v in out.items()})
        self._c(load().pic_get_particles(self.h, s, C.byref(p), self._s))
        # the library returns the slots it wrote (a binned layout is compacted first)
        return {k: v[:p.n] for k, v in out.items()}

    def get_particles_f64(self, s):
        n = self.count(s)
        out = {k: np.empty(n, np.int32 if k in _INT_KEYS else np.float64) for k in self._pkeys}
        p = pic_particles_f64_t(n=n, **{k: _ptr(v, _I32P if v.dtype == np.int32 else _F64P)
                                        for k, v in out.items()})
        self._c(load().pic_get_particles_f64(self.h, s, C.byref(p), self._s))
        return {k: v[:p.n] for k, v in out.items()}

    def get_fields_f64(self):
        out = {k: np.empty(self._mesh_shape, np.float64) for k in self.FIELD_KEYS}
        out["by_left"] = np.empty(self._bnd_shape, np.float64)
        out["bz_left"] = np.empty(self._bnd_shape, np.float64)
        pf = pic_fields_f64_t(**{k: _ptr(v, _F64P) for k, v in out.items()})
        self._c(load().pic_get_fields_f64(self.h, C.byref(pf), self._s))
        return out

    def set_fields(self, f):
        keep = {}
        kw = {}
        for k, v in f.items():
            a = np.ascontiguousarray(v, dtype=np.float32)
            want = self._bnd_shape if k in ("by_left", "bz_left") else self._mesh_shape
            if a.shape != want:
                raise ValueError(f"{k}: shape {a.shape}, expected {want}")
            keep[k] = a
            kw[k] = _ptr(a, _F32P)
        pf = pic_fields_t(**kw)
        self._c(load().pic_set_fields(self.h, C.byref(pf), self._s))

    def get_fields(self):
        out = {k: np.empty(self._mesh_shape, np.float32) for k in self.FIELD_KEYS}
        out["by_left"] = np.empty(self._bnd_shape, np.float32)
        out["bz_left"] = np.empty(self._bnd_shape, np.float32)
        pf = pic_fields_t(**{k: _ptr(v, _F32P) for k, v in out.items()})
        self._c(load().pic_get_fields(self.h, C.byref(pf), self._s))
        return out

    def set_step(self, n):
        self._c(load().pic_set_step(self.h, int(n)))

    def get_step(self):
        v = C.c_int64()
        self._c(load().pic_get_step(self.h, C.byref(v)))
        return v.value

    # method parts ---------------------------------------------------------
    def gather_push_spin(self):
        self._c(load().pic_gather_push_spin(self.h, self._s))

    def deposit(self):
        self._c(load().pic_deposit(self.h, self._s))

    def field_update(self):
        self._c(load().pic_field_update(self.h, self._s))

    def sort(self):
        self._c(load().pic_sort(self.h, self._s))

    def push_deposit(self):
        self._c(load().pic_push_deposit(self.h, self._s))

    def step(self, nsteps=1):
        self._c(load().pic_step(self.h, int(nsteps), self._s))

    def launch_count(self):
        v = C.c_int64()
        self._c(load().pic_launch_count(self.h, C.byref(v)))
        return v.value

    def set_graphs(self, max_steps):
        """pic_set_graphs: longest stretch pic_step replays from a CUDA graph (0: off)."""
        self._c(load().pic_set_graphs(self.h, int(max_steps)))

    def graph_stats(self):
        """pic_graph_stats: (captures, replays)."""
        a, b = C.c_int64(), C.c_int64()
        self._c(load().pic_graph_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def polarization(self, s, emin=-math.inf, emax=math.inf):
        m = pic_moments_t()
        self._c(load().pic_polarization(self.h, s, float(emin), float(emax), C.byref(m), self._s))
        return dict(P=np.array(m.P[:]), sum_w=m.sum_w, count=m.count, ekin_mean=m.ekin_mean,
                    ekin_var=m.ekin_var)

    def set_diagnostics(self, every, emin=None, emax=None):
        n = self.nspecies
        lo = (C.c_double * n)(*([-math.inf] * n if emin is None else emin))
        hi = (C.c_double * n)(*([math.inf] * n if emax is None else emax))
        self._c(load().pic_set_diagnostics(self.h, int(every), lo, hi))

    def get_diagnostics(self):
        out = (pic_moments_t * self.nspecies)()
        st = C.c_int64()
        self._c(load().pic_get_diagnostics(self.h, out, C.byref(st), self._s))
        return st.value, [dict(P=np.array(m.P[:]), sum_w=m.sum_w, count=m.count, ekin_mean=m.ekin_mean,
                               ekin_var=m.ekin_var) for m in out]

    def energy_histogram(self, s, emin, emax, nbins, log_bins=False):
        """[nbins][5]: count, sum w, sum w s (3) per kinetic-energy bin."""
        out = np.zeros(5 * nbins)
        self._c(load().pic_energy_histogram(self.h, s, float(emin), float(emax), int(nbins),
                                            1 if log_bins else 0, _ptr(out, C.POINTER(C.c_double)), self._s))
        return out.reshape(nbins, 5)

    def capture_background(self):
        self._c(load().pic_capture_background(self.h, self._s))

    def gauss_residual(self):
        out = (C.c_double * 2)()
        self._c(load().pic_gauss_residual(self.h, out, self._s))
        return out[0], out[1]

    def sync(self):
        self._c(load().pic_sync(self.h, self._s))

    # adjoint (2D3V) ----------------------------------------------------------
    @staticmethod
    def _loss(species=0, axis=1, e_cut_mev=50.0, e_width_mev=5.0):
        return pic_loss_t(species=species, axis=axis, e_cut_mev=e_cut_mev, e_width_mev=e_width_mev)

    def loss(self, **kw):
        """pic_loss of the current state (keywords: species, axis, e_cut_mev, e_width_mev)."""
        v = C.c_double()
        self._c(load().pic_loss(self.h, C.byref(self._loss(**kw)), C.byref(v), self._s))
        return v.value

    def adjoint(self, nsteps, checkpoint_every, **kw):
        """pic_adjoint: (L, dL/da0); per-particle gradients via adjoint_particle_grads."""
        v, g = C.c_double(), C.c_double()
        self._c(load().pic_adjoint(self.h, int(nsteps), int(checkpoint_every), C.byref(self._loss(**kw)),
                                   C.byref(v), C.byref(g), self._s))
        return v.value, g.value

    def adjoint_particle_grads(self, s):
        """dL/d(initial state) of the slots of species s: keys ox oy ux uy uz sx sy sz w
        (float64) and the slots' initial ix, iy and id."""
        n = self.count(s)
        keys = ("ix", "iy", "ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w", "id")
        out = {k: np.empty(max(n, 1), np.int32 if k in _INT_KEYS else np.float64) for k in keys}
        p = pic_particles_f64_t(n=len(out["ix"]), **{k: _ptr(v, _I32P if v.dtype == np.int32 else _F64P)
                                                     for k, v in out.items()})
        self._c(load().pic_adjoint_particle_grads(self.h, s, C.byref(p), self._s))
        return {k: v[:p.n] for k, v in out.items()}

    def _inject_arr(self, inject):
        keep = []
        arr = (pic_particles_t * self.nspecies)()
        for s, d in enumerate(inject):
            a = {k: np.ascontiguousarray(d[k], dtype=np.int32 if k in _INT_KEYS else np.float32)
                 for k in self._pkeys}
            keep.append(a)
            arr[s] = pic_particles_t(n=len(a["ix"]), **{k: _ptr(v, _I32P if v.dtype == np.int32 else _F32P)
                                                         for k, v in a.items()})
        return arr, keep

    def shift_window(self, ncells, inject=None):
        """pic_shift_window: inject is None or one particle dict per species."""
        if inject is None:
            self._c(load().pic_shift_window(self.h, int(ncells), None, self._s))
            return
        arr, keep = self._inject_arr(inject)
        self._c(load().pic_shift_window(self.h, int(ncells), arr, self._s))
        del keep

    def set_window(self, ncells, start_step=0, speed=1.0):
        """pic_set_window: pic_step moves the box by ncells cells whenever it
        lags a front leaving at start_step with `speed` (units of c) by
        ncells; ncells = 0 switches it off."""
        self._c(load().pic_set_window(self.h, int(ncells), int(start_step), float(speed)))

    def stage_injection(self, inject):
        """pic_stage_injection: one particle dict per species, the plasma of
        one future move."""
        arr, keep = self._inject_arr(inject)
        self._c(load().pic_stage_injection(self.h, arr, self._s))
        del keep

    def buffer_sizes(self):
        """pic_buffer_sizes: (ld, plane, real bytes, [capacity per species])."""
        ld, plane, rb = C.c_int64(), C.c_int64(), C.c_int()
        cap = (C.c_int64 * 4)()
        self._c(load().pic_buffer_sizes(self.h, C.byref(ld), C.byref(plane), C.byref(rb), cap))
        return ld.value, plane.value, rb.value, list(cap)[:self.nspecies]

    def bind_torch(self, mesh=True, particles=True):
        """pic_bind_buffers with torch tensors allocated here on the current
        CUDA device: from then on they are the context's state (no copies).
        Returns {"eb": [6][nz][ny][ld], "j": [3][nz][ny][ld],
        "sp": [[buffer 0 dict, buffer 1 dict] per species]} (cell words as
        int32 bit patterns)."""
        import torch
        ld, plane, rb, caps = self.buffer_sizes()
        dt = torch.float32 if rb == 4 else torch.float64
        dev = torch.device("cuda", torch.cuda.current_device())
        b = pic_buffers_t()
        out = {"eb": None, "j": None, "sp": []}
        if mesh:
            out["eb"] = torch.zeros((6, self.nz, self.ny, ld), dtype=dt, device=dev)
            out["j"] = torch.zeros((3, self.nz, self.ny, ld), dtype=dt, device=dev)
            b.eb, b.j = out["eb"].data_ptr(), out["j"].data_ptr()
        for s in range(self.nspecies):
            pair = []
            for q in range(2):
                if not particles:
                    pair.append(None)
                    continue
                t = {"cell": torch.empty(caps[s], dtype=torch.int32, device=dev),
                     "id": torch.empty(caps[s], dtype=torch.int32, device=dev)}
                for k in _BUF_REALS:
                    if k != "oz" or self.dim == 3:
                        t[k] = torch.empty(caps[s], dtype=dt, device=dev)
                slot = b.sp[s][q]
                for k, v in t.items():
                    setattr(slot, k, v.data_ptr())
                pair.append(t)
            out["sp"].append(pair)
        self._c(load().pic_bind_buffers(self.h, C.byref(b), self._s))
        self._bound = out
        return out

    def particle_views(self, s):
        """Species s's particles in bound memory (bind_torch), no copy: the
        current buffer's tensors cut to pic_get_count slots."""
        which = C.c_int()
        self._c(load().pic_current_buffer(self.h, int(s), C.byref(which)))
        n = self.count(s)
        return {k: v[:n] for k, v in self._bound["sp"][s][which.value].items()}

    def binned(self, s):
        """pic_get_layout: True when species s is in the binned 3D3V layout."""
        v = C.c_int()
        self._c(load().pic_get_layout(self.h, int(s), C.byref(v)))
        return bool(v.value)

    def staged_injections(self):
        v = C.c_int64()
        self._c(load().pic_staged_injections(self.h, C.byref(v)))
        return v.value

    def window(self):
        v = C.c_int64()
        self._c(load().pic_get_window(self.h, C.byref(v)))
        return v.value


class Batch:
    """A batch of independent 2D3V runs (pic_batch_*): one persistent fused
    launch and one batched field update per step for every run, sort-free
    stretches replayed as CUDA graphs."""

    def __init__(self, cfgs, nsteps, stream=None):
        L = load()
        n = len(cfgs)
        arr = (pic_config_t * n)(*cfgs)
        steps = (C.c_int64 * n)(*[int(v) for v in nsteps])
        h = C.c_void_p()
        st = L.pic_batch_create(arr, n, steps, _stream(stream), C.byref(h))
        if st != 0:
            msg = L.pic_batch_last_error(None)
            raise PicError(st, msg.decode() if msg else "")
        self.h = h
        self.n = n
        self.cfgs = list(cfgs)
        self.stream = stream

    def _c(self, status):
        if status != 0:
            msg = load().pic_batch_last_error(self.h)
            raise PicError(status, msg.decode() if msg else "")

    def run(self, r):
        """Simulation view of run r (owned by the batch)."""
        h = C.c_void_p()
        self._c(load().pic_batch_run(self.h, int(r), C.byref(h)))
        return Simulation(self.cfgs[r], stream=self.stream, handle=h)

    def step(self, nsteps):
        self._c(load().pic_batch_step(self.h, int(nsteps), _stream(self.stream)))

    def steps_done(self):
        out = (C.c_int64 * self.n)()
        self._c(load().pic_batch_steps_done(self.h, out))
        return list(out)

    def launch_count(self):
        v = C.c_int64()
        self._c(load().pic_batch_launch_count(self.h, C.byref(v)))
        return v.value

    def tune(self, probe_steps, tiles=((16, 8), (32, 8)), sorts=(16, 32, 64)):
        t = (C.c_int * (2 * len(tiles)))(*[v for tt in tiles for v in tt])
        q = (C.c_int * len(sorts))(*sorts)
        out = (C.c_int * 3)()
        self._c(load().pic_batch_tune(self.h, int(probe_steps), t, len(tiles), q, len(sorts), out,
                                      _stream(self.stream)))
        return tuple(out)

    def close(self):
        if getattr(self, "h", None):
            load().pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
