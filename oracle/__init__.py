"""FP64 CPU oracle of the 2D3V and 3D3V PIC + Thomas-BMT step (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  It does not import, link or share code
with the CUDA library.

The arithmetic is plain C (``pic_oracle.c`` for 2D3V, ``pic_oracle3.c`` for
3D3V); this module builds it with gcc, derives the oracle's own units from a
workload (length c/omega0, time 1/omega0, dt = cfl / sqrt(sum 1/dx_i^2)) and
holds the state in float64 numpy arrays.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# the same sources built with OpenMP: the multi-core CPU baseline (its parallel
# loops have independent iterations, so it gives the plain build's bits)
_LIB_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
# a prebuilt oracle library to load instead (the mutation tests point it at
# deliberately broken copies)
_LIB_OVERRIDE = os.environ.get("PIC_ORACLE_LIB")
_lib = None
_lib_omp = None
_parallel = False

MEC2_MEV = 0.51099895
BC = {"open": 0, "periodic": 1}
POL = {"none": 0, "lp-y": 1, "cp": 2}


SOURCES = ("pic_oracle.c", "pic_oracle3.c")


def build(force: bool = False) -> str:
    """Compile the oracle sources into liboracle.so next to them (gcc, FP64, no
    FMA contraction), and the same sources with OpenMP into liboracle_omp.so."""
    srcs = [os.path.join(_HERE, f) for f in SOURCES]
    newest = max(os.path.getmtime(f) for f in srcs + [os.path.join(_HERE, "pic_oracle.h")])
    for path, extra in ((_LIB_PATH, []), (_LIB_OMP_PATH, ["-fopenmp"])):
        if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
            continue
        tmp = path + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                               *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return _LIB_PATH


@contextlib.contextmanager
def parallel():
    """Oracle calls inside the block run on the OpenMP build (every host core
    unless OMP_NUM_THREADS says otherwise); the results are the plain build's."""
    global _parallel
    old = _parallel
    _parallel = True
    try:
        yield threads()
    finally:
        _parallel = old


def threads() -> int:
    """Threads the oracle calls use now (1 outside `parallel()`)."""
    return int(lib().or_threads())


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("bc_x", C.c_int), ("pol", C.c_int), ("a0", C.c_double),
                ("w0", C.c_double), ("tau", C.c_double), ("t_peak", C.c_double)]


class Spec(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("a", C.c_double)]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


class Fields(C.Structure):
    _fields_ = [(k, _DP) for k in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz", "byL", "bzL")]


class Parts(C.Structure):
    _fields_ = [("n", C.c_long)] + [(k, _DP) for k in
                                    ("x", "y", "ux", "uy", "uz", "sx", "sy", "sz", "w")] + [("alive", _IP)]


class Grid3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double), ("bc_x", C.c_int),
                ("pol", C.c_int), ("a0", C.c_double), ("w0", C.c_double), ("tau", C.c_double),
                ("t_peak", C.c_double)]


class Fields3(C.Structure):
    _fields_ = [(k, _DP) for k in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz", "byL", "bzL")]


class Parts3(C.Structure):
    _fields_ = [("n", C.c_long)] + [(k, _DP) for k in
                                    ("x", "y", "z", "ux", "uy", "uz", "sx", "sy", "sz", "w")] + [("alive", _IP)]


def lib():
    global _lib, _lib_omp
    if _parallel and not _LIB_OVERRIDE:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(C.CDLL(_LIB_OMP_PATH))
        return _lib_omp
    if _lib is None:
        if _LIB_OVERRIDE:
            L = C.CDLL(_LIB_OVERRIDE)
        else:
            build()
            L = C.CDLL(_LIB_PATH)
        _lib = _declare(L)
    return _lib


def _declare(L):
    if True:
        G, S, F, P = C.POINTER(Grid), C.POINTER(Spec), C.POINTER(Fields), C.POINTER(Parts)
        G3, F3, P3 = C.POINTER(Grid3), C.POINTER(Fields3), C.POINTER(Parts3)
        d = C.c_double
        sig = {
            "or3_gather": (None, [G3, F3, d, d, d, _DP, _DP]),
            "or3_deposit_one": (None, [G3, F3, d, d, d, d, d, d, d]),
            "or3_push": (None, [G3, S, P3, F3, _DP, _DP, _DP]),
            "or3_deposit": (None, [G3, S, P3, _DP, _DP, _DP, F3]),
            "or3_laser": (None, [G3, d, d, d, C.c_int, _DP]),
            "or3_field_update": (None, [G3, F3, C.c_long]),
            "or3_step": (None, [G3, S, P3, _IP, C.c_int, F3, C.c_long]),
            "or3_rho": (None, [G3, S, P3, _DP]),
            "or3_div_e": (None, [G3, F3, _DP]),
            "or3_div_b": (None, [G3, F3, _DP]),
            "or_gather": (None, [G, F, C.c_double, C.c_double, _DP, _DP]),
            "or_boris": (None, [C.c_double, C.c_double, _DP, _DP, _DP]),
            "or_omega": (None, [C.c_double, C.c_double, _DP, _DP, _DP, _DP]),
            "or_spin_rotate": (None, [_DP, C.c_double, _DP]),
            "or_deposit_one": (None, [G, F, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double]),
            "or_push": (None, [G, S, P, F, _DP, _DP, _DP]),
            "or_deposit": (None, [G, S, P, _DP, _DP, _DP, F]),
            "or_field_update": (None, [G, F, C.c_long]),
            "or_laser": (None, [G, C.c_double, C.c_double, C.c_int, _DP]),
            "or_step": (None, [G, S, P, _IP, C.c_int, F, C.c_long]),
            "or_rho": (None, [G, S, P, _DP]),
            "or_div_e": (None, [G, F, _DP]),
            "or_div_b": (None, [G, F, _DP]),
            "or_moments": (None, [S, P, C.c_double, C.c_double, _DP]),
            "or_histogram": (None, [S, P, C.c_double, C.c_double, C.c_int, C.c_int, _DP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if hasattr(L, "or_threads"):
            L.or_threads.restype = C.c_int
            L.or_threads.argtypes = []
        else:                     # a mutation copy built without the helper
            L.or_threads = lambda: 1
    return L


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _v3(x):
    return (C.c_double * 3)(*[float(v) for v in x])


# ---------------------------------------------------------------------------
# single-particle parts, for closed-form tests
# ---------------------------------------------------------------------------
def boris(qm, dt, E, B, u):
    uu = _v3(u)
    lib().or_boris(qm, dt, _v3(E), _v3(B), uu)
    return np.array(uu[:])


def omega(qm, a, ubar, E, B):
    out = _v3((0, 0, 0))
    lib().or_omega(qm, a, _v3(ubar), _v3(E), _v3(B), out)
    return np.array(out[:])


def spin_rotate(Om, dt, s):
    ss = _v3(s)
    lib().or_spin_rotate(_v3(Om), dt, ss)
    return np.array(ss[:])


def derive_grid(wl):
    """The oracle's own units: lengths in c/omega0 (lambda = 2 pi), time in 1/omega0."""
    if wl.dim == 3:
        return derive_grid3(wl)
    two_pi = 2.0 * math.pi
    dx, dy = wl.dx_lambda * two_pi, wl.dy_lambda * two_pi
    dt = wl.cfl / math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2)
    tau = wl.fwhm_periods * two_pi / math.sqrt(2.0 * math.log(2.0))
    return Grid(nx=wl.nx, ny=wl.ny, dx=dx, dy=dy, dt=dt, bc_x=BC[wl.bc_x],
                pol=POL[wl.pol] if wl.bc_x == "open" else 0, a0=wl.a0,
                w0=wl.waist_lambda * two_pi, tau=tau, t_peak=wl.t_peak_periods * two_pi)


def derive_grid3(wl) -> Grid3:
    """derive_grid for a 3D3V workload: dt = cfl / sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)."""
    two_pi = 2.0 * math.pi
    dx, dy, dz = wl.dx_lambda * two_pi, wl.dy_lambda * two_pi, wl.dz_lambda * two_pi
    dt = wl.cfl / math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2 + 1.0 / dz ** 2)
    tau = wl.fwhm_periods * two_pi / math.sqrt(2.0 * math.log(2.0))
    return Grid3(nx=wl.nx, ny=wl.ny, nz=wl.nz, dx=dx, dy=dy, dz=dz, dt=dt, bc_x=BC[wl.bc_x],
                 pol=POL[wl.pol] if wl.bc_x == "open" else 0, a0=wl.a0,
                 w0=wl.waist_lambda * two_pi, tau=tau, t_peak=wl.t_peak_periods * two_pi)


class OracleSim:
    """State of one oracle simulation: float64 mesh and particle arrays.

    ``particles`` is the per-species list of dicts from
    ``workloads.generate_particles``; positions become global cell coordinates
    x = ix + ox, y = iy + oy.
    """

    FIELD_KEYS = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")

    def __new__(cls, wl, *args, **kw):
        if cls is OracleSim and wl.dim == 3:
            return super().__new__(OracleSim3)
        return super().__new__(cls)

    def __init__(self, wl, particles, fields=None, step=0):
        self.wl = wl
        self.grid = derive_grid(wl)
        ny, nx = wl.ny, wl.nx
        self.f = {k: np.zeros((ny, nx)) for k in self.FIELD_KEYS}
        self.f["byL"] = np.zeros(ny)
        self.f["bzL"] = np.zeros(ny)
        if fields is not None:
            for k, v in fields.items():
                self.f[k][...] = np.asarray(v, dtype=np.float64)
        self.spec = [Spec(q=s.q, m=s.m, a=s.a) for s in wl.species]
        self.mobile = np.array([1 if s.mobile else 0 for s in wl.species], dtype=np.int32)
        self.p = []
        for d in particles:
            self.p.append(dict(
                x=d["ix"].astype(np.float64) + d["ox"].astype(np.float64),
                y=d["iy"].astype(np.float64) + d["oy"].astype(np.float64),
                ux=d["ux"].astype(np.float64), uy=d["uy"].astype(np.float64),
                uz=d["uz"].astype(np.float64), sx=d["sx"].astype(np.float64),
                sy=d["sy"].astype(np.float64), sz=d["sz"].astype(np.float64),
                w=d["w"].astype(np.float64), alive=np.ones(len(d["ix"]), np.int32),
                id=d["id"].copy()))
        self.step_index = step
        self.rho_bg = np.zeros((ny, nx))
        if wl.neutralizing_background:
            self.rho_bg = -self.rho()

    # ctypes views --------------------------------------------------------
    def _fields(self):
        return Fields(**{k: _dp(self.f[k]) for k in self.f})

    def _parts(self, s):
        d = self.p[s]
        kw = {k: _dp(d[k]) for k in ("x", "y", "ux", "uy", "uz", "sx", "sy", "sz", "w")}
        return Parts(n=len(d["x"]), alive=d["alive"].ctypes.data_as(_IP), **kw)

    # method parts ----------------------------------------------------------
    def push(self, s):
        """a1-a4 for species s; returns (x_old, y_old, vz) for the deposit."""
        n = len(self.p[s]["x"])
        xo, yo, vz = np.zeros(n), np.zeros(n), np.zeros(n)
        pp = self._parts(s)
        lib().or_push(C.byref(self.grid), C.byref(self.spec[s]), C.byref(pp),
                      C.byref(self._fields()), _dp(xo), _dp(yo), _dp(vz))
        return xo, yo, vz

    def deposit(self, s, xo, yo, vz):
        """a5 for species s (adds into J)."""
        pp = self._parts(s)
        lib().or_deposit(C.byref(self.grid), C.byref(self.spec[s]), C.byref(pp),
                         _dp(xo), _dp(yo), _dp(vz), C.byref(self._fields()))

    def zero_current(self):
        for k in ("jx", "jy", "jz"):
            self.f[k][...] = 0.0

    def field_update(self):
        """a6 at the current step index, which then advances by one."""
        lib().or_field_update(C.byref(self.grid), C.byref(self._fields()), self.step_index)
        self.step_index += 1

    def step(self, nsteps=1):
        """Whole steps: zero J, push and deposit every mobile species, a6."""
        nsp = len(self.p)
        for _ in range(nsteps):
            parts = (Parts * nsp)(*[self._parts(s) for s in range(nsp)])
            specs = (Spec * nsp)(*self.spec)
            lib().or_step(C.byref(self.grid), specs, parts,
                          self.mobile.ctypes.data_as(_IP), nsp, C.byref(self._fields()),
                          self.step_index)
            self.step_index += 1

    # diagnostics -------------------------------------------------------------
    def rho(self):
        r = np.zeros((self.wl.ny, self.wl.nx))
        for s in range(len(self.p)):
            pp = self._parts(s)
            lib().or_rho(C.byref(self.grid), C.byref(self.spec[s]), C.byref(pp), _dp(r))
        return r

    def div_e(self):
        d = np.zeros((self.wl.ny, self.wl.nx))
        lib().or_div_e(C.byref(self.grid), C.byref(self._fields()), _dp(d))
        return d

    def div_b(self):
        d = np.zeros((self.wl.ny, self.wl.nx))
        lib().or_div_b(C.byref(self.grid), C.byref(self._fields()), _dp(d))
        return d

    def gauss_residual(self):
        """div E - rho - rho_background on nodes; interior nodes only with open x
        (nodes 0..2 and nx-3..nx-1 see the removal of particles)."""
        r = self.div_e() - self.rho() - self.rho_bg
        if self.wl.bc_x == "open":
            r = r[:, 3:self.wl.nx - 3]
        return r

    def moments(self, s, emin=-np.inf, emax=np.inf):
        out = (C.c_double * 7)()
        pp = self._parts(s)
        lib().or_moments(C.byref(self.spec[s]), C.byref(pp), float(emin), float(emax), out)
        return np.array(out[:])

    def histogram(self, s, emin, emax, nbins, log_bins=False):
        """[nbins][5]: count, sum w, sum w s (3) per kinetic-energy bin."""
        out = np.zeros(5 * nbins)
        pp = self._parts(s)
        lib().or_histogram(C.byref(self.spec[s]), C.byref(pp), float(emin), float(emax), int(nbins),
                           1 if log_bins else 0, _dp(out))
        return out.reshape(nbins, 5)

    def laser(self, t, y, comp):
        v = C.c_double()
        lib().or_laser(C.byref(self.grid), t, y, comp, C.byref(v))
        return v.value

    def loss(self, s, axis=1, e_cut_mev=50.0, e_width_mev=5.0):
        """L = sum a_i s_i / sum a_i over the live particles of species s, with
        a_i = w_i e_i sig((e_i - e_cut) / e_width), e_i = (gamma - 1) m c^2 [MeV]
        and s_i the spin component `axis`: the energy-weighted polarization
        (Eq. 4) of the energetic part of the beam."""
        d = self.p[s]
        live = d["alive"] > 0
        u2 = d["ux"][live] ** 2 + d["uy"][live] ** 2 + d["uz"][live] ** 2
        e = (np.sqrt(1.0 + u2) - 1.0) * self.spec[s].m * MEC2_MEV
        a = d["w"][live] * e / (1.0 + np.exp(-(e - e_cut_mev) / e_width_mev))
        spin = d[("sx", "sy", "sz")[axis]][live]
        return float((a * spin).sum() / a.sum()) if a.sum() > 0 else 0.0

    # moving window -----------------------------------------------------------
    POS = ("x", "y")

    def shift_window(self, ncells, inject=None):
        """Co-moving window (Sec. 2: the simulation box follows the laser): the
        box moves ncells cells in +x between two steps.  In box coordinates
        every mesh array and the neutralizing background slide ncells columns
        toward x_min (columns that leave are dropped, the uncovered columns at
        x_max start at zero), the left boundary values By(-1/2), Bz(-1/2) are
        those of the column now at x = -1/2, particles move by -ncells cells
        and the ones whose cell falls below the plasma region (x < 2) are
        removed.  ``inject`` (one dict per species, workloads layout) is the
        plasma of the uncovered columns; with a neutralizing background its
        immobile ions (minus its charge density) join the background."""
        n = int(ncells)
        assert 1 <= n <= self.wl.nx - 8 and self.wl.bc_x == "open"
        self.f["byL"][...] = self.f["by"][..., n - 1]
        self.f["bzL"][...] = self.f["bz"][..., n - 1]
        for k in self.FIELD_KEYS:
            a = self.f[k]
            a[..., :-n] = a[..., n:].copy()
            a[..., -n:] = 0.0
        self.rho_bg[..., :-n] = self.rho_bg[..., n:].copy()
        self.rho_bg[..., -n:] = 0.0
        for d in self.p:
            d["x"] -= n
            d["alive"][d["x"] < 2.0] = 0
        if inject is not None:
            new = [self._particles_from(d) for d in inject]
            if self.wl.neutralizing_background:
                keep = self.p
                self.p = new
                self.rho_bg -= self.rho()
                self.p = keep
            for s, d in enumerate(new):
                for k in d:
                    self.p[s][k] = np.concatenate([self.p[s][k], d[k]])

    def _particles_from(self, d):
        out = dict(ux=d["ux"].astype(np.float64), uy=d["uy"].astype(np.float64),
                   uz=d["uz"].astype(np.float64), sx=d["sx"].astype(np.float64),
                   sy=d["sy"].astype(np.float64), sz=d["sz"].astype(np.float64),
                   w=d["w"].astype(np.float64), alive=np.ones(len(d["ix"]), np.int32),
                   id=d["id"].copy())
        for a in self.POS:
            out[a] = d["i" + a].astype(np.float64) + d["o" + a].astype(np.float64)
        return out


class OracleSim3(OracleSim):
    """OracleSim of a 3D3V workload: mesh arrays [nz][ny][nx], left boundary
    arrays [nz][ny], particle positions x = ix + ox, y = iy + oy, z = iz + oz.
    ``OracleSim(wl, ...)`` returns one of these when ``wl.dim == 3``."""

    POS = ("x", "y", "z")

    def __init__(self, wl, particles, fields=None, step=0):
        self.wl = wl
        self.grid = derive_grid3(wl)
        shape = (wl.nz, wl.ny, wl.nx)
        self.f = {k: np.zeros(shape) for k in self.FIELD_KEYS}
        self.f["byL"] = np.zeros((wl.nz, wl.ny))
        self.f["bzL"] = np.zeros((wl.nz, wl.ny))
        if fields is not None:
            for k, v in fields.items():
                self.f[k][...] = np.asarray(v, dtype=np.float64)
        self.spec = [Spec(q=s.q, m=s.m, a=s.a) for s in wl.species]
        self.mobile = np.array([1 if s.mobile else 0 for s in wl.species], dtype=np.int32)
        self.p = []
        for d in particles:
            self.p.append(dict(
                x=d["ix"].astype(np.float64) + d["ox"].astype(np.float64),
                y=d["iy"].astype(np.float64) + d["oy"].astype(np.float64),
                z=d["iz"].astype(np.float64) + d["oz"].astype(np.float64),
                ux=d["ux"].astype(np.float64), uy=d["uy"].astype(np.float64),
                uz=d["uz"].astype(np.float64), sx=d["sx"].astype(np.float64),
                sy=d["sy"].astype(np.float64), sz=d["sz"].astype(np.float64),
                w=d["w"].astype(np.float64), alive=np.ones(len(d["ix"]), np.int32),
                id=d["id"].copy()))
        self.step_index = step
        self.rho_bg = np.zeros(shape)
        if wl.neutralizing_background:
            self.rho_bg = -self.rho()

    def _fields(self):
        return Fields3(**{k: _dp(self.f[k]) for k in self.f})

    def _parts(self, s):
        d = self.p[s]
        kw = {k: _dp(d[k]) for k in ("x", "y", "z", "ux", "uy", "uz", "sx", "sy", "sz", "w")}
        return Parts3(n=len(d["x"]), alive=d["alive"].ctypes.data_as(_IP), **kw)

    def push(self, s):
        """a1-a4 for species s; returns the old positions (x, y, z) for the deposit."""
        n = len(self.p[s]["x"])
        xo, yo, zo = np.zeros(n), np.zeros(n), np.zeros(n)
        pp = self._parts(s)
        lib().or3_push(C.byref(self.grid), C.byref(self.spec[s]), C.byref(pp),
                       C.byref(self._fields()), _dp(xo), _dp(yo), _dp(zo))
        return xo, yo, zo

    def deposit(self, s, xo, yo, zo):
        pp = self._parts(s)
        lib().or3_deposit(C.byref(self.grid), C.byref(self.spec[s]), C.byref(pp),
                          _dp(xo), _dp(yo), _dp(zo), C.byref(self._fields()))

    def field_update(self):
        lib().or3_field_update(C.byref(self.grid), C.byref(self._fields()), self.step_index)
        self.step_index += 1

    def step(self, nsteps=1):
        nsp = len(self.p)
        for _ in range(nsteps):
            parts = (Parts3 * nsp)(*[self._parts(s) for s in range(nsp)])
            specs = (Spec * nsp)(*self.spec)
            lib().or3_step(C.byref(self.grid), specs, parts,
                           self.mobile.ctypes.data_as(_IP), nsp, C.byref(self._fields()),
                           self.step_index)
            self.step_index += 1

    def _mesh(self):
        return np.zeros((self.wl.nz, self.wl.ny, self.wl.nx))

    def rho(self):
        r = self._mesh()
        for s in range(len(self.p)):
            pp = self._parts(s)
            lib().or3_rho(C.byref(self.grid), C.byref(self.spec[s]), C.byref(pp), _dp(r))
        return r

    def div_e(self):
        d = self._mesh()
        lib().or3_div_e(C.byref(self.grid), C.byref(self._fields()), _dp(d))
        return d

    def div_b(self):
        d = self._mesh()
        lib().or3_div_b(C.byref(self.grid), C.byref(self._fields()), _dp(d))
        return d

    def gauss_residual(self):
        r = self.div_e() - self.rho() - self.rho_bg
        if self.wl.bc_x == "open":
            r = r[:, :, 3:self.wl.nx - 3]
        return r

    def _moment_parts(self, s):
        # the moments and spectra read only u, s, w and alive: the 2D view serves
        d = self.p[s]
        kw = {k: _dp(d[k]) for k in ("x", "y", "ux", "uy", "uz", "sx", "sy", "sz", "w")}
        return Parts(n=len(d["x"]), alive=d["alive"].ctypes.data_as(_IP), **kw)

    def moments(self, s, emin=-np.inf, emax=np.inf):
        out = (C.c_double * 7)()
        pp = self._moment_parts(s)
        lib().or_moments(C.byref(self.spec[s]), C.byref(pp), float(emin), float(emax), out)
        return np.array(out[:])

    def histogram(self, s, emin, emax, nbins, log_bins=False):
        out = np.zeros(5 * nbins)
        pp = self._moment_parts(s)
        lib().or_histogram(C.byref(self.spec[s]), C.byref(pp), float(emin), float(emax), int(nbins),
                           1 if log_bins else 0, _dp(out))
        return out.reshape(nbins, 5)

    def laser(self, t, y, z, comp):
        v = C.c_double()
        lib().or3_laser(C.byref(self.grid), t, y, z, comp, C.byref(v))
        return v.value
