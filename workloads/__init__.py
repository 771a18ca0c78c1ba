"""Seeded synthetic workloads shared by the CUDA path and the oracle.

This module holds data only: the workload parameters (the paper's setup of
Sec. 2 scaled to the 2D3V and 3D3V cases built here) and seeded random draws of the
initial particle state and, for single-step tests, of random mesh fields.  It
contains none of the method's arithmetic; both the oracle and the CUDA
library derive their own time step, units and boundary handling from these
parameters.

Particle state of one species (all arrays of length n):
  ix, iy   int32   cell indices (node i sits at x = i dx)
  ox, oy   float32 offsets inside the cell, in [0, 1)
  iz, oz   the same along z (3D3V workloads only)
  ux,uy,uz float32 momentum u = p / (m c)
  sx,sy,sz float32 unit spin
  w        float32 density carried by the macro-particle [n_c]
  id       int32   particle identity (index at creation)
Every float is drawn as a float32 value, so the oracle's float64 copy of the
state is exactly the state the GPU holds.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["Species", "Workload", "CONFIG1", "CONFIG2", "CONFIG3", "CONFIG5", "batch_scan", "ramp_weights",
           "generate_particles",
           "injection_particles", "random_fields", "small_case", "small_case3", "scaled"]


@dataclass(frozen=True)
class Species:
    name: str
    q: float            # charge [e]
    m: float            # mass [m_e]
    a: float            # gyromagnetic anomaly
    n0: float           # density [n_c]
    ppc: int            # macro-particles per cell
    u_th: float         # thermal spread of each momentum component [m c]
    s0: tuple           # initial spin (unit vector)
    mobile: bool = True
    colocate_with: int = -1   # reuse the positions of this species (a neutral start)


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    dx_lambda: float          # cell size in laser wavelengths
    dy_lambda: float
    cfl: float                # dt = cfl / sqrt(1/dx^2 + 1/dy^2 [+ 1/dz^2])
    steps: int
    species: tuple
    a0: float = 0.0
    waist_lambda: float = 4.0
    fwhm_periods: float = 10.0   # FWHM of the intensity, in laser periods
    t_peak_periods: float = 15.0
    pol: str = "lp-y"            # "lp-y", "cp" or "none"
    bc_x: str = "open"           # "open" (laser enters at x_min) or "periodic"
    neutralizing_background: bool = False  # immobile ions = -rho_e at t = 0
    seed: int = 1
    lambda_um: float = 0.8
    dim: int = 2                 # 2: 2D3V mesh [ny][nx]; 3: 3D3V mesh [nz][ny][nx]
    nz: int = 1
    dz_lambda: float = 1.0


ELECTRON = dict(q=-1.0, m=1.0, a=0.00116)
PROTON = dict(q=1.0, m=1836.0, a=1.793)

# 2D3V uniform electron plasma with immobile ions, LP laser a0 = 4 (131,072 electrons).
CONFIG1 = Workload(
    name="2d3v-256x128-ppc4-lp-a0_4",
    nx=256, ny=128, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=0.95, steps=400,
    species=(Species("electron", n0=0.01, ppc=4, u_th=1e-3, s0=(0.0, 1.0, 0.0), **ELECTRON),),
    a0=4.0, waist_lambda=4.0, fwhm_periods=10.0, t_peak_periods=15.0, pol="lp-y",
    bc_x="open", neutralizing_background=True, seed=1)

# 2D3V high-density pre-polarised hydrogen: 8 ppc electrons + 8 ppc protons
# (67,043,328 particles: every cell but the two-cell vacuum margins at x_min and
# x_max; 67,108,864 with all cells filled), spins +x, CP laser a0 = 60.
CONFIG3 = Workload(
    name="2d3v-4096x1024-e8p8-cp-a0_60",
    nx=4096, ny=1024, dx_lambda=1 / 32, dy_lambda=1 / 32, cfl=0.95, steps=5000,
    species=(Species("electron", n0=0.2, ppc=8, u_th=1e-3, s0=(1.0, 0.0, 0.0), **ELECTRON),
             Species("proton", n0=0.2, ppc=8, u_th=1e-3 * math.sqrt(1 / 1836.0),
                     s0=(1.0, 0.0, 0.0), colocate_with=0, **PROTON)),
    a0=60.0, waist_lambda=8.0, fwhm_periods=10.0, t_peak_periods=15.0, pol="cp",
    bc_x="open", neutralizing_background=False, seed=3)


# 3D3V laser-wakefield precision study: 512x256x256 cells, dx = lambda/20,
# dy = dz = lambda/8, 2 ppc electrons at 0.003 n_c over immobile ions (66,584,576
# electrons: every cell but the two-cell vacuum margins along x), spins +y, LP
# Gaussian laser a0 = 3 (waist 8 lambda: the setup leaves it open).
CONFIG2 = Workload(
    name="3d3v-512x256x256-ppc2-lp-a0_3",
    nx=512, ny=256, dx_lambda=1 / 20, dy_lambda=1 / 8, cfl=0.95, steps=2000,
    species=(Species("electron", n0=0.003, ppc=2, u_th=1e-3, s0=(0.0, 1.0, 0.0), **ELECTRON),),
    a0=3.0, waist_lambda=8.0, fwhm_periods=10.0, t_peak_periods=15.0, pol="lp-y",
    bc_x="open", neutralizing_background=True, seed=2, dim=3, nz=256, dz_lambda=1 / 8)


def batch_scan(nruns: int = 256, seed: int = 4, size_scale: float = 1.0, step_scale: float = 1.0):
    """Parameter scan of independent 2D3V runs of uneven sizes: per run Nx in
    {128, 256, 512, 1024} (equal odds: uniform in log Nx), Ny = Nx/2,
    dx = dy = lambda/16, electron density n0 ~ U(0.001, 0.05) n_c over immobile
    ions, ppc ~ U{2..8}, LP laser a0 ~ U(2, 20) (waist a quarter of the box
    height, FWHM 10 periods, peak at 15 periods), spins +y, steps ~
    U{300..1500}; seed-drawn.  size_scale / step_scale shrink the meshes and
    run lengths for tests.  Returns [(Workload, steps)]."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(nruns):
        nx = int(rng.choice([128, 256, 512, 1024]))
        nx = max(16, int(round(nx * size_scale / 8)) * 8)
        ny = max(8, nx // 2)
        n0 = float(rng.uniform(0.001, 0.05))
        a0 = float(rng.uniform(2.0, 20.0))
        ppc = int(rng.integers(2, 9))
        steps = max(1, int(round(int(rng.integers(300, 1501)) * step_scale)))
        sp = Species("electron", n0=n0, ppc=ppc, u_th=1e-3, s0=(0.0, 1.0, 0.0), **ELECTRON)
        wl = Workload(name=f"scan{r}-{nx}x{ny}-ppc{ppc}", nx=nx, ny=ny, dx_lambda=1 / 16, dy_lambda=1 / 16,
                      cfl=0.95, steps=steps, species=(sp,), a0=a0, waist_lambda=ny / 16 / 4,
                      fwhm_periods=10.0, t_peak_periods=15.0, pol="lp-y", bc_x="open",
                      neutralizing_background=True, seed=seed * 1000 + r)
        out.append((wl, steps))
    return out


# 2D3V gradient study: 1024x512 cells (dx = dy = lambda/16), 8 ppc electrons
# whose density follows a 64-knot piecewise-linear ramp (ramp_weights), LP
# laser a0 = 5, spins +y; 1000 steps, checkpoint every 50 (the run length and
# interval belong to the adjoint call).
CONFIG5 = Workload(
    name="2d3v-1024x512-ppc8-ramp64-lp-a0_5",
    nx=1024, ny=512, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=0.95, steps=1000,
    species=(Species("electron", n0=0.01, ppc=8, u_th=1e-3, s0=(0.0, 1.0, 0.0), **ELECTRON),),
    a0=5.0, waist_lambda=8.0, fwhm_periods=10.0, t_peak_periods=15.0, pol="lp-y",
    bc_x="open", neutralizing_background=True, seed=5)


def ramp_knots(nknots: int = 64, n0: float = 0.01, ramp_fraction: float = 0.25):
    """Knot values of a smooth up-ramp to n0 over the first ramp_fraction of
    the plasma, flat after (a smoothstep sampled at the knots)."""
    t = np.clip(np.linspace(0.0, 1.0, nknots) / ramp_fraction, 0.0, 1.0)
    return n0 * t * t * (3.0 - 2.0 * t)


def ramp_weights(wl: Workload, particles, knots):
    """Weights n(x)/ppc of the first species for a piecewise-linear density
    with the given knot values, knots spread evenly over the plasma [2, nx-2)."""
    d = particles[0]
    x = d["ix"].astype(np.float64) + d["ox"].astype(np.float64)
    xk = np.linspace(2.0, wl.nx - 2.0, len(knots))
    i = np.clip(np.searchsorted(xk, x) - 1, 0, len(xk) - 2)
    t = (x - xk[i]) / (xk[i + 1] - xk[i])
    return (np.asarray(knots)[i] * (1.0 - t) + np.asarray(knots)[i + 1] * t) / wl.species[0].ppc


def scaled(wl: Workload, **kw) -> Workload:
    """A copy of a workload with some fields replaced."""
    return dataclasses.replace(wl, **kw)


def small_case(nx=40, ny=24, ppc=2, bc_x="open", seed=11, pol="lp-y", a0=4.0,
               two_species=False, u_th=0.05) -> Workload:
    """Few-tile test workload; nx, ny need not be tile multiples (ragged edges)."""
    sp = [Species("electron", n0=0.05, ppc=ppc, u_th=u_th, s0=(0.0, 1.0, 0.0), **ELECTRON)]
    if two_species:
        sp.append(Species("proton", n0=0.05, ppc=ppc, u_th=u_th / 20, s0=(1.0, 0.0, 0.0),
                          colocate_with=0, **PROTON))
    return Workload(name=f"small-{nx}x{ny}", nx=nx, ny=ny, dx_lambda=1 / 16, dy_lambda=1 / 16,
                    cfl=0.95, steps=10, species=tuple(sp), a0=a0, waist_lambda=1.0,
                    fwhm_periods=2.0, t_peak_periods=1.0, pol=pol, bc_x=bc_x,
                    neutralizing_background=not two_species, seed=seed)


def small_case3(nx=24, ny=16, nz=12, ppc=2, bc_x="open", seed=12, pol="lp-y", a0=4.0,
                two_species=False, u_th=0.05, dx_lambda=1 / 16, dy_lambda=1 / 12,
                dz_lambda=1 / 10) -> Workload:
    """Few-tile 3D3V test workload; sizes need not be tile multiples."""
    base = small_case(nx=nx, ny=ny, ppc=ppc, bc_x=bc_x, seed=seed, pol=pol, a0=a0,
                      two_species=two_species, u_th=u_th)
    return dataclasses.replace(base, name=f"small3-{nx}x{ny}x{nz}", dim=3, nz=nz,
                               dx_lambda=dx_lambda, dy_lambda=dy_lambda, dz_lambda=dz_lambda)


def _region_x(wl: Workload):
    """Cells that hold plasma along x: all of them when x is periodic, else a
    two-cell vacuum margin at each end (particles live in [2, nx-2))."""
    if wl.bc_x == "periodic":
        return 0, wl.nx
    return 2, wl.nx - 2


def generate_particles(wl: Workload, seed: int | None = None):
    """Initial particles of every species: uniform random positions inside
    each cell, Gaussian thermal momenta, equal spins and weights.

    Order is ppc-major (all cells for the first macro-particle of each cell,
    then the second, ...), so neighbouring entries sit in neighbouring cells.
    Returns a list with one dict of arrays per species.
    """
    rng = np.random.default_rng(wl.seed if seed is None else seed)
    x0, x1 = _region_x(wl)
    ncx = x1 - x0
    three = wl.dim == 3
    nzc = wl.nz if three else 1
    gz, gy, gx = np.meshgrid(np.arange(nzc, dtype=np.int32), np.arange(wl.ny, dtype=np.int32),
                             np.arange(x0, x1, dtype=np.int32), indexing="ij")
    out = []
    for s, sp in enumerate(wl.species):
        n = sp.ppc * ncx * wl.ny * nzc
        extra = {}
        if sp.colocate_with >= 0:
            ref = out[sp.colocate_with]
            if len(ref["ix"]) != n:
                raise ValueError("co-located species need the same particle count")
            ix, iy, ox, oy = ref["ix"], ref["iy"], ref["ox"], ref["oy"]
            if three:
                extra = dict(iz=ref["iz"], oz=ref["oz"])
        else:
            ix = np.tile(gx.ravel(), sp.ppc)
            iy = np.tile(gy.ravel(), sp.ppc)
            ox = rng.random(n, dtype=np.float32)
            oy = rng.random(n, dtype=np.float32)
            if three:
                extra = dict(iz=np.tile(gz.ravel(), sp.ppc), oz=rng.random(n, dtype=np.float32))
        uth = np.float32(sp.u_th)
        ux = rng.standard_normal(n, dtype=np.float32) * uth
        uy = rng.standard_normal(n, dtype=np.float32) * uth
        uz = rng.standard_normal(n, dtype=np.float32) * uth
        s0 = np.asarray(sp.s0, dtype=np.float32)
        out.append(dict(
            ix=ix, iy=iy, ox=ox, oy=oy, ux=ux, uy=uy, uz=uz,
            sx=np.full(n, s0[0], np.float32), sy=np.full(n, s0[1], np.float32),
            sz=np.full(n, s0[2], np.float32),
            w=np.full(n, np.float32(sp.n0 / sp.ppc), np.float32),
            id=np.arange(n, dtype=np.int32), **extra))
    return out


def injection_particles(wl: Workload, ncells: int, seed: int, id_base: int = 0):
    """Plasma for the ncells columns that a moving-window shift by ncells
    uncovers at the right end: cells [nx-2-ncells, nx-2) along x (the last two
    columns stay vacuum), drawn with the workload's recipe (uniform in the cell,
    Gaussian thermal momenta, the species' spin and weight).  Ids start at
    id_base.  One dict per species, as generate_particles returns."""
    sub = dataclasses.replace(wl, nx=ncells, bc_x="periodic")
    parts = generate_particles(sub, seed=seed)
    x0 = wl.nx - 2 - ncells
    for d in parts:
        d["ix"] = (d["ix"] + x0).astype(np.int32)
        d["id"] = (d["id"] + id_base).astype(np.int32)
    return parts


def random_fields(wl: Workload, seed: int, e_amp: float = 0.5, b_amp: float = 0.5):
    """Random mesh fields (float32, [ny][nx] or [nz][ny][nx]) for single-step tests."""
    rng = np.random.default_rng(seed)
    shape = (wl.nz, wl.ny, wl.nx) if wl.dim == 3 else (wl.ny, wl.nx)
    f = {}
    for k, amp in (("ex", e_amp), ("ey", e_amp), ("ez", e_amp),
                   ("bx", b_amp), ("by", b_amp), ("bz", b_amp)):
        f[k] = (rng.standard_normal(shape, dtype=np.float32) * np.float32(amp))
    return f
