"""Pins of the 3D3V FP64 oracle to facts fixed outside the oracle itself.

The 3D step is pinned three ways: with one periodic z cell it must reduce to
the (separately pinned) 2D3V oracle; a mirror that swaps y and z must map a
run onto the run of the mirrored state, which ties every z term to its
already pinned y twin; and closed forms that involve all three axes at once
(the Yee dispersion relation, discrete charge continuity by brute force,
exact interpolation of linear fields, the injected wave).
"""
import ctypes as C
import dataclasses
import math

import numpy as np
import pytest

import workloads as W

KEYS = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")
PKEYS = ("ux", "uy", "uz", "sx", "sy", "sz")


def _vacuum3(nx, ny, nz, bc="periodic", dx=1 / 16, dy=1 / 10, dz=1 / 12, cfl=0.9, **kw):
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.0, ppc=0, u_th=0.0, s0=(1, 0, 0))
    return W.Workload(name="vac3", nx=nx, ny=ny, dx_lambda=dx, dy_lambda=dy, cfl=cfl, steps=1,
                      species=(sp,), bc_x=bc, dim=3, nz=nz, dz_lambda=dz, **kw)


def _empty3():
    return [dict(ix=np.zeros(0, np.int32), iy=np.zeros(0, np.int32), iz=np.zeros(0, np.int32),
                 **{k: np.zeros(0, np.float32) for k in
                    ("ox", "oy", "oz", "ux", "uy", "uz", "sx", "sy", "sz", "w")},
                 id=np.zeros(0, np.int32))]


def _energy(sim):
    return sum((sim.f[k] ** 2).sum() for k in ("ex", "ey", "ez", "bx", "by", "bz"))


# ---------------------------------------------------------------------------
# reduction to the 2D3V oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", ["open", "periodic"])
def test_one_z_cell_reduces_to_2d3v(oracle_mod, bc):
    # with a single periodic z cell every z difference vanishes, the z shape
    # factors sum to one, and the z current of the prefix sums collapses to
    # q w v_z times the 2D path-averaged weight: the 3D step is the 2D step
    wl2 = W.small_case(nx=20, ny=12, ppc=2, bc_x=bc, pol="none", u_th=0.4, seed=21)
    wl3 = dataclasses.replace(wl2, dim=3, nz=1, dz_lambda=8.0)
    p2 = W.generate_particles(wl2)
    rng = np.random.default_rng(22)
    p3 = [dict(d, iz=np.zeros_like(d["ix"]), oz=rng.random(len(d["ix"]), dtype=np.float32)) for d in p2]
    f2 = W.random_fields(wl2, seed=23, e_amp=0.4, b_amp=0.4)
    f3 = {k: v[None] for k, v in f2.items()}
    s2 = oracle_mod.OracleSim(wl2, p2, fields=f2)
    s3 = oracle_mod.OracleSim(wl3, p3, fields=f3)
    assert type(s3).__name__ == "OracleSim3"
    s3.grid.dt = s2.grid.dt          # dz -> infinity limit of the 3D time step
    s3.rho_bg[...] = s2.rho_bg[None]
    for _ in range(6):
        s2.step(1)
        s3.step(1)
    for k in KEYS:
        a, b = s3.f[k][0], s2.f[k]
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max()), k
    for k in ("byL", "bzL"):
        np.testing.assert_allclose(s3.f[k][0], s2.f[k], atol=1e-12)
    q2, q3 = s2.p[0], s3.p[0]
    assert np.array_equal(q2["alive"], q3["alive"]) and q2["alive"].sum() < len(q2["alive"]) + (bc == "periodic")
    m = q2["alive"].astype(bool)
    for k in ("x", "y") + PKEYS:
        np.testing.assert_allclose(q3[k][m], q2[k][m], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(s3.gauss_residual()[0], s2.gauss_residual(), atol=1e-10)


# ---------------------------------------------------------------------------
# y <-> z mirror
# ---------------------------------------------------------------------------
def _T(a):
    return np.ascontiguousarray(np.swapaxes(a, 0, 1))


def _mirror_fields(f):
    # polar vectors (E, J): components swap; axial vectors (B): swap and flip
    g = dict(ex=_T(f["ex"]), ey=_T(f["ez"]), ez=_T(f["ey"]),
             bx=-_T(f["bx"]), by=-_T(f["bz"]), bz=-_T(f["by"]))
    if "jx" in f:
        g.update(jx=_T(f["jx"]), jy=_T(f["jz"]), jz=_T(f["jy"]))
    if "byL" in f:
        g["byL"] = -_T(f["bzL"])
        g["bzL"] = -_T(f["byL"])
    return g


def _mirror_parts(d):
    return dict(ix=d["ix"], iy=d["iz"], iz=d["iy"], ox=d["ox"], oy=d["oz"], oz=d["oy"],
                ux=d["ux"], uy=d["uz"], uz=d["uy"], sx=-d["sx"], sy=-d["sz"], sz=-d["sy"],
                w=d["w"], id=d["id"])


@pytest.mark.parametrize("bc", ["open", "periodic"])
def test_mirror_y_z_maps_runs_onto_runs(oracle_mod, bc):
    # ny = nz and dy = dz: reflecting the state in the plane y = z (E, J, u
    # polar; B, s axial) and running must equal running and then reflecting
    wl = W.small_case3(nx=16, ny=10, nz=10, ppc=2, bc_x=bc, pol="none", u_th=0.5, seed=31,
                       dy_lambda=1 / 11, dz_lambda=1 / 11)
    parts = W.generate_particles(wl)
    f = W.random_fields(wl, seed=32, e_amp=0.5, b_amp=0.5)
    a = oracle_mod.OracleSim(wl, parts, fields=f)
    b = oracle_mod.OracleSim(wl, [_mirror_parts(d) for d in parts], fields=_mirror_fields(f))
    for _ in range(5):
        a.step(1)
        b.step(1)
    ma = _mirror_fields(a.f)
    for k in KEYS + ("byL", "bzL"):
        scale = max(1.0, np.abs(b.f[k]).max())
        assert np.abs(ma[k] - b.f[k]).max() <= 1e-12 * scale, k
    pa, pb = a.p[0], b.p[0]
    assert np.array_equal(pa["alive"], pb["alive"])
    m = pa["alive"].astype(bool)
    for ka, kb, sg in (("x", "x", 1), ("y", "z", 1), ("z", "y", 1), ("ux", "ux", 1), ("uy", "uz", 1),
                       ("uz", "uy", 1), ("sx", "sx", -1), ("sy", "sz", -1), ("sz", "sy", -1)):
        np.testing.assert_allclose(sg * pa[ka][m], pb[kb][m], rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------------------
# Yee update in 3D
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["e", "b"])
def test_yee3_discrete_dispersion_oblique_mode(oracle_mod, which):
    # a standing plane mode cos(k.x) with amplitude A perpendicular to the
    # discrete wave vector kappa_i = (2/dx_i) sin(k_i dx_i/2), sampled at each
    # component's Yee position, is an eigenmode of the periodic vacuum mesh:
    # it oscillates as cos(n phi), sin^2(phi/2)/dt^2 = |kappa|^2/4
    nx, ny, nz = 24, 16, 12
    sim = oracle_mod.OracleSim(_vacuum3(nx, ny, nz, pol="none"), _empty3())
    g = sim.grid
    k = np.array([2 * math.pi * 3 / (nx * g.dx), 2 * math.pi * 2 / (ny * g.dy), 2 * math.pi * 1 / (nz * g.dz)])
    d = np.array([g.dx, g.dy, g.dz])
    kap = 2 / d * np.sin(k * d / 2)
    A = np.cross(kap, [0.3, -0.8, 0.5])
    A /= np.linalg.norm(A)
    stag = ({"ex": (0.5, 0, 0), "ey": (0, 0.5, 0), "ez": (0, 0, 0.5)} if which == "e" else
            {"bx": (0, 0.5, 0.5), "by": (0.5, 0, 0.5), "bz": (0.5, 0.5, 0)})
    shapes = {}
    for c, (key, (sx, sy, sz)) in enumerate(stag.items()):
        X = (np.arange(nx) + sx) * g.dx
        Y = (np.arange(ny) + sy) * g.dy
        Z = (np.arange(nz) + sz) * g.dz
        ph = k[0] * X[None, None, :] + k[1] * Y[None, :, None] + k[2] * Z[:, None, None]
        shapes[key] = A[c] * np.cos(ph)
        sim.f[key][...] = shapes[key]
    phi = 2 * math.asin(g.dt * np.linalg.norm(kap) / 2)
    N = 113
    sim.step(N)
    for key, s in shapes.items():
        np.testing.assert_allclose(sim.f[key], s * math.cos(N * phi), atol=3e-12)
    # sharp: the continuum frequency is visibly different after N steps
    assert abs(math.cos(N * phi) - math.cos(N * g.dt * np.linalg.norm(k))) > 1e-3


def test_div_b_and_gauss_invariants_periodic_3d(oracle_mod):
    wl = W.small_case3(nx=12, ny=10, nz=8, ppc=2, bc_x="periodic", u_th=0.3, seed=41)
    parts = W.generate_particles(wl)
    f = W.random_fields(wl, seed=42, e_amp=0.3, b_amp=0.3)
    sim = oracle_mod.OracleSim(wl, parts, fields=f)
    db0, ge0 = sim.div_b().copy(), sim.gauss_residual().copy()
    sim.step(25)
    np.testing.assert_allclose(sim.div_b(), db0, atol=1e-12)
    np.testing.assert_allclose(sim.gauss_residual(), ge0, atol=1e-11)


@pytest.mark.parametrize("cfl", [0.95, 0.99])
def test_open_boundary_is_stable_for_3d_fields(oracle_mod, cfl):
    # random vacuum fields varying along all axes, open x ends: the field
    # energy may rise transiently but must not grow
    wl = _vacuum3(40, 12, 10, bc="open", pol="none", cfl=cfl)
    sim = oracle_mod.OracleSim(wl, _empty3(), fields=W.random_fields(wl, seed=5, e_amp=0.1, b_amp=0.1))
    e0 = _energy(sim)
    es = []
    for _ in range(10):
        sim.step(40)
        es.append(_energy(sim))
    assert max(es) < 1.5 * e0, es
    assert es[-1] < e0, es


def test_gauss_law_from_neutral_start_with_laser_3d(oracle_mod):
    wl = W.small_case3(nx=40, ny=12, nz=10, ppc=2, a0=6.0, u_th=0.02, seed=43)
    sim = oracle_mod.OracleSim(wl, W.generate_particles(wl))
    assert np.abs(sim.gauss_residual()).max() < 1e-14
    sim.step(40)
    assert np.abs(sim.f["ey"]).max() > 1.0
    assert np.abs(sim.gauss_residual()).max() < 1e-11


# ---------------------------------------------------------------------------
# laser injection in 3D
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pol", ["lp-y", "cp"])
def test_laser3_plane_wave_limit(oracle_mod, pol):
    # waist >> box: a plane wave enters at x_min and moves in +x with
    # E_y = B_z (and E_z = -B_y), carrying the source waveform
    nx, a0 = 300, 2.0
    wl = _vacuum3(nx, 4, 4, bc="open", pol=pol, a0=a0, waist_lambda=1e6, fwhm_periods=4.0,
                  t_peak_periods=4.0, dx=1 / 16)
    sim = oracle_mod.OracleSim(wl, _empty3())
    g = sim.grid
    steps = int(round(12 * 2 * math.pi / g.dt))
    comp, key = (0, "ey") if pol == "lp-y" else (1, "ez")
    peak, rec, ref = 0.0, [], []
    for n in range(steps):
        sim.step(1)
        v = sim.f[key][1, 2, 120]
        peak = max(peak, abs(v))
        rec.append(v)
        ref.append(sim.laser((n + 1) * g.dt - 120 * g.dx, 2 * g.dy, 1.5 * g.dz, comp))
    amp = a0 if pol == "lp-y" else a0 / math.sqrt(2)
    assert peak == pytest.approx(amp, rel=0.02)
    rec, ref = np.array(rec), np.array(ref)
    assert rec @ ref / np.sqrt((rec @ rec) * (ref @ ref)) > 0.95
    sl = slice(20, nx - 40)
    ey, bz = sim.f["ey"][1, 2], sim.f["bz"][1, 2]
    assert np.abs(ey[1:-1][sl] - 0.5 * (bz[1:-1] + bz[:-2])[sl]).max() < 0.05 * a0
    ez, by = sim.f["ez"][1, 2], sim.f["by"][1, 2]
    assert np.abs(ez[1:-1][sl] + 0.5 * (by[1:-1] + by[:-2])[sl]).max() < 0.05 * a0
    if pol == "lp-y":
        assert np.abs(sim.f["ez"]).max() < 1e-12


def test_laser3_transverse_profile_is_centred_gaussian(oracle_mod):
    # a focused beam: E_y near x_min is mirror symmetric about the box axis
    # (y, z) = (ny dy/2, nz dz/2) and falls to about 1/e at radius w0
    ny = nz = 32
    wl = _vacuum3(64, ny, nz, bc="open", pol="lp-y", a0=1.0, waist_lambda=1.0, fwhm_periods=3.0,
                  t_peak_periods=3.0, dx=1 / 16, dy=1 / 8, dz=1 / 8)
    sim = oracle_mod.OracleSim(wl, _empty3())
    g = sim.grid
    nsteps = int(round(3 * 2 * math.pi / g.dt))
    best = None
    for _ in range(nsteps + 40):
        sim.step(1)
        e = sim.f["ey"][:, :, 2]
        if best is None or np.abs(e).max() > np.abs(best).max():
            best = e.copy()
    # Ey sits at y = (j+1/2) dy, z = k dz: the mirror images are j -> ny-1-j, k -> nz-k
    jm = ny - 1 - np.arange(ny)
    km = (nz - np.arange(nz)) % nz
    np.testing.assert_allclose(best[np.ix_(km, jm)], best, atol=1e-12)
    centre = best[nz // 2, ny // 2 - 1]
    assert abs(centre) == pytest.approx(np.abs(best).max(), rel=1e-12)
    # w0 = 8 cells: the node at y = 23.5 dy is 7.5 cells off axis, the centre
    # node 0.5 cells, so the ratio is exp(-(7.5^2 - 0.5^2) / 8^2)
    ratio = best[nz // 2, ny // 2 - 1 + 8] / centre
    assert ratio == pytest.approx(math.exp(-(7.5 ** 2 - 0.5 ** 2) / 64), rel=0.05)
    # and along z: the node 8 cells off axis in z (the same 0.5 cells in y)
    ratio_z = best[nz // 2 + 8, ny // 2 - 1] / centre
    assert ratio_z == pytest.approx(math.exp(-(8.0 ** 2) / 64), rel=0.05)


# ---------------------------------------------------------------------------
# gather and current in 3D
# ---------------------------------------------------------------------------
STAGGER3 = {"ex": (0.5, 0, 0), "ey": (0, 0.5, 0), "ez": (0, 0, 0.5),
            "bx": (0, 0.5, 0.5), "by": (0.5, 0, 0.5), "bz": (0.5, 0.5, 0)}


def _gather(oracle_mod, sim, X, Y, Z):
    E, B = (C.c_double * 3)(), (C.c_double * 3)()
    oracle_mod.lib().or3_gather(C.byref(sim.grid), C.byref(sim._fields()), X, Y, Z, E, B)
    return dict(zip(("ex", "ey", "ez", "bx", "by", "bz"), list(E) + list(B)))


def test_gather3_reproduces_linear_fields(oracle_mod):
    # trilinear interpolation is exact for fields linear in x, y and z,
    # provided every component is read at its own Yee position
    n = 12
    sim = oracle_mod.OracleSim(_vacuum3(n, n, n), _empty3())
    coef = {k: (0.3 + i, 0.11 * (i + 1), -0.07 * (i + 2), 0.05 * (3 - i)) for i, k in enumerate(STAGGER3)}
    for k, (sx, sy, sz) in STAGGER3.items():
        a, b, c, d = coef[k]
        X = np.arange(n) + sx
        sim.f[k][...] = a + b * X[None, None, :] + c * X[None, :, None] * 0 + c * (np.arange(n) + sy)[None, :, None] \
            + d * (np.arange(n) + sz)[:, None, None]
    rng = np.random.default_rng(7)
    for _ in range(60):
        X, Y, Z = rng.uniform(2, 9, 3)
        got = _gather(oracle_mod, sim, X, Y, Z)
        for k in STAGGER3:
            a, b, c, d = coef[k]
            assert got[k] == pytest.approx(a + b * X + c * Y + d * Z, rel=1e-13), k


def _deposit3(oracle_mod, X0, Y0, Z0, X1, Y1, Z1, qw, n=8):
    sim = oracle_mod.OracleSim(_vacuum3(n, n, n), _empty3())
    oracle_mod.lib().or3_deposit_one(C.byref(sim.grid), C.byref(sim._fields()), qw, X0, Y0, Z0, X1, Y1, Z1)
    return sim


def _rho3(X, Y, Z, qw, n):
    r = np.zeros((n, n, n))
    ax = np.arange(n)
    sx = np.clip(1 - np.abs(X - ax), 0, None)
    sy = np.clip(1 - np.abs(Y - ax), 0, None)
    sz = np.clip(1 - np.abs(Z - ax), 0, None)
    return qw * sz[:, None, None] * sy[None, :, None] * sx[None, None, :] + r


def test_esirkepov3_continuity_brute_force(oracle_mod):
    # (rho^{n+1} - rho^n)/dt + div J = 0 on every node, for random moves of
    # up to a cell along every axis; the total current is charge x velocity
    rng = np.random.default_rng(8)
    n = 8
    for _ in range(150):
        P0 = rng.uniform(2, 6, 3)
        dP = rng.uniform(-0.999, 0.999, 3)
        qw = rng.uniform(-1, 1)
        sim = _deposit3(oracle_mod, *P0, *(P0 + dP), qw, n)
        g = sim.grid
        jx, jy, jz = sim.f["jx"], sim.f["jy"], sim.f["jz"]
        divj = ((jx - np.roll(jx, 1, axis=2)) / g.dx + (jy - np.roll(jy, 1, axis=1)) / g.dy +
                (jz - np.roll(jz, 1, axis=0)) / g.dz)
        drho = _rho3(*(P0 + dP), qw, n) - _rho3(*P0, qw, n)
        np.testing.assert_allclose(drho / g.dt + divj, 0.0, atol=1e-13 * (1 + abs(qw) / g.dt))
        for key, dd, h in (("jx", dP[0], g.dx), ("jy", dP[1], g.dy), ("jz", dP[2], g.dz)):
            assert sim.f[key].sum() * g.dt == pytest.approx(qw * dd * h, rel=1e-12, abs=1e-15)


def test_esirkepov3_in_cell_current_is_path_average(oracle_mod):
    # a move inside one cell: J_x at (i+1/2, j+b, k+c) is q w (dx/dt) dX times
    # the average of S_y S_z along the straight path (brute-force quadrature);
    # likewise J_y and J_z.  A particle at rest carries no current.
    rng = np.random.default_rng(10)
    t = np.linspace(0.0, 1.0, 2001)

    def simpson(f):
        return (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum()) / (3 * 2000)

    for _ in range(20):
        P0 = 3 + rng.uniform(0.05, 0.95, 3)
        P1 = 3 + rng.uniform(0.05, 0.95, 3)
        qw = 0.8
        sim = _deposit3(oracle_mod, *P0, *P1, qw)
        g = sim.grid
        Pt = P0[None, :] + t[:, None] * (P1 - P0)[None, :]
        S = [np.stack([np.clip(1 - np.abs(Pt[:, a] - i), 0, None) for i in (3, 4)]) for a in range(3)]
        for b in (0, 1):
            for c in (0, 1):
                want_x = qw * g.dx / g.dt * (P1[0] - P0[0]) * simpson(S[1][b] * S[2][c])
                want_y = qw * g.dy / g.dt * (P1[1] - P0[1]) * simpson(S[0][b] * S[2][c])
                want_z = qw * g.dz / g.dt * (P1[2] - P0[2]) * simpson(S[0][b] * S[1][c])
                assert sim.f["jx"][3 + c, 3 + b, 3] == pytest.approx(want_x, rel=1e-9, abs=1e-13)
                assert sim.f["jy"][3 + c, 3, 3 + b] == pytest.approx(want_y, rel=1e-9, abs=1e-13)
                assert sim.f["jz"][3, 3 + c, 3 + b] == pytest.approx(want_z, rel=1e-9, abs=1e-13)
    sim = _deposit3(oracle_mod, 3.3, 4.1, 2.7, 3.3, 4.1, 2.7, 0.5)
    assert all(np.all(sim.f[k] == 0) for k in ("jx", "jy", "jz"))


def test_free_streaming_particle_3d(oracle_mod):
    # no fields: the position advances by dt u / gamma along each axis (in its
    # own cell size), u and s unchanged, periodic wrap in y and z
    wl = _vacuum3(10, 9, 8)
    u = np.array([0.6, -2.0, 1.5], dtype=np.float32)
    d = _empty3()[0]
    one = dict(ix=np.array([4], np.int32), iy=np.array([3], np.int32), iz=np.array([5], np.int32),
               ox=np.float32([0.25]), oy=np.float32([0.5]), oz=np.float32([0.75]),
               ux=u[:1], uy=u[1:2], uz=u[2:], sx=np.float32([1.0]), sy=np.float32([0.0]),
               sz=np.float32([0.0]), w=np.float32([1.0]), id=np.array([0], np.int32))
    assert set(one) == set(d)
    sim = oracle_mod.OracleSim(wl, [one])
    g = sim.grid
    uu = u.astype(float)
    gam = math.sqrt(1 + uu @ uu)
    for _ in range(30):
        sim.push(0)
    p = sim.p[0]
    assert p["x"][0] == pytest.approx((4.25 + 30 * g.dt * uu[0] / gam / g.dx) % 10, rel=1e-12)
    assert p["y"][0] == pytest.approx((3.5 + 30 * g.dt * uu[1] / gam / g.dy) % 9, rel=1e-12)
    assert p["z"][0] == pytest.approx((5.75 + 30 * g.dt * uu[2] / gam / g.dz) % 8, rel=1e-12)
    assert p["ux"][0] == uu[0] and p["sx"][0] == 1.0


def test_laser3_cp_components_are_staggered_like_e(oracle_mod):
    # CP beam: E_y sits at (j+1/2, k) and E_z at (j, k+1/2), so near x_min E_y
    # is mirror symmetric under j -> ny-1-j, k -> nz-k and E_z under
    # j -> ny-j, k -> nz-1-k (both about the box axis)
    ny = nz = 16
    wl = _vacuum3(24, ny, nz, bc="open", pol="cp", a0=1.0, waist_lambda=0.5, fwhm_periods=2.0,
                  t_peak_periods=0.5, dx=1 / 16, dy=1 / 8, dz=1 / 8)
    sim = oracle_mod.OracleSim(wl, _empty3())
    sim.step(10)
    ey, ez = sim.f["ey"][:, :, 2], sim.f["ez"][:, :, 2]
    assert np.abs(ey).max() > 0.05 and np.abs(ez).max() > 0.05
    jh, jn = ny - 1 - np.arange(ny), (ny - np.arange(ny)) % ny
    kh, kn = nz - 1 - np.arange(nz), (nz - np.arange(nz)) % nz
    np.testing.assert_allclose(ey[np.ix_(kn, jh)], ey, atol=1e-12 * np.abs(ey).max())
    np.testing.assert_allclose(ez[np.ix_(kh, jn)], ez, atol=1e-12 * np.abs(ez).max())


def test_split_calls_equal_the_whole_step_3d(oracle_mod):
    # as in 2D3V: the calls one by one are the whole step, bit for bit, with
    # the laser entering (the field update reads the step index for it)
    wl = W.small_case3(nx=20, ny=8, nz=6, ppc=1, u_th=0.3, two_species=True)
    parts = W.generate_particles(wl)
    a, b = oracle_mod.OracleSim(wl, parts, step=3), oracle_mod.OracleSim(wl, parts, step=3)
    a.step(3)
    for _ in range(3):
        b.zero_current()
        saved = [b.push(s) for s in range(len(b.p))]
        for s, old in enumerate(saved):
            b.deposit(s, *old)
        b.field_update()
    assert np.abs(a.f["ey"]).max() > 0
    for k in a.f:
        assert np.array_equal(a.f[k], b.f[k]), k
    for s in range(2):
        for k in a.p[s]:
            assert np.array_equal(a.p[s][k], b.p[s][k]), (s, k)


@pytest.mark.parametrize("dim", [2, 3])
def test_immobile_species_is_never_moved(oracle_mod, dim):
    # an immobile species (the ions) keeps its particles bit for bit through
    # whole steps in strong fields, while the mobile one moves
    wl = (W.small_case(nx=20, ny=8, ppc=1, u_th=0.3, two_species=True, bc_x="periodic", pol="none") if dim == 2
          else W.small_case3(nx=12, ny=8, nz=6, ppc=1, u_th=0.3, two_species=True, bc_x="periodic", pol="none"))
    wl = dataclasses.replace(wl, species=(wl.species[0], dataclasses.replace(wl.species[1], mobile=False)))
    parts = W.generate_particles(wl)
    sim = oracle_mod.OracleSim(wl, parts, fields=W.random_fields(wl, seed=8, e_amp=0.5, b_amp=0.5))
    before = {k: v.copy() for k, v in sim.p[1].items()}
    x0 = sim.p[0]["x"].copy()
    sim.step(3)
    for k, v in before.items():
        assert np.array_equal(sim.p[1][k], v), k
    assert not np.array_equal(sim.p[0]["x"], x0)


def test_spectra_of_3d_particles_are_those_of_their_momenta(oracle_mod):
    # the spectra read only u, s, w and the alive flag: a 3D3V species gives
    # the (pinned) 2D3V spectra of the same momenta, linear and log bins
    wl3 = W.small_case3(nx=12, ny=8, nz=6, ppc=2, u_th=0.8, bc_x="periodic")
    wl2 = W.small_case(nx=12, ny=8 * 6, ppc=2, u_th=0.8, bc_x="periodic")
    p3 = W.generate_particles(wl3)[0]
    p2 = {k: v for k, v in p3.items() if k not in ("iz", "oz")}
    p2["iy"] = (p3["iy"] + 8 * p3["iz"]).astype(np.int32)
    s3, s2 = oracle_mod.OracleSim(wl3, [p3]), oracle_mod.OracleSim(wl2, [p2])
    for log_bins, (lo, hi) in ((False, (0.0, 0.5)), (True, (0.01, 0.5))):
        np.testing.assert_array_equal(s3.histogram(0, lo, hi, 9, log_bins), s2.histogram(0, lo, hi, 9, log_bins))
    np.testing.assert_array_equal(s3.moments(0, 0.01, 0.5), s2.moments(0, 0.01, 0.5))
