"""Pins of the FP64 oracle to facts fixed outside the oracle itself.

Every test here checks the oracle against a closed form, an invariant, a
special case with a textbook answer, brute force, or values worked by hand
from Eq. (4) (tests/golden/).  None re-types the oracle's own formula.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cross(a, b):
    return np.cross(np.asarray(a, float), np.asarray(b, float))


# ---------------------------------------------------------------------------
# Boris push (a2)
# ---------------------------------------------------------------------------
def test_boris_pure_electric_field_is_exact_kick(oracle_mod):
    # with B = 0 the Boris scheme reduces to u^{n+1/2} = u^{n-1/2} + (q/m) E dt
    for qm, E, u in [(-1.0, (0.3, -2.0, 0.7), (0.1, 5.0, -3.0)),
                     (1 / 1836, (40.0, 1.0, 0.0), (0.0, 0.0, 0.0))]:
        dt = 0.2
        got = oracle_mod.boris(qm, dt, E, (0, 0, 0), u)
        want = np.asarray(u) + qm * dt * np.asarray(E)
        np.testing.assert_allclose(got, want, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("gamma_u", [0.01, 1.0, 30.0])
def test_boris_pure_magnetic_field_rotation_angle(oracle_mod, gamma_u):
    # pure B: |u| is conserved and u turns by exactly 2 atan(|q/m| B dt / (2 gamma))
    qm, dt, B0 = -1.0, 0.26, 1.7
    u = np.array([gamma_u, 0.0, 0.3 * gamma_u])   # has a component along B
    B = np.array([0.0, 0.0, B0])
    g = math.sqrt(1 + u @ u)
    un = oracle_mod.boris(qm, dt, (0, 0, 0), B, u)
    assert abs(np.linalg.norm(un) - np.linalg.norm(u)) < 1e-14 * np.linalg.norm(u)
    assert un[2] == pytest.approx(u[2], rel=1e-14)          # parallel part untouched
    ang = math.atan2(_cross(u[:2].tolist() + [0], un[:2].tolist() + [0])[2], u[:2] @ un[:2])
    want = 2 * math.atan(abs(qm) * B0 * dt / (2 * g))
    # an electron (q < 0) turns counter-clockwise about +B
    assert ang == pytest.approx(want, rel=1e-12)


def test_boris_crossed_fields_drift(oracle_mod):
    # E x B drift: for |E| < |B| the mean velocity is E x B / B^2
    qm, dt = -1.0, 0.02
    E, B = np.array([0.0, 0.3, 0.0]), np.array([0.0, 0.0, 1.0])
    u = np.zeros(3)
    x = np.zeros(3)
    steps = 20000
    for _ in range(steps):
        u = oracle_mod.boris(qm, dt, E, B, u)
        x += dt * u / math.sqrt(1 + u @ u)
    vd = x / (steps * dt)
    np.testing.assert_allclose(vd, _cross(E, B) / (B @ B), atol=3e-3)


def test_boris_plane_wave_drift_velocity(oracle_mod):
    # electron starting at rest at a zero of the vector potential of a linearly
    # polarised plane wave (E_y = B_z = a0 cos(t - x)) drifts along x at
    # a0^2 / (4 + a0^2), with the figure-of-eight amplitudes of the textbook
    # orbit
    a0, qm, dt = 1.5, -1.0, 2 * math.pi / 600
    x, t = 0.0, 0.0
    x_half = 0.0
    # positions at integer times, momentum at half times: u^{-1/2} is the
    # exact orbit of the electron at rest at t = 0, taken at t = -dt/2
    # (u_y = -a0 sin(phi), u_x = u_y^2 / 2); starting from u^{-1/2} = 0 would
    # leave the canonical momentum off by a0 dt / 2 and y drifting
    uy0 = a0 * math.sin(0.5 * dt)
    u = np.array([0.5 * uy0 ** 2, uy0, 0.0])
    periods = 0
    t0 = x0 = None
    phi_prev = 0.0
    y, ys, uxs = 0.0, [0.0], [0.0]
    while periods < 6:
        ph = t - x
        E = (0.0, a0 * math.cos(ph), 0.0)
        Bf = (0.0, 0.0, a0 * math.cos(ph))
        u = oracle_mod.boris(qm, dt, E, Bf, u)
        g = math.sqrt(1 + u @ u)
        x += dt * u[0] / g
        y += dt * u[1] / g
        ys.append(y)
        uxs.append(u[0])
        t += dt
        phi = t - x
        if math.floor(phi / (2 * math.pi)) > math.floor(phi_prev / (2 * math.pi)):
            # interpolate the crossing of phi = 2 pi k
            k = math.floor(phi / (2 * math.pi))
            fr = (2 * math.pi * k - phi_prev) / (phi - phi_prev)
            tc, xc = t - dt + fr * dt, x - dt * u[0] / g * (1 - fr)
            if t0 is None:
                t0, x0 = tc, xc
            periods += 1
        phi_prev = phi
    vd = (xc - x0) / (tc - t0)
    assert vd == pytest.approx(a0 ** 2 / (4 + a0 ** 2), rel=2e-3)
    # the figure of eight: u_y = -a0 sin(phi) (canonical momentum), so
    # y = a0 (cos(phi) - 1), a transverse excursion of 2 a0, and
    # u_x = u_y^2 / 2 peaks at a0^2 / 2
    assert max(ys) - min(ys) == pytest.approx(2 * a0, rel=2e-3)
    assert max(uxs) == pytest.approx(a0 ** 2 / 2, rel=2e-3)


# ---------------------------------------------------------------------------
# Thomas-BMT precession vector, Eqs. (2)-(3)
# ---------------------------------------------------------------------------
def test_omega_at_rest_is_one_plus_a_times_B(oracle_mod):
    # gamma = 1: Eq. (3) gives Om_B = 1 + a; the v terms vanish
    for qm, a in [(-1.0, 0.00116), (1 / 1836, 1.793)]:
        B = np.array([0.2, -1.1, 0.7])
        E = np.array([3.0, 1.0, -2.0])
        Om = oracle_mod.omega(qm, a, (0, 0, 0), E, B)
        np.testing.assert_allclose(Om, qm * (1 + a) * B, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("gam", [1.5, 10.0, 2000.0])
def test_omega_longitudinal_field(oracle_mod, gam):
    # v parallel to B, E = 0: the spin precesses about B at (q/m)(1 + a) B / gamma
    # (textbook: longitudinal spin precession is not enhanced by gamma)
    qm, a = -1.0, 0.00116
    u = math.sqrt(gam ** 2 - 1) * np.array([1.0, 2.0, -2.0]) / 3.0
    B = 0.8 * np.array([1.0, 2.0, -2.0]) / 3.0
    Om = oracle_mod.omega(qm, a, u, (0, 0, 0), B)
    np.testing.assert_allclose(Om, qm * (1 + a) * B / gam, rtol=1e-12)


@pytest.mark.parametrize("gam", [1.2, 5.0, 100.0])
def test_omega_transverse_field_spin_tune(oracle_mod, gam):
    # v perpendicular to B, E = 0: relative to the momentum (which turns at
    # (q/m) B / gamma) the spin turns at (q/m) a B: spin tune a gamma
    qm, a = 1 / 1836, 1.793
    u = math.sqrt(gam ** 2 - 1) * np.array([1.0, 0.0, 0.0])
    B = np.array([0.0, 0.0, 2.5])
    Om = oracle_mod.omega(qm, a, u, (0, 0, 0), B)
    np.testing.assert_allclose(Om - qm * B / gam, qm * a * B, rtol=1e-12, atol=1e-15)


def test_omega_magic_energy_freezes_spin_relative_to_momentum(oracle_mod):
    # pure E perpendicular to v: spin and momentum turn together when
    # a = 1/(gamma^2 - 1) (the 'magic' momentum of electrostatic storage rings,
    # 0.7007 GeV/c for protons)
    qm, a = 1 / 1836, 1.793
    gam = math.sqrt(1 + 1 / a)
    assert math.sqrt(gam ** 2 - 1) * 938.272 == pytest.approx(700.7, abs=0.1)
    uhat = np.array([0.6, 0.8, 0.0])
    u = math.sqrt(gam ** 2 - 1) * uhat
    E = np.array([-0.8, 0.6, 0.0]) * 7.0
    Om = oracle_mod.omega(qm, a, u, E, (0, 0, 0))
    # ds/dt = -Om x s rotates s with angular velocity -Om; u rotates with
    # (q/m) (uhat x E) / |u|  (du/dt = (q/m) E)
    w_u = qm * _cross(uhat, E) / np.linalg.norm(u)
    np.testing.assert_allclose(-Om, w_u, rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------------------
# Spin rotation through a whole particle push (a1-a4 on the mesh)
# ---------------------------------------------------------------------------
def _one_particle_sim(oracle_mod, fields, u=(0, 0, 0), s=(1, 0, 0), species=None, nx=16, ny=16):
    sp = species or W.Species("e", q=-1.0, m=1.0, a=0.00116, n0=0.01, ppc=1, u_th=0.0,
                              s0=tuple(s))
    wl = W.Workload(name="one", nx=nx, ny=ny, dx_lambda=1 / 16, dy_lambda=1 / 12, cfl=0.95,
                    steps=1, species=(sp,), pol="none", bc_x="periodic")
    f32 = np.float32
    parts = [dict(ix=np.array([nx // 2], np.int32), iy=np.array([ny // 2], np.int32),
                  ox=np.array([0.3], f32), oy=np.array([0.6], f32),
                  ux=np.array([u[0]], f32), uy=np.array([u[1]], f32), uz=np.array([u[2]], f32),
                  sx=np.array([s[0]], f32), sy=np.array([s[1]], f32), sz=np.array([s[2]], f32),
                  w=np.array([1e-12], f32), id=np.array([0], np.int32))]
    full = {k: np.full((ny, nx), v) for k, v in fields.items()}
    return oracle_mod.OracleSim(wl, parts, fields=full)


def test_spin_precession_in_uniform_B_at_rest(oracle_mod):
    # particle at rest in uniform B_z: after N pushes the spin has turned by
    # exactly N (1 + a) |q/m| B dt, counter-clockwise about +z for an electron,
    # and |s| stays 1
    B0 = 0.9
    sim = _one_particle_sim(oracle_mod, {"bz": B0})
    dt = sim.grid.dt
    N = 50
    for _ in range(N):
        sim.push(0)       # fields are not advanced: uniform static B
    p = sim.p[0]
    s = np.array([p["sx"][0], p["sy"][0], p["sz"][0]])
    th = N * (1 + 0.00116) * B0 * dt
    np.testing.assert_allclose(s, [math.cos(th), math.sin(th), 0.0], atol=1e-13)
    assert np.linalg.norm(s) == pytest.approx(1.0, abs=1e-14)
    assert p["ux"][0] == 0.0 and p["uy"][0] == 0.0


def test_spin_follows_momentum_when_anomaly_zero(oracle_mod):
    # a = 0, E = 0 (g = 2): the spin turns with the momentum; the Boris and the
    # spin rotation angles differ only at third order in (omega dt)
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    sim = _one_particle_sim(oracle_mod, {"bz": 0.05}, u=(0.5, 0, 0), s=(1, 0, 0), species=sp,
                            nx=64, ny=64)
    angles = []
    for _ in range(120):
        sim.push(0)
        p = sim.p[0]
        u = np.array([p["ux"][0], p["uy"][0]])
        s = np.array([p["sx"][0], p["sy"][0]])
        angles.append(math.atan2(u[0] * s[1] - u[1] * s[0], u @ s))
    # the momentum at half steps vs the spin at half steps: both turn ~0.03 rad/step
    assert max(abs(a) for a in angles) < 1e-4


# ---------------------------------------------------------------------------
# Esirkepov deposit (a5): discrete continuity, brute force
# ---------------------------------------------------------------------------
def _deposit_case(oracle_mod, X0, Y0, X1, Y1, vz, qw=-0.37, nx=8, ny=8):
    import ctypes as C
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    wl = W.Workload(name="dep", nx=nx, ny=ny, dx_lambda=1 / 16, dy_lambda=1 / 12, cfl=0.95,
                    steps=1, species=(sp,), pol="none", bc_x="periodic")
    sim = oracle_mod.OracleSim(wl, [dict(ix=np.zeros(0, np.int32), iy=np.zeros(0, np.int32),
                                         **{k: np.zeros(0, np.float32) for k in
                                            ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w")},
                                         id=np.zeros(0, np.int32))])
    oracle_mod.lib().or_deposit_one(C.byref(sim.grid), C.byref(sim._fields()), qw, X0, Y0, X1, Y1, vz)
    return sim


def _rho_point(X, Y, qw, nx, ny):
    # CIC charge of one particle at nodes (brute force over all nodes)
    r = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            dxs = min(abs(X - i), nx - abs(X - i))
            dys = min(abs(Y - j), ny - abs(Y - j))
            r[j, i] = qw * max(0.0, 1 - dxs) * max(0.0, 1 - dys)
    return r


def test_esirkepov_continuity_brute_force(oracle_mod):
    rng = np.random.default_rng(5)
    nx = ny = 8
    for _ in range(200):
        X0, Y0 = rng.uniform(2, 6, 2)
        dX, dY = rng.uniform(-0.999, 0.999, 2)
        qw, vz = rng.uniform(-1, 1), rng.uniform(-1, 1)
        sim = _deposit_case(oracle_mod, X0, Y0, X0 + dX, Y0 + dY, vz, qw=qw)
        g = sim.grid
        jx, jy = sim.f["jx"], sim.f["jy"]
        divj = (jx - np.roll(jx, 1, axis=1)) / g.dx + (jy - np.roll(jy, 1, axis=0)) / g.dy
        drho = _rho_point(X0 + dX, Y0 + dY, qw, nx, ny) - _rho_point(X0, Y0, qw, nx, ny)
        np.testing.assert_allclose(drho / g.dt + divj, 0.0, atol=1e-13 * (1 + abs(qw) / g.dt))
        # the zero mode: total current = charge x mean velocity
        assert jx.sum() * g.dt == pytest.approx(qw * dX * g.dx, rel=1e-12, abs=1e-15)
        assert jy.sum() * g.dt == pytest.approx(qw * dY * g.dy, rel=1e-12, abs=1e-15)
        assert sim.f["jz"].sum() == pytest.approx(qw * vz, rel=1e-12, abs=1e-15)


def test_esirkepov_particle_at_rest_and_x_move(oracle_mod):
    X0, Y0, qw, vz = 3.3, 4.8, 0.5, 0.25
    sim = _deposit_case(oracle_mod, X0, Y0, X0, Y0, vz, qw=qw)
    assert np.all(sim.f["jx"] == 0) and np.all(sim.f["jy"] == 0)
    np.testing.assert_allclose(sim.f["jz"], qw * vz * _rho_point(X0, Y0, 1.0, 8, 8), atol=1e-16)
    sim = _deposit_case(oracle_mod, X0, Y0, X0 + 0.7, Y0, vz, qw=qw)
    assert np.all(sim.f["jy"] == 0)
    assert np.abs(sim.f["jx"]).max() > 0


# ---------------------------------------------------------------------------
# Yee update (a6)
# ---------------------------------------------------------------------------
def _vacuum(nx, ny, bc="periodic", **kw):
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.0, ppc=0, u_th=0.0, s0=(1, 0, 0))
    return W.Workload(name="vac", nx=nx, ny=ny, dx_lambda=1 / 16, dy_lambda=1 / 10, cfl=0.9,
                      steps=1, species=(sp,), bc_x=bc, **kw)


def _empty():
    return [dict(ix=np.zeros(0, np.int32), iy=np.zeros(0, np.int32),
                 **{k: np.zeros(0, np.float32) for k in
                    ("ox", "oy", "ux", "uy", "uz", "sx", "sy", "sz", "w")},
                 id=np.zeros(0, np.int32))]


@pytest.mark.parametrize("mode", ["tm", "te"])
def test_yee_discrete_dispersion_standing_wave(oracle_mod, mode):
    # a standing eigenmode cos(k.x) of the periodic vacuum mesh oscillates as
    # cos(n phi) with sin^2(phi/2)/dt^2 = sum_i sin^2(k_i dx_i/2)/dx_i^2  (Yee)
    nx, ny, mx, my = 48, 30, 5, 3
    wl = _vacuum(nx, ny, pol="none")
    sim = oracle_mod.OracleSim(wl, _empty())
    g = sim.grid
    kx, ky = 2 * math.pi * mx / (nx * g.dx), 2 * math.pi * my / (ny * g.dy)
    # TM: Ez at nodes (i, j); TE: Bz at (i+1/2, j+1/2)
    sh = 0.0 if mode == "tm" else 0.5
    X = (np.arange(nx) + sh) * g.dx
    Y = (np.arange(ny) + sh) * g.dy
    shape = np.cos(kx * X[None, :] + ky * Y[:, None])
    sim.f["ez" if mode == "tm" else "bz"][...] = shape
    phi = 2 * math.asin(g.dt * math.sqrt((math.sin(kx * g.dx / 2) / g.dx) ** 2 +
                                         (math.sin(ky * g.dy / 2) / g.dy) ** 2))
    N = 137
    sim.step(N)
    got = sim.f["ez" if mode == "tm" else "bz"]
    np.testing.assert_allclose(got, shape * math.cos(N * phi), atol=2e-12)
    # the continuum frequency would be visibly off: the pin is sharp
    assert abs(math.cos(N * phi) - math.cos(N * g.dt * math.hypot(kx, ky))) > 1e-3


def test_div_b_and_gauss_invariants_periodic(oracle_mod):
    wl = W.small_case(nx=24, ny=20, ppc=3, bc_x="periodic", u_th=0.3)
    parts = W.generate_particles(wl)
    f = W.random_fields(wl, seed=3, e_amp=0.3, b_amp=0.3)
    sim = oracle_mod.OracleSim(wl, parts, fields=f)
    db0 = sim.div_b().copy()
    ge0 = sim.gauss_residual().copy()
    sim.step(30)
    np.testing.assert_allclose(sim.div_b(), db0, atol=1e-12)
    np.testing.assert_allclose(sim.gauss_residual(), ge0, atol=1e-11)


def test_gauss_law_holds_from_neutral_start_with_laser(oracle_mod):
    # neutral start (immobile ions = -rho_e), open x with the laser entering:
    # div E - rho stays at round-off on the interior nodes
    wl = W.small_case(nx=64, ny=24, ppc=2, a0=6.0, u_th=0.02)
    sim = oracle_mod.OracleSim(wl, W.generate_particles(wl))
    assert np.abs(sim.gauss_residual()).max() < 1e-14
    sim.step(60)
    assert np.abs(sim.f["ey"]).max() > 1.0      # the laser is in the box
    assert np.abs(sim.gauss_residual()).max() < 1e-11


def test_laser_injection_amplitude_and_direction(oracle_mod):
    # plane-wave limit (waist >> box): the wave injected at x_min moves in +x
    # with E_y = B_z and peak |E_y| = a0
    nx, ny, a0 = 400, 4, 2.0
    wl = _vacuum(nx, ny, bc="open", pol="lp-y", a0=a0, waist_lambda=1e6, fwhm_periods=4.0,
                 t_peak_periods=4.0)
    sim = oracle_mod.OracleSim(wl, _empty())
    g = sim.grid
    steps = int(round(14 * 2 * math.pi / g.dt))
    peak = 0.0
    rec, ref = [], []
    for n in range(steps):
        sim.step(1)
        peak = max(peak, abs(sim.f["ey"][0, 150]))
        rec.append(sim.f["ey"][0, 150])
        ref.append(sim.laser((n + 1) * g.dt - 150 * g.dx, 0.5 * g.dy, 0))
    assert peak == pytest.approx(a0, rel=0.02)
    # the wave at x is the source waveform delayed by x / c (same sign)
    rec, ref = np.array(rec), np.array(ref)
    assert rec @ ref / np.sqrt((rec @ rec) * (ref @ ref)) > 0.95
    ey, bz = sim.f["ey"][0], sim.f["bz"][0]
    # B_z on (i+1/2): average to nodes; right-moving wave has B_z = E_y
    bz_n = 0.5 * (bz[1:-1] + bz[:-2])
    sl = slice(20, nx - 40)
    assert np.abs(ey[1:-1][sl] - bz_n[sl]).max() < 0.05 * a0
    assert np.abs(sim.f["ez"]).max() == 0.0


def test_silver_mueller_absorbs_outgoing_pulse(oracle_mod):
    # a right-moving pulse leaves through x_max; what stays in the box is the
    # first-order boundary's reflection, a small fraction of the energy
    nx, ny = 300, 4
    wl = _vacuum(nx, ny, bc="open", pol="none")
    sim = oracle_mod.OracleSim(wl, _empty())
    g = sim.grid
    xn = np.arange(nx) * g.dx
    xh = (np.arange(nx) + 0.5) * g.dx
    x0, wid = 200 * g.dx, 2 * math.pi
    sim.f["ey"][...] = np.exp(-((xn - x0) / wid) ** 2)[None, :]
    # B_z^0 chosen for a right-moving pulse (B_z = E_y at t = 0 and half a step later)
    sim.f["bz"][...] = np.exp(-((xh - x0) / wid) ** 2)[None, :]
    e0 = (sim.f["ey"] ** 2 + sim.f["bz"] ** 2).sum()
    sim.step(int(250 * g.dx / g.dt))
    e1 = (sim.f["ey"] ** 2 + sim.f["bz"] ** 2).sum()
    assert e1 < 1e-3 * e0


# ---------------------------------------------------------------------------
# Eq. (4): polarisation
# ---------------------------------------------------------------------------
def _read_golden():
    parts, cases = [], []
    with open(os.path.join(GOLDEN, "polarization_eq4.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "particle":
                parts.append([float(v) for v in t[1:]])
            elif t[0] == "case":
                w = [float(v) for v in t[1].split(",")]
                cases.append((w, float(t[2]), float(t[3]), [float(v) for v in t[4:7]], int(t[7])))
    return np.array(parts), cases


def test_polarization_eq4_hand_built_ensemble(oracle_mod):
    P, cases = _read_golden()
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    wl = W.Workload(name="p", nx=8, ny=8, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=0.95,
                    steps=1, species=(sp,), pol="none", bc_x="periodic")
    for w, emin, emax, want, cnt in cases:
        n = len(P)
        f32 = np.float32
        d = dict(ix=np.full(n, 3, np.int32), iy=np.full(n, 3, np.int32),
                 ox=np.full(n, 0.5, f32), oy=np.full(n, 0.5, f32),
                 ux=P[:, 0].astype(f32), uy=P[:, 1].astype(f32), uz=P[:, 2].astype(f32),
                 sx=P[:, 3].astype(f32), sy=P[:, 4].astype(f32), sz=P[:, 5].astype(f32),
                 w=np.array(w, f32), id=np.arange(n, dtype=np.int32))
        sim = oracle_mod.OracleSim(wl, [d])
        m = sim.moments(0, emin, emax)
        np.testing.assert_allclose(m[:3], want, atol=1e-15)
        assert m[4] == cnt


def test_polarization_unchanged_without_fields(oracle_mod):
    # particles at rest, no laser, neutral: no current, no field, no precession,
    # so P = s0 exactly after any number of steps
    wl = W.small_case(nx=24, ny=16, ppc=2, pol="none", a0=0.0, u_th=0.0, bc_x="periodic")
    sim = oracle_mod.OracleSim(wl, W.generate_particles(wl))
    sim.step(10)
    m = sim.moments(0)
    np.testing.assert_array_equal(m[:3], [0.0, 1.0, 0.0])
    assert m[4] == len(sim.p[0]["x"])


def test_workload_parameter_consistency():
    # Sec. 2 setup: n_H + n_T = n_e (HT target) and the 2D3V cases built here
    assert 1e20 + 1.4e21 == pytest.approx(1.5e21)
    assert W.CONFIG1.species[0].ppc * W.CONFIG1.nx * W.CONFIG1.ny == 131072
    assert sum(s.ppc for s in W.CONFIG3.species) * W.CONFIG3.nx * W.CONFIG3.ny == 67108864


# ---------------------------------------------------------------------------
# further pins: gather layout, free streaming, the z-current weight, CP laser,
# and the time centring of the spin update
# ---------------------------------------------------------------------------
STAGGER = {"ex": (0.5, 0.0), "ey": (0.0, 0.5), "ez": (0.0, 0.0),
           "bx": (0.0, 0.5), "by": (0.5, 0.0), "bz": (0.5, 0.5)}


def test_gather_reproduces_linear_fields(oracle_mod):
    # CIC interpolation is exact for fields linear in x and y, provided every
    # component is read at its own Yee position (layout in pic_oracle.h)
    nx, ny = 16, 16
    coef = {k: (0.3 + i, 0.11 * (i + 1), -0.07 * (i + 2)) for i, k in enumerate(STAGGER)}
    fields = {}
    for k, (sx, sy) in STAGGER.items():
        X = np.arange(nx) + sx
        Y = np.arange(ny) + sy
        a, b, c = coef[k]
        fields[k] = a + b * X[None, :] + c * Y[:, None]
    sim = _one_particle_sim(oracle_mod, {})
    for k, v in fields.items():
        sim.f[k][...] = v
    import ctypes as C
    rng = np.random.default_rng(2)
    for _ in range(50):
        X, Y = rng.uniform(3, 12, 2)
        E, B = (C.c_double * 3)(), (C.c_double * 3)()
        oracle_mod.lib().or_gather(C.byref(sim.grid), C.byref(sim._fields()), X, Y, E, B)
        got = dict(zip(("ex", "ey", "ez", "bx", "by", "bz"), list(E) + list(B)))
        for k in STAGGER:
            a, b, c = coef[k]
            assert got[k] == pytest.approx(a + b * X + c * Y, rel=1e-13)


def test_free_streaming_particle(oracle_mod):
    # no fields: x^{n+1} = x^n + dt u / gamma, u and s unchanged, periodic wrap in y
    sim = _one_particle_sim(oracle_mod, {}, u=(0.6, -2.0, 0.5), nx=16, ny=16)
    g = sim.grid
    u = np.array([0.6, -2.0, 0.5], dtype=np.float32).astype(float)
    gam = math.sqrt(1 + u @ u)
    x0, y0 = sim.p[0]["x"][0], sim.p[0]["y"][0]
    for _ in range(40):
        sim.push(0)
    assert sim.p[0]["x"][0] == pytest.approx((x0 + 40 * g.dt * u[0] / gam / g.dx) % 16, rel=1e-12)
    assert sim.p[0]["y"][0] == pytest.approx((y0 + 40 * g.dt * u[1] / gam / g.dy) % 16, rel=1e-12)
    assert sim.p[0]["ux"][0] == u[0] and sim.p[0]["sx"][0] == 1.0


def test_esirkepov_z_current_is_path_average_of_shape(oracle_mod):
    # for a move that crosses no node line, Wz is the average of Sx Sy along the
    # straight path (quadrature by brute force)
    rng = np.random.default_rng(9)
    for _ in range(30):
        X0, Y0 = 3 + rng.uniform(0.05, 0.95, 2)
        X1 = 3 + rng.uniform(0.05, 0.95)
        Y1 = 3 + rng.uniform(0.05, 0.95)
        qw, vz = 0.7, -0.4
        sim = _deposit_case(oracle_mod, X0, Y0, X1, Y1, vz, qw=qw)
        t = np.linspace(0.0, 1.0, 2001)
        Xt, Yt = X0 + t * (X1 - X0), Y0 + t * (Y1 - Y0)
        for (i, j) in [(3, 3), (4, 3), (3, 4), (4, 4)]:
            sxy = np.clip(1 - np.abs(Xt - i), 0, None) * np.clip(1 - np.abs(Yt - j), 0, None)
            avg = (sxy[0] + sxy[-1] + 4 * sxy[1:-1:2].sum() + 2 * sxy[2:-1:2].sum()) / (3 * 2000)
            assert sim.f["jz"][j, i] == pytest.approx(qw * vz * avg, rel=1e-10, abs=1e-14)


def test_cp_laser_injection(oracle_mod):
    # circular polarisation: both transverse pairs move in +x (E_y = B_z,
    # E_z = -B_y), each with peak a0/sqrt(2)
    nx, ny, a0 = 400, 4, 3.0
    wl = _vacuum(nx, ny, bc="open", pol="cp", a0=a0, waist_lambda=1e6, fwhm_periods=4.0,
                 t_peak_periods=4.0)
    sim = oracle_mod.OracleSim(wl, _empty())
    g = sim.grid
    steps = int(round(14 * 2 * math.pi / g.dt))
    pk_y = pk_z = 0.0
    rec, ref = [], []
    for n in range(steps):
        sim.step(1)
        pk_y = max(pk_y, abs(sim.f["ey"][0, 150]))
        pk_z = max(pk_z, abs(sim.f["ez"][0, 150]))
        rec.append(sim.f["ez"][0, 150])
        ref.append(sim.laser((n + 1) * g.dt - 150 * g.dx, 0.0, 1))
    rec, ref = np.array(rec), np.array(ref)
    assert rec @ ref / np.sqrt((rec @ rec) * (ref @ ref)) > 0.95
    assert pk_y == pytest.approx(a0 / math.sqrt(2), rel=0.02)
    assert pk_z == pytest.approx(a0 / math.sqrt(2), rel=0.02)
    ez, by = sim.f["ez"][0], sim.f["by"][0]
    by_n = 0.5 * (by[1:-1] + by[:-2])
    sl = slice(20, nx - 40)
    assert np.abs(ez[1:-1][sl] + by_n[sl]).max() < 0.05 * a0


def test_spin_update_is_second_order_in_dt(oracle_mod):
    # uniform static E and B: the oracle's staggered push (u, s at half steps)
    # converges at second order to an accurate integration of the Lorentz
    # force and Eqs. (1)-(3)
    from scipy.integrate import solve_ivp
    qm, a = -1.0, 0.5
    E = np.array([0.05, 0.02, 0.0])
    B = np.array([0.0, 0.1, 0.3])

    def rhs(t, y):
        u, s = y[:3], y[3:]
        g = math.sqrt(1 + u @ u)
        v = u / g
        Om = qm * ((a + 1 / g) * B - a * g / (g + 1) * (v @ B) * v - (a + 1 / (1 + g)) * np.cross(v, E))
        return np.concatenate([qm * (E + np.cross(v, B)), -np.cross(Om, s)])

    y0 = np.array([0.5, 0.0, 0.2, 0.0, 0.6, 0.8])
    T = 30.0
    errs = []
    for cfl in (0.8, 0.4, 0.2):
        sp = W.Species("e", q=-1.0, m=1.0, a=a, n0=0.01, ppc=1, u_th=0.0, s0=(0, 0.6, 0.8))
        wl = W.Workload(name="cv", nx=16, ny=16, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=cfl,
                        steps=1, species=(sp,), pol="none", bc_x="periodic")
        dt = oracle_mod.derive_grid(wl).dt
        nsteps = int(round(T / dt))
        back = solve_ivp(rhs, (0, -dt / 2), y0, rtol=1e-12, atol=1e-14).y[:, -1]
        sim = _one_particle_sim(oracle_mod, {}, species=sp)
        sim.grid.dt = dt
        for k, v in zip(("ex", "ey", "ez", "bx", "by", "bz"), list(E) + list(B)):
            sim.f[k][...] = v
        p = sim.p[0]
        for k, v in zip(("ux", "uy", "uz", "sx", "sy", "sz"), back):
            p[k][0] = v
        for _ in range(nsteps):
            sim.push(0)
        ref = solve_ivp(rhs, (0, nsteps * dt - dt / 2), y0, rtol=1e-12, atol=1e-14).y[:, -1]
        s = np.array([p["sx"][0], p["sy"][0], p["sz"][0]])
        errs.append(np.linalg.norm(s - ref[3:]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


@pytest.mark.parametrize("dy_lambda,cfl", [(1 / 16, 0.95), (1 / 32, 0.99), (1 / 10, 0.9)])
def test_open_boundary_is_stable_for_2d_fields(oracle_mod, dy_lambda, cfl):
    # random vacuum fields varying along x and y in a box with open x ends:
    # the field energy may only decrease (first-order absorbing boundary)
    nx, ny = 64, 32
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.0, ppc=0, u_th=0.0, s0=(1, 0, 0))
    wl = W.Workload(name="vac", nx=nx, ny=ny, dx_lambda=1 / 16, dy_lambda=dy_lambda, cfl=cfl,
                    steps=1, species=(sp,), bc_x="open", pol="none")
    f = W.random_fields(wl, seed=4, e_amp=0.1, b_amp=0.1)
    sim = oracle_mod.OracleSim(wl, _empty(), fields=f)

    def energy():
        return sum((sim.f[k] ** 2).sum() for k in ("ex", "ey", "ez", "bx", "by", "bz"))

    # (E^2 + B^2 at one time level is not the exactly conserved discrete
    # energy of the leapfrog scheme, so allow transient rises, not growth)
    e0 = energy()
    es = []
    for _ in range(12):
        sim.step(50)
        es.append(energy())
    assert max(es) < 1.5 * e0, es
    assert es[-1] < e0, es


def test_histogram_hand_built_spectrum(oracle_mod):
    P, _ = _read_golden()
    want = []
    with open(os.path.join(GOLDEN, "histogram_dpde.txt")) as fh:
        for line in fh:
            t = line.split()
            if t and t[0] == "bin":
                want.append([float(v) for v in t[2:]])
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    wl = W.Workload(name="h", nx=8, ny=8, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=0.95,
                    steps=1, species=(sp,), pol="none", bc_x="periodic")
    n, f32 = len(P), np.float32
    d = dict(ix=np.full(n, 3, np.int32), iy=np.full(n, 3, np.int32), ox=np.full(n, 0.5, f32),
             oy=np.full(n, 0.5, f32), ux=P[:, 0].astype(f32), uy=P[:, 1].astype(f32),
             uz=P[:, 2].astype(f32), sx=P[:, 3].astype(f32), sy=P[:, 4].astype(f32),
             sz=P[:, 5].astype(f32), w=np.array([1, 1, 2, 4], f32), id=np.arange(n, dtype=np.int32))
    sim = oracle_mod.OracleSim(wl, [d])
    np.testing.assert_allclose(sim.histogram(0, 0.0, 3.0, 3), np.array(want), atol=1e-15)


@pytest.mark.parametrize("log_bins", [False, True])
def test_histogram_sums_to_the_eq4_moments(oracle_mod, log_bins):
    # summing the bins gives back the count, weight and weighted spin of the
    # whole window (Eq. 4 over the window); dP/dE of one bin is Eq. (4) over it
    wl = W.small_case(nx=24, ny=16, ppc=4, u_th=0.8, bc_x="periodic")
    sim = oracle_mod.OracleSim(wl, W.generate_particles(wl))
    sim.p[0]["sx"][:] = np.cos(np.arange(len(sim.p[0]["sx"])))
    sim.p[0]["sy"][:] = np.sin(np.arange(len(sim.p[0]["sx"])))
    emin, emax = (0.01, 0.5) if log_bins else (0.0, 0.5)
    h = sim.histogram(0, emin, emax, 17, log_bins)
    m = sim.moments(0, emin, emax)
    assert h[:, 0].sum() == m[4]
    assert h[:, 1].sum() == pytest.approx(m[3], rel=1e-13)
    np.testing.assert_allclose(h[:, 2:5].sum(axis=0) / h[:, 1].sum(), m[:3], atol=1e-13)
    b = int(np.argmax(h[:, 0]))
    edges = (emin * (emax / emin) ** (np.arange(18) / 17) if log_bins
             else emin + (emax - emin) * np.arange(18) / 17)
    mb = sim.moments(0, edges[b], edges[b + 1])
    assert h[b, 0] == mb[4]
    np.testing.assert_allclose(h[b, 2:5] / h[b, 1], mb[:3], atol=1e-12)


# ---------------------------------------------------------------------------
# a4 and the current's v_z use the new momentum u^{n+1/2}
# ---------------------------------------------------------------------------
def test_advance_and_vz_use_the_new_momentum(oracle_mod):
    # from rest in uniform E (B = 0) one push gives u^{n+1/2} = (q/m) E dt
    # exactly (Boris' kick); the particle then moves by dt u / gamma(u) and the
    # out-of-plane velocity handed to the deposit is u_z / gamma(u)
    E = (0.4, -0.3, 0.7)
    sim = _one_particle_sim(oracle_mod, {"ex": E[0], "ey": E[1], "ez": E[2]})
    g = sim.grid
    x0, y0 = float(sim.p[0]["x"][0]), float(sim.p[0]["y"][0])
    _, _, vz = sim.push(0)
    u = -1.0 * g.dt * np.asarray(E)
    gam = math.sqrt(1.0 + u @ u)
    p = sim.p[0]
    np.testing.assert_allclose([p["ux"][0], p["uy"][0], p["uz"][0]], u, rtol=1e-14)
    assert p["x"][0] == pytest.approx(x0 + g.dt * u[0] / gam / g.dx, rel=1e-14)
    assert p["y"][0] == pytest.approx(y0 + g.dt * u[1] / gam / g.dy, rel=1e-14)
    assert vz[0] == pytest.approx(u[2] / gam, rel=1e-14)


# ---------------------------------------------------------------------------
# a6 with a current: Ampere's law, and div E with unequal cells
# ---------------------------------------------------------------------------
def test_uniform_current_drives_e_by_minus_dt_j(oracle_mod):
    # dE/dt = curl B - J: with no fields and a uniform current every E
    # component changes by exactly -dt J in one update, and B stays zero
    wl = _vacuum(12, 10)
    sim = oracle_mod.OracleSim(wl, _empty())
    J = {"jx": 0.3, "jy": -0.7, "jz": 1.1}
    for k, v in J.items():
        sim.f[k][...] = v
    sim.field_update()
    dt = sim.grid.dt
    for e, j in (("ex", "jx"), ("ey", "jy"), ("ez", "jz")):
        np.testing.assert_allclose(sim.f[e], -dt * J[j], rtol=1e-15)
    for b in ("bx", "by", "bz"):
        assert np.all(sim.f[b] == 0.0)


def test_div_e_of_a_linear_field_with_unequal_cells(oracle_mod):
    # E = (alpha x, beta y) sampled at the Yee positions has div E = alpha +
    # beta at every node whose stencil does not cross the periodic seam
    wl = _vacuum(12, 10)                          # dx = lambda/16, dy = lambda/10
    sim = oracle_mod.OracleSim(wl, _empty())
    g = sim.grid
    assert g.dx != g.dy
    alpha, beta = 0.37, -1.9
    i = np.arange(wl.nx)[None, :]
    j = np.arange(wl.ny)[:, None]
    sim.f["ex"][...] = alpha * (i + 0.5) * g.dx + 0.0 * j
    sim.f["ey"][...] = beta * (j + 0.5) * g.dy + 0.0 * i
    d = sim.div_e()
    np.testing.assert_allclose(d[1:, 1:], alpha + beta, rtol=1e-12)


# ---------------------------------------------------------------------------
# Eq. (4) moments: the energy window and the weighted spread
# ---------------------------------------------------------------------------
def _energy_particles(k_list, w_list):
    # particles along x with gamma = 1 + k, so (gamma - 1) m c^2 = k m c^2
    n = len(k_list)
    ux = np.array([math.sqrt((1 + k) ** 2 - 1) for k in k_list])
    f32 = np.float32
    return dict(ix=np.full(n, 3, np.int32), iy=np.full(n, 3, np.int32),
                ox=np.full(n, 0.5, f32), oy=np.full(n, 0.5, f32),
                ux=ux.astype(np.float64), uy=np.zeros(n), uz=np.zeros(n),
                sx=np.zeros(n, f32), sy=np.ones(n, f32), sz=np.zeros(n, f32),
                w=np.array(w_list, f32), id=np.arange(n, dtype=np.int32))


def _moments_of(oracle_mod, d, emin=-np.inf, emax=np.inf):
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(0, 1, 0))
    wl = W.Workload(name="m", nx=8, ny=8, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=0.95,
                    steps=1, species=(sp,), pol="none", bc_x="periodic")
    sim = oracle_mod.OracleSim(wl, [d])    # keeps the float64 momenta (gamma = 1 + k to rounding)
    return sim.moments(0, emin, emax)


def test_energy_moments_are_weight_weighted(oracle_mod):
    # kinetic energies 1, 2, 4 (units of m_e c^2) with weights 1, 1, 2:
    # mean (1 + 2 + 8) / 4 = 2.75; variance
    # (1.75^2 + 0.75^2 + 2 * 1.25^2) / 4 = 6.75 / 4 = 1.6875
    mec2 = 0.51099895
    m = _moments_of(oracle_mod, _energy_particles([1.0, 2.0, 4.0], [1.0, 1.0, 2.0]))
    assert m[3] == pytest.approx(4.0)
    assert m[4] == 3
    assert m[5] == pytest.approx(2.75 * mec2, rel=1e-12)
    assert m[6] == pytest.approx(1.6875 * mec2 ** 2, rel=1e-12)


def test_energy_window_is_closed_below_and_open_above(oracle_mod):
    # a particle at rest has kinetic energy exactly 0: it is in [0, 1) and
    # not in [-1, 0)
    d = _energy_particles([0.0, 0.0], [1.0, 3.0])
    assert _moments_of(oracle_mod, d, 0.0, 1.0)[4] == 2
    assert _moments_of(oracle_mod, d, -1.0, 0.0)[4] == 0


# ---------------------------------------------------------------------------
# open x: particles live in [2, nx - 2)
# ---------------------------------------------------------------------------
def test_open_x_removes_particles_leaving_the_plasma_region(oracle_mod):
    # four free particles (no fields) cross or approach the two edges of the
    # plasma region [2, nx - 2); the ones whose new x lies outside it are
    # removed after the step, the others stay
    nx, ny = 16, 8
    wl = _vacuum(nx, ny, bc="open", pol="none")
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    wl = dataclasses.replace(wl, species=(sp,))
    sim0 = oracle_mod.OracleSim(wl, _empty())
    g = sim0.grid
    v = 0.6 * g.dx / g.dt                        # 0.6 cells a step
    ux = v / math.sqrt(1 - v * v)
    x = np.array([2.3, 2.9, nx - 2.3, nx - 2.9])
    u = np.array([-ux, -ux, ux, ux])
    f32 = np.float32
    d = dict(ix=np.floor(x).astype(np.int32), iy=np.full(4, 3, np.int32),
             ox=(x - np.floor(x)).astype(f32), oy=np.full(4, 0.5, f32),
             ux=u.astype(f32), uy=np.zeros(4, f32), uz=np.zeros(4, f32),
             sx=np.ones(4, f32), sy=np.zeros(4, f32), sz=np.zeros(4, f32),
             w=np.full(4, 0.01, f32), id=np.arange(4, dtype=np.int32))
    sim = oracle_mod.OracleSim(wl, [d])
    sim.step(1)
    # new x: 1.7 (out), 2.3 (in), nx - 1.7 (out), nx - 2.3 (in)
    np.testing.assert_array_equal(sim.p[0]["alive"], [0, 1, 0, 1])


# ---------------------------------------------------------------------------
# laser source: centred on the box axis, staggered like E, phase at the peak
# ---------------------------------------------------------------------------
def test_laser_source_is_centred_and_staggered(oracle_mod):
    # CP beam of waist 4 cells: after a few steps E_z (nodes, y = j dy) is
    # mirror symmetric about the node j = ny/2 on the box axis, E_y (y =
    # (j + 1/2) dy) about the half node between j = ny/2 - 1 and ny/2
    nx, ny = 24, 32
    wl = _vacuum(nx, ny, bc="open", pol="cp", a0=1.0, waist_lambda=0.4, fwhm_periods=2.0,
                 t_peak_periods=0.5)
    sim = oracle_mod.OracleSim(wl, _empty())
    sim.step(12)
    ez, ey = sim.f["ez"][:, 3], sim.f["ey"][:, 3]
    jz = (ny - np.arange(ny)) % ny                # node mirror about j = ny/2
    jy = ny - 1 - np.arange(ny)                   # half-node mirror
    assert np.abs(ez).max() > 0.05 and np.abs(ey).max() > 0.05
    np.testing.assert_allclose(ez[jz], ez, atol=1e-12 * np.abs(ez).max())
    np.testing.assert_allclose(ey[jy], ey, atol=1e-12 * np.abs(ey).max())


def test_laser_carrier_phase_is_zero_at_the_envelope_peak(oracle_mod):
    # the LP source sin(t - t_peak) a0 envelope(t) profile(y): zero at the
    # envelope peak and a0 a quarter period later on the axis (envelope
    # 1/e time tau = FWHM / sqrt(2 ln 2)); t_peak of 1.25 periods is not a
    # whole number of periods, so a phase counted from t = 0 would differ
    wl = _vacuum(16, 8, bc="open", pol="lp-y", a0=2.0, waist_lambda=1e6, fwhm_periods=4.0,
                 t_peak_periods=1.25)
    sim = oracle_mod.OracleSim(wl, _empty())
    tp = 1.25 * 2 * math.pi
    tau = 4.0 * 2 * math.pi / math.sqrt(2 * math.log(2))
    yc = 0.5 * wl.ny * sim.grid.dy
    assert abs(sim.laser(tp, yc, 0)) < 1e-12
    q = tp + 0.5 * math.pi
    assert sim.laser(q, yc, 0) == pytest.approx(2.0 * math.exp(-((0.5 * math.pi) / tau) ** 2), rel=1e-9)
    assert sim.laser(q, yc, 1) == 0.0


def test_laser_waist_is_the_field_1_over_e_radius(oracle_mod):
    # the LP source at a quarter period after the envelope peak: on the axis
    # a0 times the envelope; w0 = waist off axis e^-1 times that (the waist
    # is the 1/e radius of the field, in wavelengths: lambda = 2 pi c/omega0)
    waist = 0.4
    wl = _vacuum(16, 8, bc="open", pol="lp-y", a0=1.0, waist_lambda=waist, fwhm_periods=4.0,
                 t_peak_periods=1.0)
    sim = oracle_mod.OracleSim(wl, _empty())
    t = 2 * math.pi + 0.5 * math.pi
    yc = 0.5 * wl.ny * sim.grid.dy
    w0 = waist * 2 * math.pi
    assert sim.laser(t, yc + w0, 0) / sim.laser(t, yc, 0) == pytest.approx(math.exp(-1.0), rel=1e-12)
    assert sim.laser(t, yc - 0.5 * w0, 0) / sim.laser(t, yc, 0) == pytest.approx(math.exp(-0.25), rel=1e-12)


def test_cp_components_are_a_quarter_period_apart(oracle_mod):
    # CP (a0/sqrt 2 in each of Ey and Ez): on the axis of a wide beam, at the
    # envelope peak the Ey source is 0 and the Ez source a0/sqrt 2; a quarter
    # period later (envelope e^-((pi/2)/tau)^2) the roles swap
    wl = _vacuum(16, 8, bc="open", pol="cp", a0=2.0, waist_lambda=1e6, fwhm_periods=4.0,
                 t_peak_periods=1.0)
    sim = oracle_mod.OracleSim(wl, _empty())
    tp = 2 * math.pi
    tau = 4.0 * 2 * math.pi / math.sqrt(2 * math.log(2))
    yc = 0.5 * wl.ny * sim.grid.dy
    amp = 2.0 / math.sqrt(2.0)
    assert abs(sim.laser(tp, yc, 0)) < 1e-12
    assert sim.laser(tp, yc, 1) == pytest.approx(amp, rel=1e-12)
    q = tp + 0.5 * math.pi
    env = math.exp(-((0.5 * math.pi) / tau) ** 2)
    assert sim.laser(q, yc, 0) == pytest.approx(amp * env, rel=1e-12)
    assert abs(sim.laser(q, yc, 1)) < 1e-12


def test_gather_of_uniform_fields_everywhere(oracle_mod):
    # the CIC weights of every staggered component sum to one at any position,
    # within half a cell of the periodic seams too: uniform fields are
    # gathered exactly
    vals = {"ex": 0.3, "ey": -1.1, "ez": 0.7, "bx": 2.0, "by": -0.4, "bz": 1.3}
    sim = _one_particle_sim(oracle_mod, vals, nx=8, ny=8)
    rng = np.random.default_rng(9)
    pts = [(0.1, 0.2), (0.45, 7.9), (7.95, 0.05), (3.3, 0.4)] + [tuple(v) for v in rng.uniform(0, 8, (20, 2))]
    import ctypes as C
    for X, Y in pts:
        E, B = (C.c_double * 3)(), (C.c_double * 3)()
        oracle_mod.lib().or_gather(C.byref(sim.grid), C.byref(sim._fields()), X, Y, E, B)
        np.testing.assert_allclose(list(E), [vals["ex"], vals["ey"], vals["ez"]], rtol=1e-14)
        np.testing.assert_allclose(list(B), [vals["bx"], vals["by"], vals["bz"]], rtol=1e-14)


def test_div_b_of_a_linear_field_with_unequal_cells(oracle_mod):
    # B = (alpha x, beta y) at the Yee positions of Bx (i, j+1/2) and By
    # (i+1/2, j): div B on the cell centres is alpha + beta wherever the
    # stencil does not cross the periodic seam
    wl = _vacuum(12, 10)
    sim = oracle_mod.OracleSim(wl, _empty())
    g = sim.grid
    assert g.dx != g.dy
    alpha, beta = -0.8, 1.7
    i = np.arange(wl.nx)[None, :]
    j = np.arange(wl.ny)[:, None]
    sim.f["bx"][...] = alpha * i * g.dx + 0.0 * j
    sim.f["by"][...] = beta * j * g.dy + 0.0 * i
    d = sim.div_b()
    np.testing.assert_allclose(d[:-1, :-1], alpha + beta, rtol=1e-12)


def test_histogram_keeps_a_particle_just_below_emax_in_the_last_bin(oracle_mod):
    # a particle one ulp below emax is inside [emin, emax); with log bins its
    # bin coordinate log(e/emin)/log(emax/emin) rounds to exactly 1.0, one bin
    # past the last, and must still be counted in the last bin
    sp = W.Species("e", q=-1.0, m=1.0, a=0.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    wl = W.Workload(name="h", nx=8, ny=8, dx_lambda=1 / 16, dy_lambda=1 / 16, cfl=0.95,
                    steps=1, species=(sp,), pol="none", bc_x="periodic")
    f32 = np.float32
    d = dict(ix=np.array([3], np.int32), iy=np.array([3], np.int32), ox=np.array([0.5], f32),
             oy=np.array([0.5], f32), ux=np.array([3.0], f32), uy=np.zeros(1, f32), uz=np.zeros(1, f32),
             sx=np.zeros(1, f32), sy=np.ones(1, f32), sz=np.zeros(1, f32), w=np.ones(1, f32),
             id=np.zeros(1, np.int32))
    sim = oracle_mod.OracleSim(wl, [d])
    ek = sim.moments(0)[5]                      # the particle's kinetic energy (weight 1)
    emax = float(np.nextafter(ek, np.inf))
    emin, nbins = ek / 100.0, 8
    # the case is the one the clamp exists for: the bin coordinate rounds to 1
    assert math.floor(math.log(ek / emin) / math.log(emax / emin) * nbins) == nbins
    assert sim.moments(0, emin, emax)[4] == 1
    h = sim.histogram(0, emin, emax, nbins, True)
    assert h[:, 0].sum() == 1 and h[-1, 0] == 1 and h[-1, 3] == 1.0


def test_split_calls_equal_the_whole_step(oracle_mod):
    # push + deposit of every species and then the field update, called one
    # by one, is the whole step (whose laser injection is pinned above): the
    # same state bit for bit after several steps with the laser entering
    wl = W.small_case(nx=24, ny=12, ppc=2, u_th=0.3, two_species=True)
    parts = W.generate_particles(wl)
    a, b = oracle_mod.OracleSim(wl, parts, step=3), oracle_mod.OracleSim(wl, parts, step=3)
    a.step(4)
    for _ in range(4):
        b.zero_current()
        saved = [b.push(s) for s in range(len(b.p))]
        for s, old in enumerate(saved):
            b.deposit(s, *old)
        b.field_update()
    assert a.step_index == b.step_index == 7
    assert np.abs(a.f["ey"]).max() > 0
    for k in a.f:
        assert np.array_equal(a.f[k], b.f[k]), k
    for s in range(2):
        for k in a.p[s]:
            assert np.array_equal(a.p[s][k], b.p[s][k]), (s, k)


@pytest.mark.parametrize("u0", [0.3, 4.0])
def test_boris_gyro_radius(oracle_mod, u0):
    # pure B_z: the orbit is a circle of radius u_perp / (|q/m| B) (gyration
    # frequency |q/m| B / gamma, speed u / gamma), here to O((omega dt)^2)
    qm, B0 = -1.0, 0.8
    gam = math.sqrt(1 + u0 * u0)
    omega = abs(qm) * B0 / gam
    dt = 0.1 / omega
    u = np.array([u0, 0.0, 0.0])
    x = np.zeros(2)
    xs = []
    for _ in range(int(2 * math.pi / (omega * dt)) + 2):
        u = oracle_mod.boris(qm, dt, (0, 0, 0), (0, 0, B0), u)
        x += dt * u[:2] / gam
        xs.append(x.copy())
    xs = np.array(xs)
    r = 0.25 * (xs[:, 0].max() - xs[:, 0].min() + xs[:, 1].max() - xs[:, 1].min())
    assert r == pytest.approx(u0 / (abs(qm) * B0), rel=(omega * dt) ** 2)


@pytest.mark.parametrize("u0", [0.5, 5.0])
def test_spin_gains_on_the_momentum_at_the_anomaly_rate(oracle_mod, u0):
    # moving across a uniform B_z with the spin along the momentum: the spin
    # turns at (q/m)(a + 1/gamma) B, the momentum at (q/m) B / gamma, so the
    # angle between them grows at |q/m| a B per unit time (the spin tune a
    # gamma per turn) whatever the energy; a = 1 keeps the O((omega dt)^2)
    # terms of the discrete steps small against it
    sp = W.Species("x", q=-1.0, m=1.0, a=1.0, n0=0.01, ppc=1, u_th=0.0, s0=(1, 0, 0))
    B0 = 0.02
    sim = _one_particle_sim(oracle_mod, {"bz": B0}, u=(u0, 0, 0), s=(1, 0, 0), species=sp, nx=64, ny=64)
    dt = sim.grid.dt
    n = 200
    rel = 0.0
    for _ in range(n):
        p = sim.p[0]
        a_u = math.atan2(p["uy"][0], p["ux"][0])
        a_s = math.atan2(p["sy"][0], p["sx"][0])
        sim.push(0)
        p = sim.p[0]
        d_u = math.atan2(p["uy"][0], p["ux"][0]) - a_u
        d_s = math.atan2(p["sy"][0], p["sx"][0]) - a_s
        rel += (d_s - d_u + math.pi) % (2 * math.pi) - math.pi
    # an electron: both turn counter-clockwise about +z, the spin ahead
    assert rel == pytest.approx(n * 1.0 * B0 * dt, rel=1e-3)
