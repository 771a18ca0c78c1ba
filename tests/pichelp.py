"""Shared helpers of the GPU parity tests: build a library context and an
oracle simulation from the same seeded state, and compare them."""
import math

import numpy as np

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W


def make_pair(wl, fields=None, step=0, capacity_factor=1.0, sort_every=0, tile=None, parts=None,
              precision=32, bins=None, window_cells=0):
    parts = W.generate_particles(wl) if parts is None else parts
    cfg = pic.config_from_workload(wl, capacity_factor=capacity_factor, sort_every=sort_every, tile=tile,
                                   precision=precision, bins=bins, window_cells=window_cells)
    sim = pic.Simulation(cfg)
    for s, d in enumerate(parts):
        sim.set_particles(s, d)
    if fields is not None:
        sim.set_fields(fields)
    sim.set_step(step)
    if wl.neutralizing_background:
        sim.capture_background()
    orc = oracle.OracleSim(wl, parts, fields=fields, step=step)
    return sim, orc, parts


def gpu_by_id(sim, s, n_total, f64=False):
    """GPU particles of species s reordered by id; removed ones flagged."""
    g = sim.get_particles_f64(s) if f64 else sim.get_particles(s)
    pos = ("x", "y", "z") if "iz" in g else ("x", "y")
    out = {k: np.full(n_total, np.nan) for k in pos + ("ux", "uy", "uz", "sx", "sy", "sz")}
    alive = np.zeros(n_total, bool)
    ids = g["id"]
    live = g["ix"] >= 0
    assert len(np.unique(ids)) == len(ids), "duplicate particle ids"
    for a in pos:
        out[a][ids[live]] = g["i" + a][live] + g["o" + a][live].astype(np.float64)
    for k in ("ux", "uy", "uz", "sx", "sy", "sz"):
        out[k][ids[live]] = g[k][live]
    alive[ids[live]] = True
    return out, alive


def periodic_diff(a, b, n):
    d = a - b
    return d - n * np.round(d / n)


def compare_particles(sim, orc, s, u_tol=1e-5, s_tol=1e-5, x_tol=1e-5, u_floor=1e-3, f64=False):
    """Per-particle comparison: u relative (floor u_floor), s absolute, x in cells."""
    p = orc.p[s]
    n = len(p["x"])
    g, alive = gpu_by_id(sim, s, n, f64=f64)
    oal = p["alive"].astype(bool)
    assert np.array_equal(alive, oal), f"alive sets differ: {np.sum(alive != oal)} particles"
    if not alive.any():
        return {}
    m = alive
    du = np.sqrt(sum((g[k][m] - p[k][m]) ** 2 for k in ("ux", "uy", "uz")))
    un = np.maximum(np.sqrt(sum(p[k][m] ** 2 for k in ("ux", "uy", "uz"))), u_floor)
    ds = np.sqrt(sum((g[k][m] - p[k][m]) ** 2 for k in ("sx", "sy", "sz")))
    dpos = [np.abs(periodic_diff(g["x"][m], p["x"][m], orc.wl.nx)).max(),
            np.abs(periodic_diff(g["y"][m], p["y"][m], orc.wl.ny)).max()]
    if "z" in p:
        dpos.append(np.abs(periodic_diff(g["z"][m], p["z"][m], orc.wl.nz)).max())
    err = dict(u=float((du / un).max()), s=float(ds.max()), x=float(max(dpos)))
    assert err["u"] <= u_tol, err
    assert err["s"] <= s_tol, err
    assert err["x"] <= x_tol, err
    return err


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def rel_max(a, b, scale=None):
    """Largest element-wise difference relative to the largest reference
    magnitude (or `scale`): a wrong value in a single cell (a tile seam, a
    ghost column, a node wrapped at a periodic edge) shows here even where the
    L2 norm hides it."""
    mb = (float(np.abs(b).max()) if b.size else 0.0) if scale is None else scale
    d = float(np.abs(a - b).max()) if b.size else 0.0
    return d / mb if mb > 0 else d


# library read-back names of the left boundary values and the oracle's
ORACLE_KEY = {"by_left": "byL", "bz_left": "bzL"}
# E, B and J are vectors: a component's error is measured against the
# magnitude of its vector.  With float32 cell offsets every displacement is
# quantised at about 6e-8 cells, so a component that stays small next to the
# others (Jz and Ex under a y-polarised laser in a cold plasma) carries a
# large error relative to its own size but not relative to the vector's.
VECTOR = {k: ("ex", "ey", "ez") for k in ("ex", "ey", "ez")}
VECTOR.update({k: ("bx", "by", "bz") for k in ("bx", "by", "bz", "by_left", "bz_left")})
VECTOR.update({k: ("jx", "jy", "jz") for k in ("jx", "jy", "jz")})


def compare_fields(sim, orc, keys, tol, region=None, f64=False, max_tol=None):
    """Mesh comparison, element by element and in norm, each component
    against its vector's magnitude: max |a - b| <= max_tol * max |V| (max_tol
    defaults to tol) and ||a - b||_2 <= tol * ||V||_2 / sqrt(3), with V the
    oracle's E, B or J."""
    f = sim.get_fields_f64() if f64 else sim.get_fields()
    max_tol = tol if max_tol is None else max_tol
    errs = {}
    for k in keys:
        a, b = f[k].astype(np.float64), orc.f[ORACLE_KEY.get(k, k)]
        comps = [orc.f[c] for c in VECTOR[k]]
        if region is not None and k not in ORACLE_KEY:
            a, b = a[region], b[region]
            comps = [c[region] for c in comps]
        vmax = max(float(np.abs(c).max()) for c in comps)
        vnorm = math.sqrt(sum(float(np.sum(c * c)) for c in comps) / 3.0)
        d2 = float(np.linalg.norm(a - b))
        errs[k] = (d2 / vnorm if vnorm > 0 else d2, rel_max(a, b, vmax))
        assert errs[k][0] <= tol and errs[k][1] <= max_tol, (k, errs)
    return errs


# co-moving window on the stepping path -------------------------------------
def window_schedule(start, steps, n0, dt, dx, speed, ncells):
    """Step indices before which the rule moves the box, one entry per move."""
    out, moved = [], 0
    for n in range(n0, n0 + steps):
        while n >= start and moved + ncells <= math.floor((n - start) * dt * speed / dx):
            out.append(n)
            moved += ncells
    return out


def window_plasmas(wl, ncells, count, ids, seed0=300):
    """count plasmas of the uncovered columns; the ids continue each species'."""
    out = []
    for k in range(count):
        inj = W.injection_particles(wl, ncells, seed=seed0 + k, id_base=ids[0])
        if len(wl.species) > 1:
            inj2 = W.injection_particles(wl, ncells, seed=seed0 + k, id_base=ids[1])
            inj = [inj[0], inj2[1]]
        for s in range(len(ids)):
            ids[s] += len(inj[s]["ix"])
        out.append(inj)
    return out


def window_oracle_run(orc, steps, start, dt, dx, speed, ncells, slabs):
    """steps oracle steps with the co-moving window's rule: before the step
    from index n, while n >= start and moved + ncells <= floor((n - start) dt
    speed / dx), one orc.shift_window(ncells, next plasma or None).  Returns
    the cells moved."""
    moved, k = 0, 0
    for _ in range(steps):
        n = orc.step_index
        while n >= start and moved + ncells <= math.floor((n - start) * dt * speed / dx):
            orc.shift_window(ncells, slabs[k] if k < len(slabs) else None)
            k += 1
            moved += ncells
        orc.step(1)
    return moved
