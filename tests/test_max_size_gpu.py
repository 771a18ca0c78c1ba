"""GPU parity at the largest meshes the library accepts.

- 3D3V: 2044 x 1028 x 1020 cells. The default 16 x 4 x 4 tiles pad this to
  2,147,450,880 cells (8,388,480 tiles), just below the 2^31 limit of the tile
  sort's cell key. Each mesh component holds 2.1e9 reals, so E and B together
  hold 1.3e10.
- 2D3V: 32767 x 32767 cells (4,194,304 tiles of 32 x 8).

E, B and J are bound to torch tensors (pic_bind_buffers), so small blocks of
them can be set and read on the device. A random field patch and a few
hundred particles sit in the mesh's last tiles, where the mesh, tile and sort
key indices are largest. The patch straddles the periodic y (and z) edge, so
the step wraps there.

One step is compared with the FP64 oracle on a 16-cell periodic box that
holds the same patch and particles. Yee's update and the particle step reach
at most three cells in a step, and the box's 5-cell margins stay zero, so the
two must agree cell by cell. Every other cell of the large mesh must stay
exactly zero; that catches a write at a wrapped index anywhere.
Tolerances as in the one-step parity tests.

Device memory: about 210 GB at the peak of the 3D3V binding (the context's
130 GB plus the bound E, B and J), so unreferenced contexts are collected
and torch's cache is emptied first.
"""
import gc

import numpy as np
import pytest

import oracle
import paper_2002_02211_gb300 as pic
import workloads as W
from pichelp import rel_max

pytestmark = pytest.mark.gpu

M, P = 5, 6          # margin and patch width of the small box (cells)
NS = 2 * M + P       # small box: 16 cells per axis


def _cases(dim):
    """(large workload, small periodic workload, region origin on the large
    mesh per axis (x, y[, z]))."""
    if dim == 3:
        small = W.small_case3(nx=NS, ny=NS, nz=NS, ppc=1, bc_x="periodic", pol="none")
        big = W.scaled(small, nx=2044, ny=1028, nz=1020, bc_x="open")
    else:
        small = W.small_case(nx=NS, ny=NS, ppc=1, bc_x="periodic", pol="none")
        big = W.scaled(small, nx=32767, ny=32767, bc_x="open")
    # x: the region ends 3 cells before the open x_max boundary; y, z: the
    # patch fills the last P rows and the upper margin wraps onto rows 0..M-1
    origin = [big.nx - 3 - NS, big.ny - M - P] + ([big.nz - M - P] if dim == 3 else [])
    return big, small, origin


def _particles(small, rng, per_cell):
    """per_cell particles in every cell of the patch [M, M + P) of the small box."""
    three = small.dim == 3
    axes = 3 if three else 2
    grids = np.meshgrid(*[np.arange(M, M + P, dtype=np.int32)] * axes, indexing="ij")
    cells = [np.repeat(g.ravel(), per_cell) for g in grids]   # z, y, x order in 3D; y, x in 2D
    n = len(cells[0])
    d = dict(ix=cells[-1], iy=cells[-2], ox=rng.random(n, dtype=np.float32), oy=rng.random(n, dtype=np.float32),
             ux=rng.standard_normal(n, dtype=np.float32) * np.float32(0.3),
             uy=rng.standard_normal(n, dtype=np.float32) * np.float32(0.3),
             uz=rng.standard_normal(n, dtype=np.float32) * np.float32(0.3),
             sx=np.zeros(n, np.float32), sy=np.ones(n, np.float32), sz=np.zeros(n, np.float32),
             w=np.full(n, np.float32(0.05), np.float32), id=np.arange(n, dtype=np.int32))
    if three:
        d["iz"] = cells[0]
        d["oz"] = rng.random(n, dtype=np.float32)
    return d


def _region_index(torch, origin, big, dev):
    """Device index tensors of the small box's rows on the large mesh (y and
    z wrapped), and its x range."""
    y = torch.remainder(torch.arange(NS, device=dev) + origin[1], big.ny)
    z = torch.remainder(torch.arange(NS, device=dev) + origin[2], big.nz) if big.dim == 3 else None
    return slice(origin[0], origin[0] + NS), y, z


def _region(t, xs, y, z):
    """[comp][z][y][x] (3D) or [comp][y][x] (2D) block of a bound mesh tensor."""
    if z is not None:
        return t.index_select(1, z).index_select(2, y)[..., xs].double().cpu().numpy()
    return t[:, 0].index_select(1, y)[..., xs].double().cpu().numpy()


def _abs_sum(torch, t):
    """Sum of |t| in FP64, slab by slab (no temporary of the whole tensor)."""
    s = 0.0
    for c in range(t.shape[0]):
        for z0 in range(0, t.shape[1], 64):
            s += float(t[c, z0:z0 + 64].abs().sum(dtype=torch.float64))
    return s


@pytest.mark.parametrize("dim", [3, 2], ids=["3d-2044x1028x1020", "2d-32767x32767"])
def test_largest_mesh_far_corner_step_against_oracle(dim):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    gc.collect()                 # contexts of earlier tests awaiting collection free their memory
    torch.cuda.empty_cache()
    need = 225e9 if dim == 3 else 115e9   # the peaks above, with some room
    free = torch.cuda.mem_get_info()[0]
    if free < need:
        pytest.skip(f"needs about {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    big, small, origin = _cases(dim)
    rng = np.random.default_rng(61 + dim)
    ps = _particles(small, rng, per_cell=2)
    fs = W.random_fields(small, seed=62)
    patch = (slice(M, M + P),) * dim
    for k in fs:                                    # the field patch only; zero margins
        v = np.zeros_like(fs[k])
        v[patch] = fs[k][patch] * np.float32(0.6)
        fs[k] = v
    cfg = pic.config_from_workload(big)
    cfg.sp[0].capacity = 1024
    sim = pic.Simulation(cfg)
    t = {}   # every device tensor of the test, released in `finally` even on failure
    try:
        bound = sim.bind_torch(mesh=True, particles=False)
        t["eb"], t["j"] = bound["eb"], bound["j"]
        bound = None
        dev = t["eb"].device
        xs, t["y"], t["z"] = _region_index(torch, origin, big, dev)
        y, z = t["y"], t["z"]
        # the patch into the bound E, B (rows wrapped like the region's)
        comps = ("ex", "ey", "ez", "bx", "by", "bz")
        block = torch.from_numpy(np.stack([fs[k] for k in comps])).to(dev)
        if dim == 3:
            t["eb"][:, z.view(-1, 1), y.view(1, -1), xs] = block
        else:
            t["eb"][:, 0, y, xs] = block
        del block
        torch.cuda.synchronize()
        # the particles, moved onto the large mesh
        pb = {k: v.copy() for k, v in ps.items()}
        pb["ix"] = (ps["ix"] + origin[0]).astype(np.int32)
        pb["iy"] = ((ps["iy"] + origin[1]) % big.ny).astype(np.int32)
        if dim == 3:
            pb["iz"] = ((ps["iz"] + origin[2]) % big.nz).astype(np.int32)
        sim.set_particles(0, pb)
        orc = oracle.OracleSim(small, [ps], fields=fs)

        sim.push_deposit()
        orc.zero_current()
        old = orc.push(0)
        orc.deposit(0, *old)
        g = sim.get_particles(0)
        assert len(g["id"]) == len(ps["id"]), "no particle may leave"
        o = np.argsort(g["id"])
        p = orc.p[0]
        for a, off, n in zip(("x", "y", "z")[:dim], origin, (big.nx, big.ny, big.nz)[:dim]):
            xg = (g["i" + a][o] - off) % n + g["o" + a][o].astype(np.float64)
            assert np.abs(xg - p[a]).max() <= 1e-5, a
        un = np.maximum(np.sqrt(p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2), 1e-3)
        du = np.sqrt(sum((g[k][o] - p[k]) ** 2 for k in ("ux", "uy", "uz")))
        ds = np.sqrt(sum((g[k][o] - p[k]) ** 2 for k in ("sx", "sy", "sz")))
        assert (du / un).max() <= 1e-5 and ds.max() <= 1e-5
        torch.cuda.synchronize()
        jr = _region(t["j"], xs, y, z)
        jmax = max(np.abs(orc.f[k]).max() for k in ("jx", "jy", "jz"))
        assert jmax > 0
        for c, k in enumerate(("jx", "jy", "jz")):
            assert rel_max(jr[c], orc.f[k], jmax) <= 1e-5, k
        # every current value of the large mesh lies in the region
        assert _abs_sum(torch, t["j"]) == pytest.approx(float(np.abs(jr).sum()), rel=1e-6)

        sim.field_update()
        orc.field_update()
        torch.cuda.synchronize()
        er = _region(t["eb"], xs, y, z)
        for c, k in enumerate(comps):
            vec = comps[:3] if c < 3 else comps[3:]
            vmax = max(np.abs(orc.f[q]).max() for q in vec)
            assert rel_max(er[c], orc.f[k], vmax) <= 1e-5, k
        # nothing outside the region changed, and J was cleared by the E step
        assert _abs_sum(torch, t["eb"]) == pytest.approx(float(np.abs(er).sum()), rel=1e-6)
        assert _abs_sum(torch, t["j"]) == 0.0
    finally:
        sim.close()
        sim._bound = None
        t.clear()
        torch.cuda.empty_cache()
