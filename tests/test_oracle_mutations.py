"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that
the pins in test_oracle_pins.py catch every one of them."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pic_oracle.c")

# (name, exact text in pic_oracle.c, replacement)
MUTATIONS = [
    ("boris drops second half kick", "u[k] = um[k] + c[k] + 0.5 * qm * dt * E[k];", "u[k] = um[k] + c[k];"),
    ("boris rotation factor", "s[k] = 2.0 * t[k] / (1.0 + t2);", "s[k] = t[k] / (1.0 + t2);"),
    ("boris rotation sense", "cross3(up, s, c);", "cross3(s, up, c);"),
    ("boris gamma at the wrong time", "t[k] = 0.5 * qm * dt * B[k] / gm;", "t[k] = 0.5 * qm * dt * B[k];"),
    ("Om_B coefficient", "double omB = a + 1.0 / gam;", "double omB = a + 1.0;"),
    ("Om_v sign", "Om[k] = qm * (omB * B[k] - omv * vB * v[k] - omE * vxE[k]);",
     "Om[k] = qm * (omB * B[k] + omv * vB * v[k] - omE * vxE[k]);"),
    ("Om_v coefficient", "double omv = a * gam / (gam + 1.0);", "double omv = a * gam / (gam - 1.0 + 1e-300);"),
    ("Om_E coefficient", "double omE = a + 1.0 / (1.0 + gam);", "double omE = a + 1.0 / gam;"),
    ("Om_E cross order", "cross3(v, E, vxE);", "cross3(E, v, vxE);"),
    ("spin rotation sense", "double n[3] = {-Om[0] / om, -Om[1] / om, -Om[2] / om};",
     "double n[3] = {Om[0] / om, Om[1] / om, Om[2] / om};"),
    ("rodrigues last term", "s[k] = s[k] * c + nxs[k] * sn + n[k] * ns * (1.0 - c);",
     "s[k] = s[k] * c + nxs[k] * sn;"),
    ("spin uses new momentum", "double ubar[3] = {0.5 * (u0[0] + u[0]), 0.5 * (u0[1] + u[1]), 0.5 * (u0[2] + u[2])};",
     "double ubar[3] = {u0[0], u0[1], u0[2]};"),
    ("gather stagger of Ex", "E[0] = interp(g, f->ex, X, Y, 0.5, 0.0);", "E[0] = interp(g, f->ex, X, Y, 0.0, 0.5);"),
    ("gather stagger of Bz", "B[2] = interp(g, f->bz, X, Y, 0.5, 0.5);", "B[2] = interp(g, f->bz, X, Y, 0.0, 0.0);"),
    ("advance uses dy for x", "double X1 = p->x[i] + g->dt * u[0] / gam / g->dx;",
     "double X1 = p->x[i] + g->dt * u[0] / gam / g->dy;"),
    ("Wx uses S1", "acc += dSx[k] * (S0y[l] + 0.5 * dSy[l]);", "acc += dSx[k] * (S1y[l] + 0.5 * dSy[l]);"),
    ("Jx sign", "double cx = -qw * g->dx / g->dt, cy = -qw * g->dy / g->dt;",
     "double cx = qw * g->dx / g->dt, cy = -qw * g->dy / g->dt;"),
    ("Wz third-order term", "0.5 * S0x[k] * dSy[l] + dSx[k] * dSy[l] / 3.0;", "0.5 * S0x[k] * dSy[l] + dSx[k] * dSy[l] / 2.0;"),
    ("Bz curl sign", "f->bz[c] -= h / g->dx * (f->ey[j * nx + ip] - f->ey[c]) -",
     "f->bz[c] += h / g->dx * (f->ey[j * nx + ip] - f->ey[c]) -"),
    ("Bx index", "f->bx[c] -= h / g->dy * (f->ez[jp * nx + i] - f->ez[c]);",
     "f->bx[c] -= h / g->dy * (f->ez[c] - f->ez[jp * nx + i]);"),
    ("Ex uses dx", "f->ex[c] += dt * ((f->bz[c] - f->bz[jm * nx + i]) / g->dy - f->jx[c]);",
     "f->ex[c] += dt * ((f->bz[c] - f->bz[jm * nx + i]) / g->dx - f->jx[c]);"),
    ("E update ignores J", "f->ey[c] += dt * (-(f->bz[c] - bz_im) / g->dx - f->jy[c]);",
     "f->ey[c] += dt * (-(f->bz[c] - bz_im) / g->dx);"),
    ("laser source sign", "f->bzL[j] = (4.0 * gin - 2.0 * f->ey[c0] - (1.0 - r) * f->bz[c0]) / (1.0 + r);",
     "f->bzL[j] = (-4.0 * gin - 2.0 * f->ey[c0] - (1.0 - r) * f->bz[c0]) / (1.0 + r);"),
    ("CP source sign", "f->byL[j] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - q * dbx0 - 4.0 * fin) / (1.0 + r);",
     "f->byL[j] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - q * dbx0 + 4.0 * fin) / (1.0 + r);"),
    ("absorber at x_max", "f->bz[cl] = (2.0 * f->ey[cl] - (1.0 - r) * f->bz[cl - 1]) / (1.0 + r);",
     "f->bz[cl] = (2.0 * f->ey[cl] + (1.0 - r) * f->bz[cl - 1]) / (1.0 + r);"),
    ("boundary without transverse term",
     "f->byL[j] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - q * dbx0 - 4.0 * fin) / (1.0 + r);",
     "f->byL[j] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - 4.0 * fin) / (1.0 + r);"),
    ("boundary transverse sign at x_max",
     "f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1] + q * dbxl) / (1.0 + r);",
     "f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1] - q * dbxl) / (1.0 + r);"),
    ("histogram bin rounding", "int b = (int)floor(f * nbins);", "int b = (int)floor(f * nbins + 0.5);"),
    ("histogram spin unweighted", "out[5 * b + 3] += p->w[i] * p->sy[i];", "out[5 * b + 3] += p->sy[i];"),
    ("moments unweighted mean", "swy += p->w[i] * p->sy[i];", "swy += p->sy[i];"),
    ("energy uses total energy", "double ek = (sqrt(1.0 + dot3(u, u)) - 1.0) * sp->m * MEC2_MEV;\n        if (ek < emin_mev",
     "double ek = (sqrt(1.0 + dot3(u, u))) * sp->m * MEC2_MEV;\n        if (ek < emin_mev"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutated = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "pic_oracle.c")
        with open(c, "w") as fh:
            fh.write(mutated)
        import shutil
        shutil.copy(os.path.join(ROOT, "oracle", "pic_oracle.h"), td)
        so = os.path.join(td, "liboracle_mut.so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               c, "-o", so, "-lm"])
        env = dict(os.environ, PIC_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
