"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that
the pins catch every one of them: test_oracle_pins.py for the 2D3V source,
test_oracle3_pins.py for the 3D3V source, and for the Python layer (the
units derived from a workload, the beam loss, the co-moving window) the pins
file of each."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
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
    # the position advance, the deposit's v_z, Ampere's J, div E, the moments'
    # weights and window, the open-x removal and the laser source's placement
    ("advance uses old momentum", "double X1 = p->x[i] + g->dt * u[0] / gam / g->dx;",
     "double X1 = p->x[i] + g->dt * u0[0] / gam / g->dx;"),
    ("vz from old momentum", "vz[i] = u[2] / gam;", "vz[i] = u0[2] / gam;"),
    ("Jy half term dropped", "acc += dSy[l] * (S0x[k] + 0.5 * dSx[k]);", "acc += dSy[l] * S0x[k];"),
    ("Jz drops vz", "+= qw * vz * wz;", "+= qw * wz;"),
    ("Jy on the next half node", "f->jy[yj(g, j0 + l) * g->nx + xi(g, i0 + k)] += cy * acc;",
     "f->jy[yj(g, j0 + l + 1) * g->nx + xi(g, i0 + k)] += cy * acc;"),
    ("Ez ignores Jz", "(f->bx[c] - f->bx[jm * nx + i]) / g->dy - f->jz[c]);",
     "(f->bx[c] - f->bx[jm * nx + i]) / g->dy);"),
    ("By half-step sign", "f->by[c] += h / g->dx * (f->ez[j * nx + ip] - f->ez[c]);",
     "f->by[c] -= h / g->dx * (f->ez[j * nx + ip] - f->ez[c]);"),
    ("boris drops first half kick", "um[k] = u[k] + 0.5 * qm * dt * E[k];", "um[k] = u[k];"),
    ("spin angle halved", "double th = om * dt;", "double th = 0.5 * om * dt;"),
    ("omega at the new momentum",
     "double ubar[3] = {0.5 * (u0[0] + u[0]), 0.5 * (u0[1] + u[1]), 0.5 * (u0[2] + u[2])};",
     "double ubar[3] = {u[0], u[1], u[2]};"),
    ("gather stagger of Ey", "E[1] = interp(g, f->ey, X, Y, 0.0, 0.5);", "E[1] = interp(g, f->ey, X, Y, 0.5, 0.0);"),
    ("gather stagger of Bx", "B[0] = interp(g, f->bx, X, Y, 0.0, 0.5);", "B[0] = interp(g, f->bx, X, Y, 0.5, 0.0);"),
    ("gather stagger of By", "B[1] = interp(g, f->by, X, Y, 0.5, 0.0);", "B[1] = interp(g, f->by, X, Y, 0.0, 0.5);"),
    ("periodic unwrap sign", "        return X1 - n;", "        return X1 + n;"),
    ("rho y shape uses x", "shape1(p->y[i] - (double)(j0 + dj));", "shape1(p->x[i] - (double)(j0 + dj));"),
    ("div E y difference uses dx", "(f->ey[c] - f->ey[jm * nx + i]) / g->dy;",
     "(f->ey[c] - f->ey[jm * nx + i]) / g->dx;"),
    ("energy variance unweighted", "var += p->w[i] * (ek - mean) * (ek - mean);",
     "var += (ek - mean) * (ek - mean);"),
    ("count sums weights", "cnt += 1.0;", "cnt += p->w[i];"),
    ("energy window closed above", "if (ek < emin_mev || ek >= emax_mev)\n            continue;\n        sw",
     "if (ek < emin_mev || ek > emax_mev)\n            continue;\n        sw"),
    ("histogram count weighted", "out[5 * b + 0] += 1.0;", "out[5 * b + 0] += p->w[i];"),
    ("log bins linear", "double f = log_bins ? log(ek / emin_mev) / log(emax_mev / emin_mev)",
     "double f = log_bins ? (ek - emin_mev) / (emax_mev - emin_mev)"),
    ("removal at x_min from x = 1", "if (g->bc_x == OR_BC_OPEN && (p->x[i] < 2.0 ||",
     "if (g->bc_x == OR_BC_OPEN && (p->x[i] < 1.0 ||"),
    ("removal at x_max from nx - 1", "p->x[i] >= (double)(g->nx - 2)))\n            p->alive[i] = 0;",
     "p->x[i] >= (double)(g->nx - 1)))\n            p->alive[i] = 0;"),
    ("laser time at the integer step", "t = ((double)step + 0.5) * dt;", "t = (double)step * dt;"),
    ("laser envelope of the intensity",
     "double env = exp(-((t - g->t_peak) / g->tau) * ((t - g->t_peak) / g->tau));",
     "double env = exp(-0.5 * ((t - g->t_peak) / g->tau) * ((t - g->t_peak) / g->tau));"),
    ("laser centred at y = 0", "double yc = 0.5 * g->ny * g->dy;", "double yc = 0.0;"),
    ("laser phase counted from t = 0", "double ph = t - g->t_peak;", "double ph = t;"),
    ("CP at full amplitude per component", "v = g->a0 / sqrt(2.0) * env * tr", "v = g->a0 * env * tr"),
    ("laser Ez source at the Ey height", "or_laser(g, t, (double)j * g->dy, 1, &fin);",
     "or_laser(g, t, ((double)j + 0.5) * g->dy, 1, &fin);"),
    ("x_max absorber uses Ey one column in",
     "f->bz[cl] = (2.0 * f->ey[cl] - (1.0 - r) * f->bz[cl - 1]) / (1.0 + r);",
     "f->bz[cl] = (2.0 * f->ey[cl - 1] - (1.0 - r) * f->bz[cl - 1]) / (1.0 + r);"),
    ("Bx half step uses dx", "f->bx[c] -= h / g->dy * (f->ez[jp * nx + i] - f->ez[c]);",
     "f->bx[c] -= h / g->dx * (f->ez[jp * nx + i] - f->ez[c]);"),
    ("Ey source at node height", "or_laser(g, t, ((double)j + 0.5) * g->dy, 0, &gin);",
     "or_laser(g, t, (double)j * g->dy, 0, &gin);"),
    ("x_max By transverse term dropped", "f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1] + q * dbxl) / (1.0 + r);",
     "f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1]) / (1.0 + r);"),
    ("CP second component sin", "v = g->a0 / sqrt(2.0) * env * tr * (comp == 0 ? sin(ph) : cos(ph));",
     "v = g->a0 / sqrt(2.0) * env * tr * (comp == 0 ? sin(ph) : sin(ph));"),
    ("interp truncates", "long i0 = (long)floor(xs), j0 = (long)floor(ys);\n    double v = 0.0;",
     "long i0 = (long)xs, j0 = (long)ys;\n    double v = 0.0;"),
    ("Ex ignores Jx", "(f->bz[c] - f->bz[jm * nx + i]) / g->dy - f->jx[c]);",
     "(f->bz[c] - f->bz[jm * nx + i]) / g->dy);"),
    ("Ez By difference sign", "f->ez[c] += dt * ((f->by[c] - by_im) / g->dx -",
     "f->ez[c] += dt * ((by_im - f->by[c]) / g->dx -"),
    ("left boundary uses periodic values", "} else {\n                bz_im = f->bzL[j];\n                by_im = f->byL[j];",
     "} else {\n                bz_im = f->bz[j * nx + nx - 1];\n                by_im = f->byL[j];"),
    ("histogram sx unweighted", "out[5 * b + 2] += p->w[i] * p->sx[i];",
     "out[5 * b + 2] += p->sx[i];"),
    ("moments sz unweighted", "swz += p->w[i] * p->sz[i];",
     "swz += p->sz[i];"),
    ("div B y uses dx", "(f->by[jp * nx + i] - f->by[c]) / g->dy;",
     "(f->by[jp * nx + i] - f->by[c]) / g->dx;"),
    ("rho uses charge only", "rho[yj(g, j0 + dj) * g->nx + xi(g, i0 + di)] += sp->q * p->w[i] * wgt;",
     "rho[yj(g, j0 + dj) * g->nx + xi(g, i0 + di)] += sp->q * wgt;"),
    ("removal ignores the deposit", "or_deposit_one(g, f, sp->q * p->w[i], x_old[i], y_old[i], X1, Y1, vz[i]);\n        if (g->bc_x",
     "if (g->bc_x == OR_BC_OPEN && (p->x[i] < 2.0 || p->x[i] >= (double)(g->nx - 2))) { p->alive[i] = 0; continue; }\n        or_deposit_one(g, f, sp->q * p->w[i], x_old[i], y_old[i], X1, Y1, vz[i]);\n        if (g->bc_x"),
    ("Ey curl uses Bz at i+1", "f->ey[c] += dt * (-(f->bz[c] - bz_im) / g->dx - f->jy[c]);",
     "f->ey[c] += dt * (-(f->bz[j * nx + xi(g, i + 1)] - f->bz[c]) / g->dx - f->jy[c]);"),
    ("Bz half step y term sign", "h / g->dy * (f->ex[jp * nx + i] - f->ex[c]);\n            }",
     "h / g->dy * (f->ex[c] - f->ex[jp * nx + i]);\n            }"),
    ("mean energy unweighted", "swe += p->w[i] * ek;",
     "swe += ek;"),
    ("histogram top bin clamp dropped", "if (b >= nbins)\n            b = nbins - 1;",
     "if (b > nbins)\n            b = nbins - 1;"),
    ("moments P x from sy", "swx += p->w[i] * p->sx[i];",
     "swx += p->w[i] * p->sy[i];"),
    ("Jx stencil row offset", "f->jx[yj(g, j0 + l) * g->nx + xi(g, i0 + k)] += cx * acc;",
     "f->jx[yj(g, j0 + l) * g->nx + xi(g, i0 + k + 1)] += cx * acc;"),
    ("Wz first-order term", "0.5 * dSx[k] * S0y[l] +",
     "dSx[k] * S0y[l] +"),
    ("spin rotation cos/sin swapped", "s[k] = s[k] * c + nxs[k] * sn + n[k] * ns * (1.0 - c);",
     "s[k] = s[k] * sn + nxs[k] * c + n[k] * ns * (1.0 - sn);"),
    ("omega E term sign", "Om[k] = qm * (omB * B[k] - omv * vB * v[k] - omE * vxE[k]);",
     "Om[k] = qm * (omB * B[k] - omv * vB * v[k] + omE * vxE[k]);"),
    ("boris t uses gamma of u0", "double gm = sqrt(1.0 + dot3(um, um));",
     "double gm = sqrt(1.0 + dot3(u, u));"),
    ("periodic x wrap missing", "if (g->bc_x == OR_BC_PERIODIC)\n            X1 = wrap_pos(X1, (double)g->nx);\n        Y1",
     "if (0)\n            X1 = wrap_pos(X1, (double)g->nx);\n        Y1"),
    ("div E x uses the wrong neighbour", "div[c] = (f->ex[c] - f->ex[j * nx + im]) / g->dx +",
     "div[c] = (f->ex[j * nx + xi(g, i + 1)] - f->ex[c]) / g->dx +"),
    ("stencil origin off by one", "long i0 = (long)floor(X0) - 1, j0 = (long)floor(Y0) - 1;",
     "long i0 = (long)floor(X0) - 1, j0 = (long)floor(Y0);"),
    ("Wz first term from S1", "double wz = S0x[k] * S0y[l] + 0.5 * dSx[k] * S0y[l] +",
     "double wz = S1x[k] * S1y[l] + 0.5 * dSx[k] * S0y[l] +"),
    ("Wx uses dSy fully", "acc += dSx[k] * (S0y[l] + 0.5 * dSy[l]);",
     "acc += dSx[k] * (S0y[l] + dSy[l]);"),
    ("rotation n.s term sign", "s[k] = s[k] * c + nxs[k] * sn + n[k] * ns * (1.0 - c);",
     "s[k] = s[k] * c + nxs[k] * sn - n[k] * ns * (1.0 - c);"),
    ("boris s without t2", "s[k] = 2.0 * t[k] / (1.0 + t2);",
     "s[k] = 2.0 * t[k];"),
    ("boris up uses s", "cross3(um, t, c);\n    for (int k = 0; k < 3; ++k)\n        up[k] = um[k] + c[k];",
     "cross3(um, s, c);\n    for (int k = 0; k < 3; ++k)\n        up[k] = um[k] + c[k];"),
    ("omega v from u not gamma", "double v[3] = {ubar[0] / gam, ubar[1] / gam, ubar[2] / gam};",
     "double v[3] = {ubar[0], ubar[1], ubar[2]};"),
    ("interp sy ignored", "double xs = X - sx, ys = Y - sy;",
     "double xs = X - sx, ys = Y;"),
    ("shape wider", "return a < 1.0 ? 1.0 - a : 0.0;\n}\n\nstatic double dot3",
     "return a < 1.0 ? 1.0 - 0.5 * a : 0.0;\n}\n\nstatic double dot3"),
    ("E step uses half dt", "    double dt = g->dt;\n    b_half(g, f, 0.5 * dt);",
     "    double dt = 0.5 * g->dt;\n    b_half(g, f, dt);"),
    ("second B half skipped", "    b_half(g, f, 0.5 * dt);\n}\n\nvoid or_step",
     "}\n\nvoid or_step"),
]


# the same for the 3D3V source, pic_oracle3.c
MUTATIONS3 = [
    ("3d Bx z-curl sign", "f->bx[c] -= h * ((f->ez[cjp] - f->ez[c]) / g->dy - (f->ey[ckp] - f->ey[c]) / g->dz);",
     "f->bx[c] -= h * ((f->ez[cjp] - f->ez[c]) / g->dy + (f->ey[ckp] - f->ey[c]) / g->dz);"),
    ("3d By uses dy for z", "f->by[c] -= h * ((f->ex[ckp] - f->ex[c]) / g->dz",
     "f->by[c] -= h * ((f->ex[ckp] - f->ex[c]) / g->dy"),
    ("3d Ex z-difference reversed", "- (f->by[c] - f->by[ckm]) / g->dz - f->jx[c]);",
     "- (f->by[ckm] - f->by[c]) / g->dz - f->jx[c]);"),
    ("3d Ez ignores Jz", "(f->bx[c] - f->bx[cjm]) / g->dy - f->jz[c]);", "(f->bx[c] - f->bx[cjm]) / g->dy);"),
    ("3d left Bz transverse sign", "- (1.0 - r) * f->bz[c0] - qz * dzb0) / (1.0 + r);",
     "- (1.0 - r) * f->bz[c0] + qz * dzb0) / (1.0 + r);"),
    ("3d right Bz without transverse term", "- (1.0 - r) * f->bz[cl - 1] + qz * dzbl) / (1.0 + r);",
     "- (1.0 - r) * f->bz[cl - 1]) / (1.0 + r);"),
    ("3d Jz scale uses dy", "cz = -qw * g->dz / g->dt;", "cz = -qw * g->dy / g->dt;"),
    ("3d Wz third-order term", "dSx[i] * dSy[j] / 3.0;", "dSx[i] * dSy[j] / 2.0;"),
    ("3d Wx mixed term", "0.5 * S0y[j] * dSz[k] +", "0.5 * S0y[j] * S0z[k] +"),
    ("3d gather stagger of Ez", "E[2] = interp3(g, f->ez, X, Y, Z, 0.0, 0.0, 0.5);",
     "E[2] = interp3(g, f->ez, X, Y, Z, 0.0, 0.0, 0.0);"),
    ("3d gather stagger of Bx", "B[0] = interp3(g, f->bx, X, Y, Z, 0.0, 0.5, 0.5);",
     "B[0] = interp3(g, f->bx, X, Y, Z, 0.0, 0.5, 0.0);"),
    ("3d z weight of the gather", "shape1_3(zs - (double)k);", "shape1_3(zs - (double)k0);"),
    ("3d z advance uses dy", "double Z1 = p->z[i] + g->dt * u[2] / gam / g->dz;",
     "double Z1 = p->z[i] + g->dt * u[2] / gam / g->dy;"),
    ("3d laser axis off centre in z", "zc = 0.5 * g->nz * g->dz;", "zc = 0.0;"),
    ("3d laser Ey source at the Ez height", "or3_laser(g, t, ((double)j + 0.5) * g->dy, (double)k * g->dz, 0, &gin);",
     "or3_laser(g, t, ((double)j + 0.5) * g->dy, ((double)k + 0.5) * g->dz, 0, &gin);"),
    ("3d div E uses dy for z", "(f->ez[c] - f->ez[at3(g, i, j, k - 1)]) / g->dz;",
     "(f->ez[c] - f->ez[at3(g, i, j, k - 1)]) / g->dy;"),
    ("3d rho z weight", "shape1_3(p->z[n] - (double)(k0 + c));", "shape1_3(p->z[n] - (double)(k0));"),
    ("3d z advance uses old momentum", "double Z1 = p->z[i] + g->dt * u[2] / gam / g->dz;",
     "double Z1 = p->z[i] + g->dt * u0[2] / gam / g->dz;"),
    ("3d Wy drops the dSz half term", "0.5 * S0x[i] * dSz[k] +\n                        dSx[i] * dSz[k] / 3.0;",
     "dSx[i] * dSz[k] / 3.0;"),
    ("3d Jz scaled by dy", "f->jz[at3(g, i0 + i, j0 + j, k0 + k)] += cz * acc;",
     "f->jz[at3(g, i0 + i, j0 + j, k0 + k)] += cy * acc;"),
    ("3d laser radius without z",
     "double r2 = ((y - yc) * (y - yc) + (z - zc) * (z - zc)) / (g->w0 * g->w0);",
     "double r2 = ((y - yc) * (y - yc)) / (g->w0 * g->w0);"),
    ("3d Ey z-curl sign", "f->ey[c] += dt * ((f->bx[c] - f->bx[ckm]) / g->dz",
     "f->ey[c] += dt * (-(f->bx[c] - f->bx[ckm]) / g->dz"),
    ("3d Bz y-curl uses Ey", "- (f->ex[cjp] - f->ex[c]) / g->dy);\n                }",
     "- (f->ey[cjp] - f->ey[c]) / g->dy);\n                }"),
    ("3d z wrap one cell short", "p->z[i] = wrap_pos3(Z1, (double)g->nz);",
     "p->z[i] = wrap_pos3(Z1, (double)(g->nz - 1));"),
    ("3d gather stagger of By", "B[1] = interp3(g, f->by, X, Y, Z, 0.5, 0.0, 0.5);",
     "B[1] = interp3(g, f->by, X, Y, Z, 0.5, 0.0, 0.0);"),
    ("3d gather stagger of Ey", "E[1] = interp3(g, f->ey, X, Y, Z, 0.0, 0.5, 0.0);",
     "E[1] = interp3(g, f->ey, X, Y, Z, 0.0, 0.5, 0.5);"),
    ("3d x_max By without transverse term",
     "f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1] + qy * dybl) / (1.0 + r);",
     "f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1]) / (1.0 + r);"),
    ("3d div B z difference uses dy", "(f->bz[at3(g, i, j, k + 1)] - f->bz[c]) / g->dz;",
     "(f->bz[at3(g, i, j, k + 1)] - f->bz[c]) / g->dy;"),
    ("3d removal at x_min from x = 1", "if (g->bc_x == OR_BC_OPEN && (p->x[i] < 2.0 ||",
     "if (g->bc_x == OR_BC_OPEN && (p->x[i] < 1.0 ||"),
    ("3d Jx on next node", "f->jx[at3(g, i0 + i, j0 + j, k0 + k)] += cx * acc;",
     "f->jx[at3(g, i0 + i + 1, j0 + j, k0 + k)] += cx * acc;"),
    ("3d Ez source z height", "or3_laser(g, t, (double)j * g->dy, ((double)k + 0.5) * g->dz, 1, &fin);",
     "or3_laser(g, t, (double)j * g->dy, (double)k * g->dz, 1, &fin);"),
    ("3d left By source sign", "f->byL[b] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - qy * dyb0 - 4.0 * fin) / (1.0 + r);",
     "f->byL[b] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - qy * dyb0 + 4.0 * fin) / (1.0 + r);"),
    ("3d left Bz source factor", "f->bzL[b] = (4.0 * gin - 2.0 * f->ey[c0]",
     "f->bzL[b] = (2.0 * gin - 2.0 * f->ey[c0]"),
    ("3d Ex ignores Jx", "- (f->by[c] - f->by[ckm]) / g->dz - f->jx[c]);",
     "- (f->by[c] - f->by[ckm]) / g->dz);"),
    ("3d Ey z difference uses dx", "f->ey[c] += dt * ((f->bx[c] - f->bx[ckm]) / g->dz",
     "f->ey[c] += dt * ((f->bx[c] - f->bx[ckm]) / g->dx"),
    ("3d gather y weight uses x", "double w = shape1_3(xs - (double)i) * shape1_3(ys - (double)j) *",
     "double w = shape1_3(xs - (double)i) * shape1_3(xs - (double)j) *"),
    ("3d rho y weight", "shape1_3(p->y[n] - (double)(j0 + b)) *",
     "shape1_3(p->y[n] - (double)(j0)) *"),
    ("3d div E x uses dy", "div[c] = (f->ex[c] - f->ex[at3(g, i - 1, j, k)]) / g->dx +",
     "div[c] = (f->ex[c] - f->ex[at3(g, i - 1, j, k)]) / g->dy +"),
    ("3d Bx y curl uses Ey", "f->bx[c] -= h * ((f->ez[cjp] - f->ez[c]) / g->dy",
     "f->bx[c] -= h * ((f->ey[cjp] - f->ez[c]) / g->dy"),
    ("3d deposit z not unwrapped", "double Z1 = unwrap3(p->z[i], z_old[i], (double)g->nz);",
     "double Z1 = p->z[i];"),
    ("3d left dzBx sign", "double dzb0 = f->bx[c0] - f->bx[at3(g, 0, j, k - 1)];",
     "double dzb0 = f->bx[at3(g, 0, j, k - 1)] - f->bx[c0];"),
    ("3d right dyBx from the first column", "double dybl = f->bx[cl] - f->bx[at3(g, nx - 1, j - 1, k)];",
     "double dybl = f->bx[cl] - f->bx[at3(g, 0, j - 1, k)];"),
    ("3d By x curl sign", "- (f->ez[cip] - f->ez[c]) / g->dx);",
     "+ (f->ez[cip] - f->ez[c]) / g->dx);"),
    ("3d Ez x difference uses dy", "f->ez[c] += dt * ((f->by[c] - by_im) / g->dx",
     "f->ez[c] += dt * ((f->by[c] - by_im) / g->dy"),
    ("3d Ex y term uses Bx", "f->ex[c] += dt * ((f->bz[c] - f->bz[cjm]) / g->dy",
     "f->ex[c] += dt * ((f->bx[c] - f->bx[cjm]) / g->dy"),
    ("3d rho x weight", "double w = shape1_3(p->x[n] - (double)(i0 + a)) *",
     "double w = shape1_3(p->x[n] - (double)(i0)) *"),
    ("3d div B y uses dz", "(f->by[at3(g, i, j + 1, k)] - f->by[c]) / g->dy +",
     "(f->by[at3(g, i, j + 1, k)] - f->by[c]) / g->dz +"),
    ("3d laser LP into Ez", "v = comp == 0 ? g->a0 * env * sin(ph) : 0.0;",
     "v = comp == 1 ? g->a0 * env * sin(ph) : 0.0;"),
    ("3d Jy running sum drops Wy", "acc += dSy[j] * xz;",
     "acc += dSy[j] * S0x[i];"),
    ("3d Jz prefix over the wrong axis", "f->jz[at3(g, i0 + i, j0 + j, k0 + k)] += cz * acc;",
     "f->jz[at3(g, i0 + i, j0 + k, k0 + j)] += cz * acc;"),
    ("3d left Bz uses Ey at x=1", "f->bzL[b] = (4.0 * gin - 2.0 * f->ey[c0]",
     "f->bzL[b] = (4.0 * gin - 2.0 * f->ey[c0 + 1]"),
    ("3d gather z weight uses y", "shape1_3(zs - (double)k);",
     "shape1_3(ys - (double)k);"),
    ("3d E update x periodic neighbour", "by_im = f->by[at3(g, nx - 1, j, k)];",
     "by_im = f->by[at3(g, 0, j, k)];"),
    ("3d stencil origin z", "k0 = (long)floor(Z0) - 1;",
     "k0 = (long)floor(Z0);"),
    ("3d Wx yz uses S1 for dSz term", "double yz = S0y[j] * S0z[k] + 0.5 * dSy[j] * S0z[k] + 0.5 * S0y[j] * dSz[k] +",
     "double yz = S0y[j] * S0z[k] + 0.5 * dSy[j] * S0z[k] + 0.5 * S0y[j] * S0z[k] +"),
    ("3d interp sz ignored", "double xs = X - sx, ys = Y - sy, zs = Z - sz;",
     "double xs = X - sx, ys = Y - sy, zs = Z;"),
    ("3d E step uses dt/2", "    double dt = g->dt;\n    b_half3(g, f, 0.5 * dt);",
     "    double dt = 0.5 * g->dt;\n    b_half3(g, f, dt);"),
    ("3d Jz accumulates dSy", "acc += dSz[k] * xy;",
     "acc += dSy[k] * xy;"),
]

CASES = ([("pic_oracle.c", "test_oracle_pins.py") + m for m in MUTATIONS] +
         [("pic_oracle3.c", "test_oracle3_pins.py") + m for m in MUTATIONS3])


def _c_caught(src_name, pins, name, old, new):
    """(caught, detail): the pins file run against a copy of the C oracle with
    one planted mistake."""
    import shutil
    with tempfile.TemporaryDirectory() as td:
        srcs = []
        for f in ("pic_oracle.c", "pic_oracle3.c"):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            if f == src_name:
                if text.count(old) < 1:
                    return False, f"mutation anchor not found: {name}"
                text = text.replace(old, new, 1)
            srcs.append(os.path.join(td, f))
            with open(srcs[-1], "w") as fh:
                fh.write(text)
        shutil.copy(os.path.join(ROOT, "oracle", "pic_oracle.h"), td)
        so = os.path.join(td, "liboracle_mut.so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               *srcs, "-o", so, "-lm"])
        env = dict(os.environ, PIC_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", pins)],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        return r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("src_name,pins,name,old,new", CASES, ids=[c[2] for c in CASES])
def test_pins_catch_planted_mistake(outcomes, src_name, pins, name, old, new):
    caught, detail = outcomes[("c", name)]
    assert caught, detail


# planted mistakes in the oracle's Python layer (the co-moving window), caught
# by test_oracle_window_pins.py
MUTATIONS_PY = [
    ("window shifts fields the wrong way", "a[..., :-n] = a[..., n:].copy()", "a[..., n:] = a[..., :-n].copy()"),
    ("window moves particles forward", 'd["x"] -= n', 'd["x"] += n'),
    ("window removal threshold", 'd["alive"][d["x"] < 2.0] = 0', 'd["alive"][d["x"] < 1.0] = 0'),
    ("window background not shifted", "self.rho_bg[..., :-n] = self.rho_bg[..., n:].copy()", "pass"),
    ("window injects no ions", "self.rho_bg -= self.rho()", "pass"),
    ("window keeps the old columns", "a[..., -n:] = 0.0", "pass"),
]


def _run_py_pins(pins, old=None, new=None):
    """Run one pins file against a copy of the oracle package (sources
    included), optionally with one planted mistake in its Python layer;
    returns the pytest run."""
    with tempfile.TemporaryDirectory() as td:
        pkg = os.path.join(td, "oracle")
        os.makedirs(pkg)
        for f in ("pic_oracle.c", "pic_oracle3.c", "pic_oracle.h"):
            with open(os.path.join(ROOT, "oracle", f)) as src, open(os.path.join(pkg, f), "w") as dst:
                dst.write(src.read())
        text = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
        if old is not None:
            assert text.count(old) >= 1, f"mutation anchor not found: {old}"
            text = text.replace(old, new, 1)
        with open(os.path.join(pkg, "__init__.py"), "w") as fh:
            fh.write(text)
        env = dict(os.environ, PYTHONPATH=td + os.pathsep + ROOT)
        env.pop("PIC_ORACLE_LIB", None)
        return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                               os.path.join(ROOT, "tests", pins)],
                              cwd=td, env=env, capture_output=True, text=True, timeout=600)


def _run_window_pins(old=None, new=None):
    return _run_py_pins("test_oracle_window_pins.py", old, new)


def test_window_pins_pass_on_an_unmodified_copy():
    r = _run_window_pins()
    assert r.returncode == 0, r.stdout[-2000:]


def _py_caught(pins, name, old, new):
    """(caught, detail) for one planted mistake in the Python layer: caught =
    a pin failed (not an error while collecting or building)."""
    r = _run_py_pins(pins, old, new)
    last = r.stdout.splitlines()[-1] if r.stdout.strip() else ""
    return r.returncode == 1 and "failed" in last, f"pins did not catch: {name}\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name,old,new", MUTATIONS_PY, ids=[m[0] for m in MUTATIONS_PY])
def test_window_pins_catch_planted_mistake(outcomes, name, old, new):
    caught, detail = outcomes[("window", name)]
    assert caught, detail


# planted mistakes in the rest of the Python layer: the oracle's units (the
# grid it derives from a workload), the beam loss and more of the window;
# each with the pins file that catches it
MUTATIONS_PY_MORE = [
    ("dx in wavelengths", "test_oracle_pins.py", "dx, dy = wl.dx_lambda * two_pi, wl.dy_lambda * two_pi",
     "dx, dy = wl.dx_lambda, wl.dy_lambda * two_pi"),
    ("dt without the Courant factor", "test_oracle_pins.py",
     "dt = wl.cfl / math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2)\n", "dt = 1.0 / math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2)\n"),
    ("tau from the field FWHM", "test_oracle_pins.py",
     "tau = wl.fwhm_periods * two_pi / math.sqrt(2.0 * math.log(2.0))\n    return Grid(",
     "tau = wl.fwhm_periods * two_pi / (2.0 * math.sqrt(math.log(2.0)))\n    return Grid("),
    ("2d waist in wavelengths", "test_oracle_pins.py",
     "w0=wl.waist_lambda * two_pi, tau=tau, t_peak=wl.t_peak_periods * two_pi)\n\n\ndef derive_grid3",
     "w0=wl.waist_lambda, tau=tau, t_peak=wl.t_peak_periods * two_pi)\n\n\ndef derive_grid3"),
    ("2d t_peak in periods", "test_oracle_pins.py",
     "w0=wl.waist_lambda * two_pi, tau=tau, t_peak=wl.t_peak_periods * two_pi)\n\n\ndef derive_grid3",
     "w0=wl.waist_lambda * two_pi, tau=tau, t_peak=wl.t_peak_periods)\n\n\ndef derive_grid3"),
    ("3d dt without dz", "test_oracle3_pins.py",
     "dt = wl.cfl / math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2 + 1.0 / dz ** 2)",
     "dt = wl.cfl / math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2)"),
    ("3d dz in wavelengths", "test_oracle3_pins.py", "wl.dz_lambda * two_pi\n", "wl.dz_lambda\n"),
    ("3d waist in wavelengths", "test_oracle3_pins.py",
     "w0=wl.waist_lambda * two_pi, tau=tau, t_peak=wl.t_peak_periods * two_pi)\n\n\nclass OracleSim",
     "w0=wl.waist_lambda, tau=tau, t_peak=wl.t_peak_periods * two_pi)\n\n\nclass OracleSim"),
    ("loss sigmoid sign", "test_oracle_loss_pins.py",
     "a = d[\"w\"][live] * e / (1.0 + np.exp(-(e - e_cut_mev) / e_width_mev))",
     "a = d[\"w\"][live] * e / (1.0 + np.exp((e - e_cut_mev) / e_width_mev))"),
    ("loss not energy weighted", "test_oracle_loss_pins.py", "a = d[\"w\"][live] * e / (1.0",
     "a = d[\"w\"][live] / (1.0"),
    ("loss of the total energy", "test_oracle_loss_pins.py",
     "e = (np.sqrt(1.0 + u2) - 1.0) * self.spec[s].m * MEC2_MEV\n        a =",
     "e = np.sqrt(1.0 + u2) * self.spec[s].m * MEC2_MEV\n        a ="),
    ("loss of a fixed spin axis", "test_oracle_loss_pins.py", "spin = d[(\"sx\", \"sy\", \"sz\")[axis]][live]",
     "spin = d[\"sy\"][live]"),
    ("loss counts removed particles", "test_oracle_loss_pins.py", "live = d[\"alive\"] > 0\n        u2",
     "live = d[\"alive\"] >= 0\n        u2"),
    ("loss energy without the mass", "test_oracle_loss_pins.py",
     "e = (np.sqrt(1.0 + u2) - 1.0) * self.spec[s].m * MEC2_MEV\n        a =",
     "e = (np.sqrt(1.0 + u2) - 1.0) * MEC2_MEV\n        a ="),
    ("window boundary values from column n", "test_oracle_window_pins.py",
     "self.f[\"byL\"][...] = self.f[\"by\"][..., n - 1]", "self.f[\"byL\"][...] = self.f[\"by\"][..., n]"),
    ("window keeps the old Bz boundary", "test_oracle_window_pins.py",
     "self.f[\"bzL\"][...] = self.f[\"bz\"][..., n - 1]", "pass"),
    ("window renumbers injected plasma", "test_oracle_window_pins.py",
     "alive=np.ones(len(d[\"ix\"]), np.int32),\n                   id=d[\"id\"].copy())",
     "alive=np.ones(len(d[\"ix\"]), np.int32),\n                   id=np.arange(len(d[\"ix\"]), dtype=np.int32))"),
    ("2d positions drop the offsets", "test_oracle3_pins.py",
     "x=d[\"ix\"].astype(np.float64) + d[\"ox\"].astype(np.float64),\n                y=d[\"iy\"].astype(np.float64) + d[\"oy\"].astype(np.float64),\n                ux",
     "x=d[\"ix\"].astype(np.float64) + d[\"ox\"].astype(np.float64),\n                y=d[\"iy\"].astype(np.float64) + 0.5,\n                ux"),
    ("2d background with the wrong sign", "test_oracle_pins.py",
     "        self.rho_bg = np.zeros((ny, nx))\n        if wl.neutralizing_background:\n            self.rho_bg = -self.rho()",
     "        self.rho_bg = np.zeros((ny, nx))\n        if wl.neutralizing_background:\n            self.rho_bg = self.rho()"),
    ("3d background with the wrong sign", "test_oracle3_pins.py",
     "        self.rho_bg = np.zeros(shape)\n        if wl.neutralizing_background:\n            self.rho_bg = -self.rho()",
     "        self.rho_bg = np.zeros(shape)\n        if wl.neutralizing_background:\n            self.rho_bg = self.rho()"),
    ("2d gauss residual leaves out the background", "test_oracle_pins.py",
     "        r = self.div_e() - self.rho() - self.rho_bg\n        if self.wl.bc_x == \"open\":\n            r = r[:, 3:",
     "        r = self.div_e() - self.rho()\n        if self.wl.bc_x == \"open\":\n            r = r[:, 3:"),
    ("3d z offsets dropped", "test_oracle3_pins.py",
     "z=d[\"iz\"].astype(np.float64) + d[\"oz\"].astype(np.float64),",
     "z=d[\"iz\"].astype(np.float64) + 0.5,"),
    ("3d field update without the step index", "test_oracle3_pins.py",
     "lib().or3_field_update(C.byref(self.grid), C.byref(self._fields()), self.step_index)",
     "lib().or3_field_update(C.byref(self.grid), C.byref(self._fields()), 0)"),
    ("2d step index not advanced", "test_oracle_pins.py",
     "lib().or_field_update(C.byref(self.grid), C.byref(self._fields()), self.step_index)\n        self.step_index += 1",
     "lib().or_field_update(C.byref(self.grid), C.byref(self._fields()), self.step_index)"),
    ("3d immobile species pushed", "test_oracle3_pins.py",
     "        for _ in range(nsteps):\n            parts = (Parts3 * nsp)",
     "        self.mobile[...] = 1\n        for _ in range(nsteps):\n            parts = (Parts3 * nsp)"),
    ("window injected offsets dropped", "test_oracle_window_pins.py",
     "out[a] = d[\"i\" + a].astype(np.float64) + d[\"o\" + a].astype(np.float64)",
     "out[a] = d[\"i\" + a].astype(np.float64)"),
    ("3d histogram log flag ignored", "test_oracle3_pins.py",
     "1 if log_bins else 0, _dp(out))\n        return out.reshape(nbins, 5)\n\n    def laser(self, t, y, z, comp):",
     "0, _dp(out))\n        return out.reshape(nbins, 5)\n\n    def laser(self, t, y, z, comp):"),
]


@pytest.mark.parametrize("pins", sorted({m[1] for m in MUTATIONS_PY_MORE}))
def test_python_layer_pins_pass_on_an_unmodified_copy(pins):
    r = _run_py_pins(pins)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,pins,old,new", MUTATIONS_PY_MORE, ids=[m[0] for m in MUTATIONS_PY_MORE])
def test_python_layer_pins_catch_planted_mistake(outcomes, name, pins, old, new):
    caught, detail = outcomes[("python", name)]
    assert caught, detail


@pytest.fixture(scope="module")
def outcomes():
    """Every planted mistake's pins run, once, on the host cores this process
    may use (at most 16 at a time; each in its own temporary copy of the
    oracle and its own process)."""
    from concurrent.futures import ThreadPoolExecutor
    jobs = {("c", c[2]): (_c_caught, c) for c in CASES}
    jobs.update({("window", m[0]): (_py_caught, ("test_oracle_window_pins.py",) + m) for m in MUTATIONS_PY})
    jobs.update({("python", m[0]): (_py_caught, (m[1], m[0], m[2], m[3])) for m in MUTATIONS_PY_MORE})
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=max(1, min(16, cores))) as ex:
        futs = {k: ex.submit(f, *a) for k, (f, a) in jobs.items()}
        return {k: fut.result() for k, fut in futs.items()}
