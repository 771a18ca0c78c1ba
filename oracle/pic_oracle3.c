/*
 * pic_oracle3.c -- plain FP64 CPU oracle of the 3D3V step (test
 * infrastructure only; see pic_oracle.h).  Same methods and readings as the
 * 2D3V oracle in pic_oracle.c, written out for three dimensions: CIC gather
 * on the 3D Yee mesh, the Boris push and Thomas-BMT rotation of Eqs. (1)-(3)
 * (shared with the 2D oracle), the 3D Esirkepov current and the 3D Yee update
 * with the first-order Silver-Mueller boundary at the x ends.
 *
 * Mesh arrays are [nz][ny][nx]; element [k][j][i] of
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
 *   Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
 *   Jx, Jy, Jz as Ex, Ey, Ez.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

static void or3_fail(const char *what)
{
    fprintf(stderr, "pic_oracle3: %s\n", what);
    abort();
}

static long wrap3(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

static long xi3(const or_grid3_t *g, long i)
{
    if (g->bc_x == OR_BC_PERIODIC)
        return wrap3(i, g->nx);
    if (i < 0 || i >= g->nx)
        or3_fail("x node index outside the mesh");
    return i;
}

/* flat index of node (i, j, k) with the periodic y, z wraps and the x rule */
static long at3(const or_grid3_t *g, long i, long j, long k)
{
    return (wrap3(k, g->nz) * g->ny + wrap3(j, g->ny)) * g->nx + xi3(g, i);
}

static double shape1_3(double d)
{
    double a = fabs(d);
    return a < 1.0 ? 1.0 - a : 0.0;
}

/* a1: CIC interpolation of one component sitting at (i + sx, j + sy, k + sz) */
static double interp3(const or_grid3_t *g, const double *F, double X, double Y, double Z,
                      double sx, double sy, double sz)
{
    double xs = X - sx, ys = Y - sy, zs = Z - sz;
    long i0 = (long)floor(xs), j0 = (long)floor(ys), k0 = (long)floor(zs);
    double v = 0.0;
    for (long di = 0; di < 2; ++di)
        for (long dj = 0; dj < 2; ++dj)
            for (long dk = 0; dk < 2; ++dk) {
                long i = i0 + di, j = j0 + dj, k = k0 + dk;
                double w = shape1_3(xs - (double)i) * shape1_3(ys - (double)j) *
                           shape1_3(zs - (double)k);
                v += w * F[at3(g, i, j, k)];
            }
    return v;
}

void or3_gather(const or_grid3_t *g, const or_fields3_t *f, double X, double Y, double Z,
                double E[3], double B[3])
{
    E[0] = interp3(g, f->ex, X, Y, Z, 0.5, 0.0, 0.0);
    E[1] = interp3(g, f->ey, X, Y, Z, 0.0, 0.5, 0.0);
    E[2] = interp3(g, f->ez, X, Y, Z, 0.0, 0.0, 0.5);
    B[0] = interp3(g, f->bx, X, Y, Z, 0.0, 0.5, 0.5);
    B[1] = interp3(g, f->by, X, Y, Z, 0.5, 0.0, 0.5);
    B[2] = interp3(g, f->bz, X, Y, Z, 0.5, 0.5, 0.0);
}

static double wrap_pos3(double X, double n)
{
    double r = X - n * floor(X / n);
    if (r >= n)
        r -= n;
    if (r < 0.0)
        r = 0.0;
    return r;
}

static double unwrap3(double X1, double X0, double n)
{
    if (X1 - X0 > 0.5 * n)
        return X1 - n;
    if (X0 - X1 > 0.5 * n)
        return X1 + n;
    return X1;
}

/* a1-a4 for every live particle of one species (positions in cell units) */
void or3_push(const or_grid3_t *g, const or_species_t *sp, or_particles3_t *p,
              const or_fields3_t *f, double *x_old, double *y_old, double *z_old)
{
    double qm = sp->q / sp->m;
    /* particles are independent here: the OpenMP build splits them over threads */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < p->n; ++i) {
        x_old[i] = p->x[i];
        y_old[i] = p->y[i];
        z_old[i] = p->z[i];
        if (!p->alive[i])
            continue;
        double E[3], B[3];
        or3_gather(g, f, p->x[i], p->y[i], p->z[i], E, B);
        double u0[3] = {p->ux[i], p->uy[i], p->uz[i]};
        double u[3] = {u0[0], u0[1], u0[2]};
        or_boris(qm, g->dt, E, B, u);
        double ubar[3] = {0.5 * (u0[0] + u[0]), 0.5 * (u0[1] + u[1]), 0.5 * (u0[2] + u[2])};
        double Om[3], s[3] = {p->sx[i], p->sy[i], p->sz[i]};
        or_omega(qm, sp->a, ubar, E, B, Om);
        or_spin_rotate(Om, g->dt, s);
        double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double X1 = p->x[i] + g->dt * u[0] / gam / g->dx;
        double Y1 = p->y[i] + g->dt * u[1] / gam / g->dy;
        double Z1 = p->z[i] + g->dt * u[2] / gam / g->dz;
        if (g->bc_x == OR_BC_PERIODIC)
            X1 = wrap_pos3(X1, (double)g->nx);
        p->x[i] = X1;
        p->y[i] = wrap_pos3(Y1, (double)g->ny);
        p->z[i] = wrap_pos3(Z1, (double)g->nz);
        p->ux[i] = u[0];
        p->uy[i] = u[1];
        p->uz[i] = u[2];
        p->sx[i] = s[0];
        p->sy[i] = s[1];
        p->sz[i] = s[2];
    }
}

/* a5: 3D Esirkepov current of one move (cell units, |dX| < 1 per axis) on the
 * 4x4x4 node stencil starting at floor(X0) - 1:
 *   Wx = dSx (S0y S0z + dSy S0z/2 + S0y dSz/2 + dSy dSz/3), Wy and Wz likewise,
 *   Jx(i+1/2) - Jx(i-1/2) = -q w (dx/dt) Wx(i), and so on for y and z. */
void or3_deposit_one(const or_grid3_t *g, or_fields3_t *f, double qw, double X0, double Y0,
                     double Z0, double X1, double Y1, double Z1)
{
    if (fabs(X1 - X0) >= 1.0 || fabs(Y1 - Y0) >= 1.0 || fabs(Z1 - Z0) >= 1.0)
        or3_fail("particle moved a cell or more in one step (CFL)");
    long i0 = (long)floor(X0) - 1, j0 = (long)floor(Y0) - 1, k0 = (long)floor(Z0) - 1;
    double S0x[4], S0y[4], S0z[4], dSx[4], dSy[4], dSz[4];
    for (int a = 0; a < 4; ++a) {
        S0x[a] = shape1_3(X0 - (double)(i0 + a));
        S0y[a] = shape1_3(Y0 - (double)(j0 + a));
        S0z[a] = shape1_3(Z0 - (double)(k0 + a));
        dSx[a] = shape1_3(X1 - (double)(i0 + a)) - S0x[a];
        dSy[a] = shape1_3(Y1 - (double)(j0 + a)) - S0y[a];
        dSz[a] = shape1_3(Z1 - (double)(k0 + a)) - S0z[a];
    }
    double cx = -qw * g->dx / g->dt, cy = -qw * g->dy / g->dt, cz = -qw * g->dz / g->dt;
    for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 4; ++k) {
            double yz = S0y[j] * S0z[k] + 0.5 * dSy[j] * S0z[k] + 0.5 * S0y[j] * dSz[k] +
                        dSy[j] * dSz[k] / 3.0;
            double acc = 0.0;
            for (int i = 0; i < 3; ++i) {
                acc += dSx[i] * yz;
                f->jx[at3(g, i0 + i, j0 + j, k0 + k)] += cx * acc;
            }
        }
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k) {
            double xz = S0x[i] * S0z[k] + 0.5 * dSx[i] * S0z[k] + 0.5 * S0x[i] * dSz[k] +
                        dSx[i] * dSz[k] / 3.0;
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) {
                acc += dSy[j] * xz;
                f->jy[at3(g, i0 + i, j0 + j, k0 + k)] += cy * acc;
            }
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double xy = S0x[i] * S0y[j] + 0.5 * dSx[i] * S0y[j] + 0.5 * S0x[i] * dSy[j] +
                        dSx[i] * dSy[j] / 3.0;
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) {
                acc += dSz[k] * xy;
                f->jz[at3(g, i0 + i, j0 + j, k0 + k)] += cz * acc;
            }
        }
}

void or3_deposit(const or_grid3_t *g, const or_species_t *sp, or_particles3_t *p,
                 const double *x_old, const double *y_old, const double *z_old, or_fields3_t *f)
{
    for (long i = 0; i < p->n; ++i) {
        if (!p->alive[i])
            continue;
        double X1 = p->x[i];
        if (g->bc_x == OR_BC_PERIODIC)
            X1 = unwrap3(X1, x_old[i], (double)g->nx);
        double Y1 = unwrap3(p->y[i], y_old[i], (double)g->ny);
        double Z1 = unwrap3(p->z[i], z_old[i], (double)g->nz);
        or3_deposit_one(g, f, sp->q * p->w[i], x_old[i], y_old[i], z_old[i], X1, Y1, Z1);
        if (g->bc_x == OR_BC_OPEN && (p->x[i] < 2.0 || p->x[i] >= (double)(g->nx - 2)))
            p->alive[i] = 0;
    }
}

/* laser at x = 0: comp 0 the incident Ey (= Bz), comp 1 the incident Ez (= -By);
 * Gaussian in t and in the transverse radius (waist w0, centred on the box) */
void or3_laser(const or_grid3_t *g, double t, double y, double z, int comp, double *val)
{
    double e = (t - g->t_peak) / g->tau;
    double yc = 0.5 * g->ny * g->dy, zc = 0.5 * g->nz * g->dz;
    double r2 = ((y - yc) * (y - yc) + (z - zc) * (z - zc)) / (g->w0 * g->w0);
    double env = exp(-e * e) * exp(-r2), ph = t - g->t_peak, v = 0.0;
    if (g->pol == OR_POL_LP_Y)
        v = comp == 0 ? g->a0 * env * sin(ph) : 0.0;
    else if (g->pol == OR_POL_CP)
        v = g->a0 / sqrt(2.0) * env * (comp == 0 ? sin(ph) : cos(ph));
    *val = v;
}

/* B <- B - h curl E (Yee 1966); By, Bz skip the last column with open x */
static void b_half3(const or_grid3_t *g, or_fields3_t *f, double h)
{
    long nx = g->nx, ny = g->ny, nz = g->nz;
    long last = g->bc_x == OR_BC_PERIODIC ? nx : nx - 1;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = at3(g, i, j, k);
                long cjp = at3(g, i, j + 1, k), ckp = at3(g, i, j, k + 1);
                f->bx[c] -= h * ((f->ez[cjp] - f->ez[c]) / g->dy - (f->ey[ckp] - f->ey[c]) / g->dz);
                if (i < last) {
                    long cip = at3(g, i + 1, j, k);
                    f->by[c] -= h * ((f->ex[ckp] - f->ex[c]) / g->dz - (f->ez[cip] - f->ez[c]) / g->dx);
                    f->bz[c] -= h * ((f->ey[cip] - f->ey[c]) / g->dx - (f->ex[cjp] - f->ex[c]) / g->dy);
                }
            }
}

/* a6 in 3D: B half step; open x: boundary B at t^{n+1/2} from the incoming
 * characteristic with the transverse terms of both tangential E updates
 * (r = dt/dx, qy = dt/dy, qz = dt/dz):
 *   By(-1/2) = [2 Ez(0) - (1-r) By(1/2) - qy dyBx - 4 f] / (1+r)
 *   Bz(-1/2) = [4 g - 2 Ey(0) - (1-r) Bz(1/2) - qz dzBx] / (1+r)
 *   By(nx-1/2) = [-2 Ez - (1-r) By(nx-3/2) + qy dyBx] / (1+r)
 *   Bz(nx-1/2) = [ 2 Ey - (1-r) Bz(nx-3/2) + qz dzBx] / (1+r)
 * with dyBx = Bx(j+1/2) - Bx(j-1/2) at z k+1/2 and dzBx = Bx(k+1/2) - Bx(k-1/2)
 * at y j+1/2; then E full step with -J and the second B half step. */
void or3_field_update(const or_grid3_t *g, or_fields3_t *f, long step)
{
    long nx = g->nx, ny = g->ny, nz = g->nz;
    double dt = g->dt;
    b_half3(g, f, 0.5 * dt);
    if (g->bc_x == OR_BC_OPEN) {
        double r = dt / g->dx, qy = dt / g->dy, qz = dt / g->dz, t = ((double)step + 0.5) * dt;
#pragma omp parallel for schedule(static)
        for (long k = 0; k < nz; ++k)
            for (long j = 0; j < ny; ++j) {
                double fin, gin;
                or3_laser(g, t, (double)j * g->dy, ((double)k + 0.5) * g->dz, 1, &fin);
                or3_laser(g, t, ((double)j + 0.5) * g->dy, (double)k * g->dz, 0, &gin);
                long c0 = at3(g, 0, j, k), cl = at3(g, nx - 1, j, k);
                double dyb0 = f->bx[c0] - f->bx[at3(g, 0, j - 1, k)];
                double dzb0 = f->bx[c0] - f->bx[at3(g, 0, j, k - 1)];
                double dybl = f->bx[cl] - f->bx[at3(g, nx - 1, j - 1, k)];
                double dzbl = f->bx[cl] - f->bx[at3(g, nx - 1, j, k - 1)];
                long b = k * ny + j;
                f->byL[b] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - qy * dyb0 - 4.0 * fin) / (1.0 + r);
                f->bzL[b] = (4.0 * gin - 2.0 * f->ey[c0] - (1.0 - r) * f->bz[c0] - qz * dzb0) / (1.0 + r);
                f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1] + qy * dybl) / (1.0 + r);
                f->bz[cl] = (2.0 * f->ey[cl] - (1.0 - r) * f->bz[cl - 1] + qz * dzbl) / (1.0 + r);
            }
    }
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                long c = at3(g, i, j, k), cjm = at3(g, i, j - 1, k), ckm = at3(g, i, j, k - 1);
                double by_im, bz_im;
                if (i > 0) {
                    by_im = f->by[c - 1];
                    bz_im = f->bz[c - 1];
                } else if (g->bc_x == OR_BC_PERIODIC) {
                    by_im = f->by[at3(g, nx - 1, j, k)];
                    bz_im = f->bz[at3(g, nx - 1, j, k)];
                } else {
                    by_im = f->byL[k * ny + j];
                    bz_im = f->bzL[k * ny + j];
                }
                f->ex[c] += dt * ((f->bz[c] - f->bz[cjm]) / g->dy - (f->by[c] - f->by[ckm]) / g->dz - f->jx[c]);
                f->ey[c] += dt * ((f->bx[c] - f->bx[ckm]) / g->dz - (f->bz[c] - bz_im) / g->dx - f->jy[c]);
                f->ez[c] += dt * ((f->by[c] - by_im) / g->dx - (f->bx[c] - f->bx[cjm]) / g->dy - f->jz[c]);
            }
    b_half3(g, f, 0.5 * dt);
}

void or3_step(const or_grid3_t *g, const or_species_t *sp, or_particles3_t *p, const int *mobile,
              int nsp, or_fields3_t *f, long step)
{
    long nc = (long)g->nx * g->ny * g->nz;
    for (long c = 0; c < nc; ++c)
        f->jx[c] = f->jy[c] = f->jz[c] = 0.0;
    for (int s = 0; s < nsp; ++s) {
        if (!mobile[s] || p[s].n == 0)
            continue;
        long n = p[s].n;
        double *xo = malloc(sizeof(double) * n), *yo = malloc(sizeof(double) * n),
               *zo = malloc(sizeof(double) * n);
        if (!xo || !yo || !zo)
            or3_fail("out of memory");
        or3_push(g, &sp[s], &p[s], f, xo, yo, zo);
        or3_deposit(g, &sp[s], &p[s], xo, yo, zo, f);
        free(xo);
        free(yo);
        free(zo);
    }
    or3_field_update(g, f, step);
}

void or3_rho(const or_grid3_t *g, const or_species_t *sp, const or_particles3_t *p, double *rho)
{
    for (long n = 0; n < p->n; ++n) {
        if (!p->alive[n])
            continue;
        long i0 = (long)floor(p->x[n]), j0 = (long)floor(p->y[n]), k0 = (long)floor(p->z[n]);
        for (long a = 0; a < 2; ++a)
            for (long b = 0; b < 2; ++b)
                for (long c = 0; c < 2; ++c) {
                    double w = shape1_3(p->x[n] - (double)(i0 + a)) *
                               shape1_3(p->y[n] - (double)(j0 + b)) *
                               shape1_3(p->z[n] - (double)(k0 + c));
                    rho[at3(g, i0 + a, j0 + b, k0 + c)] += sp->q * p->w[n] * w;
                }
    }
}

/* div E on nodes; with open x the column i = 0 is left at 0 */
void or3_div_e(const or_grid3_t *g, const or_fields3_t *f, double *div)
{
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long c = at3(g, i, j, k);
                if (i == 0 && g->bc_x == OR_BC_OPEN) {
                    div[c] = 0.0;
                    continue;
                }
                div[c] = (f->ex[c] - f->ex[at3(g, i - 1, j, k)]) / g->dx +
                         (f->ey[c] - f->ey[at3(g, i, j - 1, k)]) / g->dy +
                         (f->ez[c] - f->ez[at3(g, i, j, k - 1)]) / g->dz;
            }
}

/* div B on cell centres (i+1/2, j+1/2, k+1/2); with open x the last column is 0 */
void or3_div_b(const or_grid3_t *g, const or_fields3_t *f, double *div)
{
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long c = at3(g, i, j, k);
                if (i == g->nx - 1 && g->bc_x == OR_BC_OPEN) {
                    div[c] = 0.0;
                    continue;
                }
                div[c] = (f->bx[at3(g, i + 1, j, k)] - f->bx[c]) / g->dx +
                         (f->by[at3(g, i, j + 1, k)] - f->by[c]) / g->dy +
                         (f->bz[at3(g, i, j, k + 1)] - f->bz[c]) / g->dz;
            }
}
