/*
 * pic_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see pic_oracle.h).
 *
 * Scalar loops, no blocking, no reordering.  Each function names the
 * equation or published method it writes out.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#define MEC2_MEV 0.51099895 /* electron rest energy [MeV] */

static void or_fail(const char *what)
{
    fprintf(stderr, "pic_oracle: %s\n", what);
    abort();
}

/* periodic wrap of a node index */
static long wrapi(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* node index along x: periodic wrap, or a range check for open boundaries */
static long xi(const or_grid_t *g, long i)
{
    if (g->bc_x == OR_BC_PERIODIC)
        return wrapi(i, g->nx);
    if (i < 0 || i >= g->nx)
        or_fail("x node index outside the mesh");
    return i;
}

static long yj(const or_grid_t *g, long j) { return wrapi(j, g->ny); }

/* first-order (cloud-in-cell) shape S(xi) = max(0, 1 - |xi|) */
static double shape1(double d)
{
    double a = fabs(d);
    return a < 1.0 ? 1.0 - a : 0.0;
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---------------------------------------------------------------------------
 * a1: CIC interpolation of one Yee component sitting at (i + sx, j + sy).
 * ------------------------------------------------------------------------- */
static double interp(const or_grid_t *g, const double *F, double X, double Y,
                     double sx, double sy)
{
    double xs = X - sx, ys = Y - sy;
    long i0 = (long)floor(xs), j0 = (long)floor(ys);
    double v = 0.0;
    for (long di = 0; di < 2; ++di)
        for (long dj = 0; dj < 2; ++dj) {
            long i = i0 + di, j = j0 + dj;
            double wgt = shape1(xs - (double)i) * shape1(ys - (double)j);
            v += wgt * F[yj(g, j) * g->nx + xi(g, i)];
        }
    return v;
}

void or_gather(const or_grid_t *g, const or_fields_t *f, double X, double Y,
               double E[3], double B[3])
{
    E[0] = interp(g, f->ex, X, Y, 0.5, 0.0);
    E[1] = interp(g, f->ey, X, Y, 0.0, 0.5);
    E[2] = interp(g, f->ez, X, Y, 0.0, 0.0);
    B[0] = interp(g, f->bx, X, Y, 0.0, 0.5);
    B[1] = interp(g, f->by, X, Y, 0.5, 0.0);
    B[2] = interp(g, f->bz, X, Y, 0.5, 0.5);
}

/* ---------------------------------------------------------------------------
 * a2: Boris push (Boris 1970) of u = gamma v over dt in fields E, B:
 * half electric kick, magnetic rotation, half electric kick.
 * ------------------------------------------------------------------------- */
void or_boris(double qm, double dt, const double E[3], const double B[3], double u[3])
{
    double um[3], t[3], s[3], up[3], c[3];
    for (int k = 0; k < 3; ++k)
        um[k] = u[k] + 0.5 * qm * dt * E[k];
    double gm = sqrt(1.0 + dot3(um, um));
    for (int k = 0; k < 3; ++k)
        t[k] = 0.5 * qm * dt * B[k] / gm;
    double t2 = dot3(t, t);
    for (int k = 0; k < 3; ++k)
        s[k] = 2.0 * t[k] / (1.0 + t2);
    cross3(um, t, c);
    for (int k = 0; k < 3; ++k)
        up[k] = um[k] + c[k];
    cross3(up, s, c);
    for (int k = 0; k < 3; ++k)
        u[k] = um[k] + c[k] + 0.5 * qm * dt * E[k];
}

/* ---------------------------------------------------------------------------
 * a3: Thomas-BMT precession vector, Eq. (2) with the coefficients of Eq. (3),
 * in units with c = 1 so q/(m c) -> q/m and v/c -> v.
 * ------------------------------------------------------------------------- */
void or_omega(double qm, double a, const double ubar[3], const double E[3],
              const double B[3], double Om[3])
{
    double gam = sqrt(1.0 + dot3(ubar, ubar));
    double v[3] = {ubar[0] / gam, ubar[1] / gam, ubar[2] / gam};
    double omB = a + 1.0 / gam;            /* Eq. (3) */
    double omv = a * gam / (gam + 1.0);    /* Eq. (3) */
    double omE = a + 1.0 / (1.0 + gam);    /* Eq. (3) */
    double vB = dot3(v, B);
    double vxE[3];
    cross3(v, E, vxE);
    for (int k = 0; k < 3; ++k)
        Om[k] = qm * (omB * B[k] - omv * vB * v[k] - omE * vxE[k]);
}

/* Eq. (1), ds/dt = -Omega x s, integrated over dt with Omega held fixed:
 * a rotation of s by theta = |Omega| dt about n = -Omega/|Omega| (Rodrigues). */
void or_spin_rotate(const double Om[3], double dt, double s[3])
{
    double om = sqrt(dot3(Om, Om));
    if (om * dt < 1e-300)
        return;
    double n[3] = {-Om[0] / om, -Om[1] / om, -Om[2] / om};
    double th = om * dt;
    double c = cos(th), sn = sin(th);
    double nxs[3];
    cross3(n, s, nxs);
    double ns = dot3(n, s);
    for (int k = 0; k < 3; ++k)
        s[k] = s[k] * c + nxs[k] * sn + n[k] * ns * (1.0 - c);
}

/* ---------------------------------------------------------------------------
 * a5: Esirkepov charge-conserving current of one particle moving from
 * (X0, Y0) to (X1, Y1) (cell units, |X1 - X0| < 1) with out-of-plane velocity
 * vz, first-order shapes on the 4x4 node stencil starting at floor(X0) - 1.
 *   Wx = dSx (S0y + dSy/2),  Wy = dSy (S0x + dSx/2),
 *   Wz = S0x S0y + dSx S0y/2 + S0x dSy/2 + dSx dSy/3,
 *   Jx(i+1/2) - Jx(i-1/2) = -q w (dx/dt) Wx(i),   likewise Jy along y,
 *   Jz = q w vz Wz.
 * ------------------------------------------------------------------------- */
void or_deposit_one(const or_grid_t *g, or_fields_t *f, double qw,
                    double X0, double Y0, double X1, double Y1, double vz)
{
    if (fabs(X1 - X0) >= 1.0 || fabs(Y1 - Y0) >= 1.0)
        or_fail("particle moved a cell or more in one step (CFL)");
    long i0 = (long)floor(X0) - 1, j0 = (long)floor(Y0) - 1;
    double S0x[4], S1x[4], S0y[4], S1y[4], dSx[4], dSy[4];
    for (int k = 0; k < 4; ++k) {
        S0x[k] = shape1(X0 - (double)(i0 + k));
        S1x[k] = shape1(X1 - (double)(i0 + k));
        S0y[k] = shape1(Y0 - (double)(j0 + k));
        S1y[k] = shape1(Y1 - (double)(j0 + k));
        dSx[k] = S1x[k] - S0x[k];
        dSy[k] = S1y[k] - S0y[k];
    }
    double cx = -qw * g->dx / g->dt, cy = -qw * g->dy / g->dt;
    /* Jx on half nodes (i0+k)+1/2, k = 0..2: running sum over k */
    for (int l = 0; l < 4; ++l) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) {
            acc += dSx[k] * (S0y[l] + 0.5 * dSy[l]);
            f->jx[yj(g, j0 + l) * g->nx + xi(g, i0 + k)] += cx * acc;
        }
    }
    /* Jy on half nodes (j0+l)+1/2, l = 0..2: running sum over l */
    for (int k = 0; k < 4; ++k) {
        double acc = 0.0;
        for (int l = 0; l < 3; ++l) {
            acc += dSy[l] * (S0x[k] + 0.5 * dSx[k]);
            f->jy[yj(g, j0 + l) * g->nx + xi(g, i0 + k)] += cy * acc;
        }
    }
    for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) {
            double wz = S0x[k] * S0y[l] + 0.5 * dSx[k] * S0y[l] +
                        0.5 * S0x[k] * dSy[l] + dSx[k] * dSy[l] / 3.0;
            f->jz[yj(g, j0 + l) * g->nx + xi(g, i0 + k)] += qw * vz * wz;
        }
}

/* position into [0, n) for a periodic axis */
static double wrap_pos(double X, double n)
{
    double r = X - n * floor(X / n);
    if (r >= n)
        r -= n;
    if (r < 0.0)
        r = 0.0;
    return r;
}

/* a1-a4 for every live particle of one species.  Saves x^n, y^n and
 * v_z^{n+1/2} for the deposit; spin and momentum live at half-integer times. */
void or_push(const or_grid_t *g, const or_species_t *sp, or_particles_t *p,
             const or_fields_t *f, double *x_old, double *y_old, double *vz)
{
    double qm = sp->q / sp->m;
    /* particles are independent here: the OpenMP build splits them over threads */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < p->n; ++i) {
        x_old[i] = p->x[i];
        y_old[i] = p->y[i];
        vz[i] = 0.0;
        if (!p->alive[i])
            continue;
        double E[3], B[3];
        or_gather(g, f, p->x[i], p->y[i], E, B);
        double u0[3] = {p->ux[i], p->uy[i], p->uz[i]};
        double u[3] = {u0[0], u0[1], u0[2]};
        or_boris(qm, g->dt, E, B, u);
        /* a3: Omega from E^n, B^n and the mean of the two half-step momenta */
        double ubar[3] = {0.5 * (u0[0] + u[0]), 0.5 * (u0[1] + u[1]), 0.5 * (u0[2] + u[2])};
        double Om[3], s[3] = {p->sx[i], p->sy[i], p->sz[i]};
        or_omega(qm, sp->a, ubar, E, B, Om);
        or_spin_rotate(Om, g->dt, s);
        /* a4: x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2} */
        double gam = sqrt(1.0 + dot3(u, u));
        double X1 = p->x[i] + g->dt * u[0] / gam / g->dx;
        double Y1 = p->y[i] + g->dt * u[1] / gam / g->dy;
        if (g->bc_x == OR_BC_PERIODIC)
            X1 = wrap_pos(X1, (double)g->nx);
        Y1 = wrap_pos(Y1, (double)g->ny);
        p->x[i] = X1;
        p->y[i] = Y1;
        p->ux[i] = u[0];
        p->uy[i] = u[1];
        p->uz[i] = u[2];
        p->sx[i] = s[0];
        p->sy[i] = s[1];
        p->sz[i] = s[2];
        vz[i] = u[2] / gam;
    }
}

/* the copy of X1 closest to X0 on a periodic axis of length n */
static double unwrap(double X1, double X0, double n)
{
    if (X1 - X0 > 0.5 * n)
        return X1 - n;
    if (X0 - X1 > 0.5 * n)
        return X1 + n;
    return X1;
}

/* a5 for every particle live at x^n; with open x boundaries a particle whose
 * new position is outside [2, nx-2) is removed after its current is laid down. */
void or_deposit(const or_grid_t *g, const or_species_t *sp, or_particles_t *p,
                const double *x_old, const double *y_old, const double *vz,
                or_fields_t *f)
{
    for (long i = 0; i < p->n; ++i) {
        if (!p->alive[i])
            continue;
        double X1 = p->x[i], Y1 = unwrap(p->y[i], y_old[i], (double)g->ny);
        if (g->bc_x == OR_BC_PERIODIC)
            X1 = unwrap(X1, x_old[i], (double)g->nx);
        or_deposit_one(g, f, sp->q * p->w[i], x_old[i], y_old[i], X1, Y1, vz[i]);
        if (g->bc_x == OR_BC_OPEN && (p->x[i] < 2.0 || p->x[i] >= (double)(g->nx - 2)))
            p->alive[i] = 0;
    }
}

/* ---------------------------------------------------------------------------
 * Laser source at x = 0.  comp 0: the incident Ey (= Bz) of the wave moving
 * in +x; comp 1: the incident Ez (= -By).  Gaussian in time (1/e field time
 * tau, peak t_peak) and in y (waist w0, centred on the box).
 * ------------------------------------------------------------------------- */
void or_laser(const or_grid_t *g, double t, double y, int comp, double *val)
{
    double env = exp(-((t - g->t_peak) / g->tau) * ((t - g->t_peak) / g->tau));
    double yc = 0.5 * g->ny * g->dy;
    double tr = exp(-((y - yc) / g->w0) * ((y - yc) / g->w0));
    double ph = t - g->t_peak;
    double v = 0.0;
    if (g->pol == OR_POL_LP_Y)
        v = comp == 0 ? g->a0 * env * tr * sin(ph) : 0.0;
    else if (g->pol == OR_POL_CP)
        v = g->a0 / sqrt(2.0) * env * tr * (comp == 0 ? sin(ph) : cos(ph));
    *val = v;
}

/* B <- B - h curl E on every B node the interior stencil reaches (Yee 1966) */
static void b_half(const or_grid_t *g, or_fields_t *f, double h)
{
    long nx = g->nx, ny = g->ny;
    long last = g->bc_x == OR_BC_PERIODIC ? nx : nx - 1; /* By, Bz columns updated */
#pragma omp parallel for schedule(static)
    for (long j = 0; j < ny; ++j) {
        long jp = yj(g, j + 1);
        for (long i = 0; i < nx; ++i) {
            long c = j * nx + i;
            f->bx[c] -= h / g->dy * (f->ez[jp * nx + i] - f->ez[c]);
            if (i < last) {
                long ip = xi(g, i + 1);
                f->by[c] += h / g->dx * (f->ez[j * nx + ip] - f->ez[c]);
                f->bz[c] -= h / g->dx * (f->ey[j * nx + ip] - f->ey[c]) -
                            h / g->dy * (f->ex[jp * nx + i] - f->ex[c]);
            }
        }
    }
}

/* a6: B half step, boundary B values, E full step with -J, B half step.
 * Open x: first-order Silver-Mueller condition at t^{n+1/2} on the B values
 * half a cell outside the outermost tangential E nodes.  The condition on
 * the incoming characteristic (Ez - By = 2f, Ey + Bz = 2g at x_min with the
 * laser's incident f, g; Ez + By = 0, Ey - Bz = 0 at x_max) is imposed on
 * the time-centred boundary values, with E^{n+1} taken from its own update,
 * including the transverse term dBx = Bx(j+1/2) - Bx(j-1/2) of the Ez
 * update (r = dt/dx, q = dt/dy):
 *   By(-1/2) = [2 Ez(0) - (1-r) By(1/2) - q dBx(0) - 4 f] / (1+r)
 *   Bz(-1/2) = [4 g - 2 Ey(0) - (1-r) Bz(1/2)] / (1+r)
 *   By(nx-1/2) = [-2 Ez(nx-1) - (1-r) By(nx-3/2) + q dBx(nx-1)] / (1+r)
 *   Bz(nx-1/2) = [ 2 Ey(nx-1) - (1-r) Bz(nx-3/2)] / (1+r)
 * (dropping the q dBx terms leaves a condition that is unstable for fields
 * varying along y). */
void or_field_update(const or_grid_t *g, or_fields_t *f, long step)
{
    long nx = g->nx, ny = g->ny;
    double dt = g->dt;
    b_half(g, f, 0.5 * dt);
    if (g->bc_x == OR_BC_OPEN) {
        double r = dt / g->dx, q = dt / g->dy, t = ((double)step + 0.5) * dt;
#pragma omp parallel for schedule(static)
        for (long j = 0; j < ny; ++j) {
            double fin, gin;
            or_laser(g, t, (double)j * g->dy, 1, &fin);
            or_laser(g, t, ((double)j + 0.5) * g->dy, 0, &gin);
            long c0 = j * nx, cl = j * nx + nx - 1, jm = yj(g, j - 1);
            double dbx0 = f->bx[c0] - f->bx[jm * nx];
            double dbxl = f->bx[cl] - f->bx[jm * nx + nx - 1];
            f->byL[j] = (2.0 * f->ez[c0] - (1.0 - r) * f->by[c0] - q * dbx0 - 4.0 * fin) / (1.0 + r);
            f->bzL[j] = (4.0 * gin - 2.0 * f->ey[c0] - (1.0 - r) * f->bz[c0]) / (1.0 + r);
            f->by[cl] = (-2.0 * f->ez[cl] - (1.0 - r) * f->by[cl - 1] + q * dbxl) / (1.0 + r);
            f->bz[cl] = (2.0 * f->ey[cl] - (1.0 - r) * f->bz[cl - 1]) / (1.0 + r);
        }
    }
#pragma omp parallel for schedule(static)
    for (long j = 0; j < ny; ++j) {
        long jm = yj(g, j - 1);
        for (long i = 0; i < nx; ++i) {
            long c = j * nx + i;
            double bz_im, by_im;
            if (i > 0) {
                bz_im = f->bz[c - 1];
                by_im = f->by[c - 1];
            } else if (g->bc_x == OR_BC_PERIODIC) {
                bz_im = f->bz[j * nx + nx - 1];
                by_im = f->by[j * nx + nx - 1];
            } else {
                bz_im = f->bzL[j];
                by_im = f->byL[j];
            }
            f->ex[c] += dt * ((f->bz[c] - f->bz[jm * nx + i]) / g->dy - f->jx[c]);
            f->ey[c] += dt * (-(f->bz[c] - bz_im) / g->dx - f->jy[c]);
            f->ez[c] += dt * ((f->by[c] - by_im) / g->dx -
                              (f->bx[c] - f->bx[jm * nx + i]) / g->dy - f->jz[c]);
        }
    }
    b_half(g, f, 0.5 * dt);
}

void or_step(const or_grid_t *g, const or_species_t *sp, or_particles_t *p,
             const int *mobile, int nsp, or_fields_t *f, long step)
{
    long nc = (long)g->nx * g->ny;
    for (long c = 0; c < nc; ++c)
        f->jx[c] = f->jy[c] = f->jz[c] = 0.0;
    for (int s = 0; s < nsp; ++s) {
        if (!mobile[s] || p[s].n == 0)
            continue;
        long n = p[s].n;
        double *xo = malloc(sizeof(double) * n), *yo = malloc(sizeof(double) * n),
               *vz = malloc(sizeof(double) * n);
        if (!xo || !yo || !vz)
            or_fail("out of memory");
        or_push(g, &sp[s], &p[s], f, xo, yo, vz);
        or_deposit(g, &sp[s], &p[s], xo, yo, vz, f);
        free(xo);
        free(yo);
        free(vz);
    }
    or_field_update(g, f, step);
}

/* ---------------------------------------------------------------------------
 * diagnostics
 * ------------------------------------------------------------------------- */
void or_rho(const or_grid_t *g, const or_species_t *sp, const or_particles_t *p,
            double *rho)
{
    for (long i = 0; i < p->n; ++i) {
        if (!p->alive[i])
            continue;
        long i0 = (long)floor(p->x[i]), j0 = (long)floor(p->y[i]);
        for (long di = 0; di < 2; ++di)
            for (long dj = 0; dj < 2; ++dj) {
                double wgt = shape1(p->x[i] - (double)(i0 + di)) *
                             shape1(p->y[i] - (double)(j0 + dj));
                rho[yj(g, j0 + dj) * g->nx + xi(g, i0 + di)] += sp->q * p->w[i] * wgt;
            }
    }
}

/* div E on nodes (i, j); with open x the column i = 0 is left at 0 */
void or_div_e(const or_grid_t *g, const or_fields_t *f, double *div)
{
    long nx = g->nx, ny = g->ny;
    for (long j = 0; j < ny; ++j) {
        long jm = yj(g, j - 1);
        for (long i = 0; i < nx; ++i) {
            long c = j * nx + i;
            if (i == 0 && g->bc_x == OR_BC_OPEN) {
                div[c] = 0.0;
                continue;
            }
            long im = xi(g, i - 1);
            div[c] = (f->ex[c] - f->ex[j * nx + im]) / g->dx +
                     (f->ey[c] - f->ey[jm * nx + i]) / g->dy;
        }
    }
}

/* div B on cell centres (i+1/2, j+1/2); with open x the last column is 0 */
void or_div_b(const or_grid_t *g, const or_fields_t *f, double *div)
{
    long nx = g->nx, ny = g->ny;
    for (long j = 0; j < ny; ++j) {
        long jp = yj(g, j + 1);
        for (long i = 0; i < nx; ++i) {
            long c = j * nx + i;
            if (i == nx - 1 && g->bc_x == OR_BC_OPEN) {
                div[c] = 0.0;
                continue;
            }
            long ip = xi(g, i + 1);
            div[c] = (f->bx[j * nx + ip] - f->bx[c]) / g->dx +
                     (f->by[jp * nx + i] - f->by[c]) / g->dy;
        }
    }
}

/* Eq. (4) over the live particles whose kinetic energy (gamma - 1) m c^2 lies
 * in [emin, emax), weighted by w (equal weights give Eq. (4) exactly). */
void or_moments(const or_species_t *sp, const or_particles_t *p,
                double emin_mev, double emax_mev, double out[7])
{
    double sw = 0, swx = 0, swy = 0, swz = 0, cnt = 0, swe = 0;
    for (long i = 0; i < p->n; ++i) {
        if (!p->alive[i])
            continue;
        double u[3] = {p->ux[i], p->uy[i], p->uz[i]};
        double ek = (sqrt(1.0 + dot3(u, u)) - 1.0) * sp->m * MEC2_MEV;
        if (ek < emin_mev || ek >= emax_mev)
            continue;
        sw += p->w[i];
        swx += p->w[i] * p->sx[i];
        swy += p->w[i] * p->sy[i];
        swz += p->w[i] * p->sz[i];
        swe += p->w[i] * ek;
        cnt += 1.0;
    }
    double mean = sw > 0 ? swe / sw : 0.0, var = 0.0;
    for (long i = 0; i < p->n && sw > 0; ++i) {
        if (!p->alive[i])
            continue;
        double u[3] = {p->ux[i], p->uy[i], p->uz[i]};
        double ek = (sqrt(1.0 + dot3(u, u)) - 1.0) * sp->m * MEC2_MEV;
        if (ek < emin_mev || ek >= emax_mev)
            continue;
        var += p->w[i] * (ek - mean) * (ek - mean);
    }
    out[0] = sw > 0 ? swx / sw : 0.0;
    out[1] = sw > 0 ? swy / sw : 0.0;
    out[2] = sw > 0 ? swz / sw : 0.0;
    out[3] = sw;
    out[4] = cnt;
    out[5] = mean;
    out[6] = sw > 0 ? var / sw : 0.0;
}

/* Energy spectra behind Figs. 1-3 (c), (d): per kinetic-energy bin the
 * particle count, the weight and the weighted spin; dP/dE of a bin is its
 * sum w s / sum w (Eq. 4 restricted to the bin). */
void or_histogram(const or_species_t *sp, const or_particles_t *p, double emin_mev,
                  double emax_mev, int nbins, int log_bins, double *out)
{
    for (int b = 0; b < 5 * nbins; ++b)
        out[b] = 0.0;
    for (long i = 0; i < p->n; ++i) {
        if (!p->alive[i])
            continue;
        double u[3] = {p->ux[i], p->uy[i], p->uz[i]};
        double ek = (sqrt(1.0 + dot3(u, u)) - 1.0) * sp->m * MEC2_MEV;
        if (ek < emin_mev || ek >= emax_mev)
            continue;
        double f = log_bins ? log(ek / emin_mev) / log(emax_mev / emin_mev)
                            : (ek - emin_mev) / (emax_mev - emin_mev);
        int b = (int)floor(f * nbins);
        if (b < 0)
            b = 0;
        if (b >= nbins)
            b = nbins - 1;
        out[5 * b + 0] += 1.0;
        out[5 * b + 1] += p->w[i];
        out[5 * b + 2] += p->w[i] * p->sx[i];
        out[5 * b + 3] += p->w[i] * p->sy[i];
        out[5 * b + 4] += p->w[i] * p->sz[i];
    }
}

/* Threads the parallel loops of this build use: 1 in the plain build; the
 * OpenMP build (the multi-core CPU baseline) parallelises only loops whose
 * iterations are independent (the per-particle push, the Yee stages by row),
 * so its results are bit-identical to the plain build's. */
#ifdef _OPENMP
#include <omp.h>
#endif
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
