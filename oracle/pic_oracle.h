/*
 * pic_oracle.h -- plain FP64 CPU oracle of one 2D3V electromagnetic PIC step
 * with Thomas-BMT spin tracking.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * reference the GPU path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (units: time 1/omega0, length c/omega0, momentum u = p/(m c),
 * fields m_e c omega0 / e, density n_c, charge e, mass m_e):
 *   - spin:          ds/dt = -Omega x s                         (Eq. 1)
 *   - precession:    Omega = (q/m)[Om_B B - Om_v (v.B) v - Om_E v x E]   (Eq. 2, c = 1)
 *   - coefficients:  Om_B = a + 1/g, Om_v = a g/(g+1), Om_E = a + 1/(1+g)  (Eq. 3)
 *   - polarization:  P = (1/N) sum s_i  (weighted form sum w s / sum w)  (Eq. 4)
 * and the particle-in-cell parts the paper leaves to its PIC code (Sec. 2):
 * CIC gather on the Yee mesh (Yee 1966), the Boris push (Boris 1970), the
 * charge-conserving current of Esirkepov (Comput. Phys. Commun. 135, 144,
 * 2001) and the Yee FDTD update with a first-order Silver-Mueller boundary
 * that injects the laser at x_min.
 *
 * Positions are global doubles in cell units: node i of the mesh sits at X = i.
 * Mesh arrays are row major [ny][nx]; staggering of element [j][i]:
 *   Ex (i+1/2, j)   Ey (i, j+1/2)   Ez (i, j)
 *   Bx (i, j+1/2)   By (i+1/2, j)   Bz (i+1/2, j+1/2)
 *   Jx, Jy, Jz as Ex, Ey, Ez.
 * With open x boundaries By[j][nx-1] and Bz[j][nx-1] (x = nx - 1/2) hold the
 * right-hand boundary values, and byL[j], bzL[j] (x = -1/2) the left-hand ones.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_BC_OPEN 0     /* Silver-Mueller at x_min (laser source) and x_max */
#define OR_BC_PERIODIC 1 /* periodic in x                                     */

#define OR_POL_NONE 0
#define OR_POL_LP_Y 1
#define OR_POL_CP 2

typedef struct {
    int nx, ny;
    double dx, dy, dt;        /* c/omega0, 1/omega0 */
    int bc_x;                 /* OR_BC_OPEN or OR_BC_PERIODIC; y is periodic */
    int pol;                  /* laser polarization (open x only) */
    double a0, w0, tau, t_peak; /* amplitude, waist [c/omega0], envelope 1/e time, peak time */
} or_grid_t;

typedef struct {
    double q, m, a;           /* charge [e], mass [m_e], gyromagnetic anomaly */
} or_species_t;

typedef struct {
    double *ex, *ey, *ez, *bx, *by, *bz;   /* [ny*nx] */
    double *jx, *jy, *jz;                  /* [ny*nx] */
    double *byL, *bzL;                     /* [ny] left boundary values */
} or_fields_t;

/* Particles of one species, structure of arrays, n entries.
 * alive[p] = 1 for a particle in the domain, 0 for a removed one. */
typedef struct {
    long n;
    double *x, *y;              /* cell units */
    double *ux, *uy, *uz;
    double *sx, *sy, *sz;
    double *w;                  /* density per macro-particle [n_c] */
    int *alive;
} or_particles_t;

/* single-particle parts (exposed for the closed-form tests) */
void or_gather(const or_grid_t *g, const or_fields_t *f, double X, double Y,
               double E[3], double B[3]);
void or_boris(double qm, double dt, const double E[3], const double B[3], double u[3]);
void or_omega(double qm, double a, const double ubar[3], const double E[3],
              const double B[3], double Om[3]);
void or_spin_rotate(const double Om[3], double dt, double s[3]);
void or_deposit_one(const or_grid_t *g, or_fields_t *f, double qw,
                    double X0, double Y0, double X1, double Y1, double vz);

/* whole-species parts: a1-a4 (saves old positions and v_z), a5, a6 */
void or_push(const or_grid_t *g, const or_species_t *sp, or_particles_t *p,
             const or_fields_t *f, double *x_old, double *y_old, double *vz);
void or_deposit(const or_grid_t *g, const or_species_t *sp, or_particles_t *p,
                const double *x_old, const double *y_old, const double *vz,
                or_fields_t *f);
void or_field_update(const or_grid_t *g, or_fields_t *f, long step);
void or_laser(const or_grid_t *g, double t, double y, int comp, double *val);

/* one full step over nsp species: push+deposit every mobile species, then fields */
void or_step(const or_grid_t *g, const or_species_t *sp, or_particles_t *p,
             const int *mobile, int nsp, or_fields_t *f, long step);

/* diagnostics */
void or_rho(const or_grid_t *g, const or_species_t *sp, const or_particles_t *p,
            double *rho);
void or_div_e(const or_grid_t *g, const or_fields_t *f, double *div);
void or_div_b(const or_grid_t *g, const or_fields_t *f, double *div);
/* out[0..2] = P (weighted Eq. 4), out[3] = sum w, out[4] = count,
 * out[5] = weighted mean kinetic energy [MeV], out[6] = weighted variance [MeV^2] */
void or_moments(const or_species_t *sp, const or_particles_t *p,
                double emin_mev, double emax_mev, double out[7]);

/* Energy spectra (the dN/dE and dP/dE panels of Figs. 1-3): live particles
 * with kinetic energy in [emin, emax) go to one of nbins bins, equal in
 * energy (log_bins = 0) or in log energy (log_bins = 1, emin > 0);
 * out[5 b + 0..4] = count, sum w, sum w sx, sum w sy, sum w sz of bin b. */
void or_histogram(const or_species_t *sp, const or_particles_t *p, double emin_mev,
                  double emax_mev, int nbins, int log_bins, double *out);

/* ---- 3D3V (pic_oracle3.c) ------------------------------------------------
 * Positions in cell units; mesh arrays [nz][ny][nx]; staggering of [k][j][i]:
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
 *   Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
 * y and z are periodic; x is open (Silver-Mueller, laser at x_min) or periodic.
 * With open x, By and Bz at i = nx-1 hold the right-hand boundary values and
 * byL, bzL ([nz][ny]) the left-hand ones at x = -1/2.  The laser profile is
 * Gaussian in the radius about the box axis (y, z) = (ny dy/2, nz dz/2). */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt;
    int bc_x, pol;
    double a0, w0, tau, t_peak;
} or_grid3_t;

typedef struct {
    double *ex, *ey, *ez, *bx, *by, *bz;   /* [nz*ny*nx] */
    double *jx, *jy, *jz;
    double *byL, *bzL;                     /* [nz*ny] */
} or_fields3_t;

typedef struct {
    long n;
    double *x, *y, *z;
    double *ux, *uy, *uz;
    double *sx, *sy, *sz;
    double *w;
    int *alive;
} or_particles3_t;

void or3_gather(const or_grid3_t *g, const or_fields3_t *f, double X, double Y, double Z,
                double E[3], double B[3]);
void or3_deposit_one(const or_grid3_t *g, or_fields3_t *f, double qw, double X0, double Y0,
                     double Z0, double X1, double Y1, double Z1);
void or3_push(const or_grid3_t *g, const or_species_t *sp, or_particles3_t *p,
              const or_fields3_t *f, double *x_old, double *y_old, double *z_old);
void or3_deposit(const or_grid3_t *g, const or_species_t *sp, or_particles3_t *p,
                 const double *x_old, const double *y_old, const double *z_old, or_fields3_t *f);
void or3_laser(const or_grid3_t *g, double t, double y, double z, int comp, double *val);
void or3_field_update(const or_grid3_t *g, or_fields3_t *f, long step);
void or3_step(const or_grid3_t *g, const or_species_t *sp, or_particles3_t *p, const int *mobile,
              int nsp, or_fields3_t *f, long step);
void or3_rho(const or_grid3_t *g, const or_species_t *sp, const or_particles3_t *p, double *rho);
void or3_div_e(const or_grid3_t *g, const or_fields3_t *f, double *div);
void or3_div_b(const or_grid3_t *g, const or_fields3_t *f, double *div);

#ifdef __cplusplus
}
#endif
#endif
