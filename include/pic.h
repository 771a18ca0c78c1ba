/*
 * pic.h -- C ABI of the GB300 (sm_103a) 2D3V and 3D3V electromagnetic
 * particle-in-cell step with Thomas-BMT spin tracking.
 *
 * The method (Sec. 2 of Huetzen et al., "Simulation of Polarized Beams from
 * Laser-Plasma Accelerators"): particles are pushed in the plasma and laser
 * fields, and each macro-particle carries a classical spin s that precesses
 * by ds/dt = -Omega x s (Eq. 1) with Omega from Eqs. (2)-(3); the beam
 * polarization is the ensemble mean of s (Eq. 4).  The particle-in-cell parts
 * the paper leaves to its PIC code are the standard ones: CIC field gather
 * on the Yee mesh, Boris push, Esirkepov charge-conserving current and Yee
 * FDTD field update.
 *
 * Units (normalised): time 1/omega0, length c/omega0, momentum u = p/(m c),
 * fields m_e c omega0 / e, density n_c, charge e, mass m_e; omega0 = 2 pi c / lambda.
 *
 * Conventions for every entry point:
 *   - the return value is a pic_status_t; nothing throws across the ABI;
 *     pic_last_error() gives a one-line reason for the last failure;
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream); compute calls are asynchronous on it; calls documented as
 *     "synchronous" wait for the stream before returning;
 *   - the context owns all device memory it allocates (cudaMalloc at
 *     pic_create, freed at pic_destroy); host pointers passed in are only
 *     read or written during the call;
 *   - a context is bound to the CUDA device that was current at pic_create;
 *     calls on one context must not overlap (one host thread at a time);
 *   - each compute entry point names the equation, section or published
 *     method it follows (a1-a8 are the steps of one PIC step with spin);
 *     the calls that only configure a context, move state between host and
 *     device, bind memory, report sizes, counters or errors, or replay steps
 *     from CUDA graphs have no counterpart in the paper.
 *
 * Mesh layout (host arrays are row-major [ny][nx] float32).  Element [j][i] of
 *   Ex sits at (i+1/2, j)   Ey at (i, j+1/2)   Ez at (i, j)
 *   Bx at (i, j+1/2)        By at (i+1/2, j)   Bz at (i+1/2, j+1/2)
 *   Jx, Jy, Jz as Ex, Ey, Ez   (node i is at x = i dx).
 * y is periodic.  With PIC_BC_OPEN along x a first-order Silver-Mueller
 * boundary absorbs outgoing waves at both ends and injects the laser at x = 0;
 * By[j][nx-1] and Bz[j][nx-1] (x = nx - 1/2) then hold boundary values, and the
 * left boundary values By(-1/2), Bz(-1/2) are the arrays by_left, bz_left [ny].
 * Particles live in [2, nx-2) along x with open boundaries (a particle that
 * leaves is removed after its current is deposited) and wrap when periodic.
 *
 * 3D3V (pic_config_t.dim = 3): host mesh arrays are [nz][ny][nx]; element
 * [k][j][i] of
 *   Ex sits at (i+1/2, j, k)     Ey at (i, j+1/2, k)     Ez at (i, j, k+1/2)
 *   Bx at (i, j+1/2, k+1/2)      By at (i+1/2, j, k+1/2) Bz at (i+1/2, j+1/2, k)
 * y and z are periodic; by_left, bz_left are [nz][ny] (at x = -1/2, the y and
 * z positions of By and Bz); particles carry iz, oz as well.  The laser
 * profile is Gaussian in the radius about the box axis (ny dy / 2, nz dz / 2).
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = -1,      /* invalid argument or configuration; nothing was done   */
    PIC_ERR_CUDA = -2,     /* a CUDA call failed (out of memory, launch failure...) */
    PIC_ERR_NAN = -3,      /* a kernel produced a non-finite momentum or spin       */
    PIC_ERR_CFL = -4,      /* a particle moved a cell or more in one step           */
    PIC_ERR_OVERFLOW = -5, /* more particles than the species capacity              */
    PIC_ERR_TIMEOUT = -6,  /* a bounded device-side wait gave up (tile staging)     */
    PIC_ERR_STATE = -7     /* call not valid in the context's current state         */
} pic_status_t;

#define PIC_MAX_SPECIES 4
#define PIC_BC_OPEN 0
#define PIC_BC_PERIODIC 1
#define PIC_POL_NONE 0
#define PIC_POL_LP_Y 1 /* linear, E along y                         */
#define PIC_POL_CP 2   /* circular, a0/sqrt(2) in each of Ey and Ez */

typedef struct {
    double q;            /* charge [e]                                  */
    double m;            /* mass [m_e]                                  */
    double a;            /* gyromagnetic anomaly (Eq. 3): e 0.00116, p 1.793 */
    int mobile;          /* 0: never pushed (contributes only to rho)   */
    int64_t capacity;    /* device slots reserved for this species      */
} pic_species_t;

typedef struct {
    int nx, ny;                  /* cells; nx >= 8, ny >= 4, both <= 32767        */
    double dx_lambda, dy_lambda; /* cell size in laser wavelengths                 */
    double cfl;                  /* dt = cfl / sqrt(1/dx^2 + 1/dy^2), 0 < cfl < 1  */
    int bc_x;                    /* PIC_BC_OPEN or PIC_BC_PERIODIC                 */
    int pol;                     /* PIC_POL_*, used with PIC_BC_OPEN               */
    double a0;                   /* peak normalised amplitude e A / (m_e c)        */
    double waist_lambda;         /* 1/e field radius at x = 0 [lambda]             */
    double fwhm_periods;         /* FWHM of the intensity [laser periods]          */
    double t_peak_periods;       /* time of the envelope peak at x = 0 [periods]   */
    int nspecies;                /* 1 .. PIC_MAX_SPECIES                           */
    pic_species_t sp[PIC_MAX_SPECIES];
    int sort_every;              /* steps between tile sorts in pic_step (0: 32)   */
    int tile_x, tile_y;          /* cells per tile: 8x4, 16x8, 32x8, 32x16 or 64x16 (0, 0: chosen
                                    from the mesh size: 32x8 from 2^19 cells, 16x8
                                    from 77,824 (4 tiles per SM), else 8x4)         */
    int precision;               /* arithmetic of particles and mesh: 32 (the
                                    production path) or 64 (the FP64 instantiation
                                    of the same kernels); 0 means 32.  Reductions
                                    are FP64 in both.                              */
    int dim;                     /* 2 (or 0): 2D3V; 3: 3D3V                        */
    int nz;                      /* 3D3V: cells along z, 4 <= nz <= 1020; nx, ny <= 2044;
                                    the mesh padded to whole tiles holds at most
                                    2^31 - 1 cells (the tile sort's cell index)    */
    double dz_lambda;            /* 3D3V: cell size along z [lambda]; then
                                    dt = cfl / sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)      */
    int tile_z;                  /* 3D3V tiles (tile_x, tile_y, tile_z): 16x4x4,
                                    8x8x4, 8x4x4, 16x8x4 or 32x4x4 (0, 0, 0: 16x4x4) */
    int bin_headroom_pct;        /* 3D3V binned layout (0: off).  Each tile owns a
                                    slot range of count + max(bin_min_extra,
                                    count * pct / 100) slots (rounded up to 8), and
                                    every step writes each particle into the range
                                    of the tile its new cell lies in, in the other
                                    particle buffer, so particles never drift out
                                    of their tile between sorts.  A range that
                                    fills spills into one shared overflow range;
                                    the tile sort (every sort_every steps, and
                                    early once the overflow range is past half
                                    full) re-sizes the ranges; particles that
                                    find the overflow range full too are lost
                                    and the next synchronising call returns
                                    PIC_ERR_OVERFLOW.  The host keeps at most 4
                                    binned steps in flight (before each it
                                    waits for the one 4 steps back), so the
                                    half-full alert acts within 4 steps
                                    however far ahead the caller queues.
                                    Mobile species need
                                    capacity >= n (1 + pct / 100) + ntiles
                                    (bin_min_extra + 7) + max(1024, n / 4);
                                    otherwise the compact layout is kept.       */
    int bin_min_extra;           /* spare slots each tile range keeps at least  */
} pic_config_t;

/* Host-side particle arrays of one species (n entries each).  ix, iy are cell
 * indices and ox, oy in [0, 1) the offsets inside the cell (x = (ix + ox) dx). */
typedef struct {
    int64_t n;
    int32_t *ix, *iy;
    float *ox, *oy;
    float *ux, *uy, *uz;  /* u = p / (m c) */
    float *sx, *sy, *sz;  /* spin          */
    float *w;             /* density carried by the macro-particle [n_c] */
    int32_t *id;          /* caller's particle identity, carried through sorts */
    int32_t *iz;          /* 3D3V only (ignored in 2D3V): cell index and offset along z */
    float *oz;
} pic_particles_t;

/* The same with float64 arrays (read-back of either precision at full width). */
typedef struct {
    int64_t n;
    int32_t *ix, *iy;
    double *ox, *oy;
    double *ux, *uy, *uz;
    double *sx, *sy, *sz;
    double *w;
    int32_t *id;
    int32_t *iz;
    double *oz;
} pic_particles_f64_t;

/* Host-side mesh arrays, [ny][nx] float32 each (by_left, bz_left: [ny]); in
 * 3D3V [nz][ny][nx] (by_left, bz_left: [nz][ny]).
 * A NULL member is skipped by pic_set_fields / pic_get_fields. */
typedef struct {
    float *ex, *ey, *ez, *bx, *by, *bz, *jx, *jy, *jz;
    float *by_left, *bz_left;
} pic_fields_t;

typedef struct {
    double *ex, *ey, *ez, *bx, *by, *bz, *jx, *jy, *jz;
    double *by_left, *bz_left;
} pic_fields_f64_t;

/* Moments of Eq. (4) over the live particles of one species whose kinetic
 * energy (gamma - 1) m c^2 lies in [emin, emax) MeV, accumulated in FP64. */
typedef struct {
    double P[3];       /* sum w s / sum w  (Eq. 4; equal weights give (1/N) sum s) */
    double sum_w;
    double count;
    double ekin_mean;  /* weighted mean kinetic energy [MeV]   */
    double ekin_var;   /* weighted variance [MeV^2]             */
} pic_moments_t;

/* Host-only check of a configuration (no CUDA call).  PIC_OK or PIC_ERR_ARG. */
pic_status_t pic_validate_config(const pic_config_t *cfg);

/* Creates a context on the current device: allocates the mesh and particle
 * storage, zero fields, no particles, step index 0.  Synchronous. */
pic_status_t pic_create(const pic_config_t *cfg, void *stream, void **ctx_out);

/* Releases everything the context owns.  NULL is accepted. */
void pic_destroy(void *ctx);

/* Time step dt [1/omega0] and cell sizes dx, dy, dz [c/omega0] the context
 * derived (dz = 0 in 2D3V).  NULL outputs are skipped. */
pic_status_t pic_get_grid(void *ctx, double *dt, double *dx, double *dy, double *dz);

/* Loads the particles of one species from host float32 arrays (widened
 * exactly with precision 64; replacing what was there) and sorts them by tile.  n <= capacity (else PIC_ERR_OVERFLOW).
 * Cells must lie in the particle region (else PIC_ERR_ARG).  Synchronous.
 * When every array is pinned (page-locked, device-mapped) host memory, one
 * kernel reads them in place over the host link and writes the particle
 * buffer, cells packed on the way; other arrays are copied (cudaMemcpyAsync)
 * and packed on the device.  Both give the same state. */
pic_status_t pic_set_particles(void *ctx, int species, const pic_particles_t *p, void *stream);

/* The same from float64 host arrays (exact with precision 64; rounded to
 * float with precision 32). */
pic_status_t pic_set_particles_f64(void *ctx, int s, const pic_particles_f64_t *p, void *stream);

/* Number of particle slots of one species (live and removed since the last
 * sort; in the binned 3D3V layout the span of the tile ranges and the
 * overflow range, whose spare slots hold no particle).  An upper bound for
 * the room pic_get_particles needs.  Synchronises the legacy default stream. */
pic_status_t pic_get_count(void *ctx, int species, int64_t *n);

/* Copies every slot into caller arrays with room for out->n entries (set
 * out->n to that room; PIC_ERR_ARG if the slots do not fit); on return out->n
 * is the slot count.  A removed particle has ix = iy = -1.  A species in the
 * binned 3D3V layout is first sorted into the compact layout (the next step
 * re-bins), so out->n may be below pic_get_count.  Returns the device error
 * flags the steps before left (PIC_ERR_OVERFLOW if a binned step lost
 * particles, PIC_ERR_NAN, ...).  Synchronous.
 * With precision 64 the values are rounded to float32; pic_get_particles_f64
 * returns them at full width (and widens float32 state exactly). */
pic_status_t pic_get_particles(void *ctx, int species, pic_particles_t *out, void *stream);
pic_status_t pic_get_particles_f64(void *ctx, int species, pic_particles_f64_t *out, void *stream);

/* Mesh arrays host <-> device (float32 host arrays for either precision;
 * pic_get_fields_f64 reads back at full width).  Synchronous. */
pic_status_t pic_set_fields(void *ctx, const pic_fields_t *f, void *stream);
pic_status_t pic_get_fields(void *ctx, pic_fields_t *f, void *stream);
pic_status_t pic_get_fields_f64(void *ctx, pic_fields_f64_t *f, void *stream);

/* Step index n (the fields are at t = n dt; the laser phase follows it). */
pic_status_t pic_set_step(void *ctx, int64_t step);
pic_status_t pic_get_step(void *ctx, int64_t *step);

/* a1-a4 for every mobile species: CIC gather of E^n, B^n at x^n, Boris push
 * u^{n-1/2} -> u^{n+1/2}, spin rotation s^{n-1/2} -> s^{n+1/2} by
 * ds/dt = -Omega x s with Omega of Eqs. (2)-(3) at the mean momentum,
 * x^{n+1} = x^n + dt u/gamma.  Keeps x^n and v_z for pic_deposit. */
pic_status_t pic_gather_push_spin(void *ctx, void *stream);

/* a5: adds the Esirkepov current J^{n+1/2} of the move made by the last
 * pic_gather_push_spin (PIC_ERR_STATE if none is pending); removes particles
 * that left the region.  J must hold what the caller wants added to (it is
 * zero after pic_create and after every field update). */
pic_status_t pic_deposit(void *ctx, void *stream);

/* a6: B^{n+1/2} = B^n - dt/2 curl E^n; boundary values at t^{n+1/2};
 * E^{n+1} = E^n + dt (curl B^{n+1/2} - J); B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1};
 * then J = 0 and n += 1. */
pic_status_t pic_field_update(void *ctx, void *stream);

/* a7: counting sort of every species by tile (drops removed particles). */
pic_status_t pic_sort(void *ctx, void *stream);

/* a1-a5 in one kernel: per tile, the field window is staged into shared
 * memory by TMA and the current is accumulated there before being added to
 * J.  Same result as pic_gather_push_spin + pic_deposit up to float rounding
 * order of the current sums. */
pic_status_t pic_push_deposit(void *ctx, void *stream);

/* nsteps whole steps: pic_sort when sort_every steps have passed since the
 * last sort (counted across calls), then pic_push_deposit and
 * pic_field_update.  No host synchronisation.
 * In the compact layout each sort-free stretch of 2 or more steps (at most
 * the pic_set_graphs limit, 32 by default) is replayed from a CUDA graph of
 * its steps, captured at the first stretch of its length, diagnostic phase
 * and buffer parity on a stream the context owns (ordered after and before
 * `stream` by events): the same kernels with the same arguments as launched
 * steps, one graph launch in place of 5-7 kernel launches a step.  The
 * binned 3D3V layout launches its steps one by one (it decides between steps,
 * on the host, whether to re-bin). */
pic_status_t pic_step(void *ctx, int nsteps, void *stream);

/* Longest stretch pic_step replays as one CUDA graph (0: launch every kernel,
 * 1 .. 4096).  Drops the graphs captured so far. */
pic_status_t pic_set_graphs(void *ctx, int max_steps);

/* Graphs pic_step has captured and replayed on this context (a capture runs
 * its stretch once; a replay re-runs a captured stretch). */
pic_status_t pic_graph_stats(void *ctx, int64_t *captures, int64_t *replays);

/* a8 inside the step: every `every` steps (0 turns it off) pic_push_deposit,
 * and so pic_step, also accumulates the Eq. (4) moments of every species over
 * the particles it has just moved (u, s at n+1/2, x at n+1; live particles
 * whose kinetic energy lies in [emin[s], emax[s]) MeV; NULL arrays mean no
 * window).  The sums are float per thread over a few particles, FP64 per CTA
 * and across CTAs; the variance is taken about the previous diagnostic's
 * mean.  No extra pass over the particles and no host synchronisation. */
pic_status_t pic_set_diagnostics(void *ctx, int every, const double *emin_mev, const double *emax_mev);

/* The moments of the last in-step diagnostic (out[nspecies]) and the step
 * index they belong to (-1 if none yet).  Synchronous. */
pic_status_t pic_get_diagnostics(void *ctx, pic_moments_t *out, int64_t *step, void *stream);

/* a8: Eq. (4) moments of one species in an energy window.  Synchronous;
 * also reports device-side error flags (PIC_ERR_NAN, PIC_ERR_TIMEOUT). */
pic_status_t pic_polarization(void *ctx, int species, double emin_mev, double emax_mev,
                              pic_moments_t *out, void *stream);

/* Energy spectra of one species (the dN/dE and dP/dE panels of Figs. 1-3):
 * live particles with kinetic energy in [emin, emax) MeV go to one of nbins
 * bins (1 <= nbins <= PIC_MAX_HIST_BINS), equal in energy (log_bins = 0) or
 * in log energy (log_bins != 0, emin > 0).  out[5 b + 0..4] (host) = count,
 * sum w, sum w sx, sum w sy, sum w sz of bin b; dN/dE = sum w / bin width and
 * dP/dE = (sum w s) / (sum w) per bin (Eq. 4 over the bin).  Per-block float
 * sums, FP64 across blocks.  Synchronous. */
#define PIC_MAX_HIST_BINS 1024
pic_status_t pic_energy_histogram(void *ctx, int species, double emin_mev, double emax_mev, int nbins,
                                  int log_bins, double *out, void *stream);

/* Sets the immobile background charge to minus the CIC charge density of
 * the current particles (a neutral start).  Asynchronous. */
pic_status_t pic_capture_background(void *ctx, void *stream);

/* Charge-conservation residual div E - rho - rho_background on the nodes
 * i in [3, nx-4] (open x) or all nodes (periodic): out[0] = max |r|,
 * out[1] = sqrt(sum r^2 / count), FP64.  Synchronous. */
pic_status_t pic_gauss_residual(void *ctx, double out[2], void *stream);

/* Co-moving window (Sec. 2: the box follows the laser through the plasma):
 * moves the box ncells cells along +x between two steps.  In box coordinates
 * every mesh array slides ncells columns toward x = 0 (the columns that leave
 * are dropped; the uncovered ones at x_max start at zero), the left boundary
 * values By(-1/2), Bz(-1/2) become those of the old column ncells - 1, every
 * particle moves by -ncells cells and those whose cell falls below x = 2 are
 * removed.  inject is NULL or an array of nspecies host particle sets (same
 * layout as pic_set_particles) holding the plasma of the uncovered columns,
 * normally cells [nx - 2 - ncells, nx - 2) in the moved box; after
 * pic_capture_background their immobile ions join the background.
 * A species in the binned 3D3V layout, with ncells a multiple of the tile
 * width along x, stays binned: its tile ranges are relabelled by whole tile
 * columns (the ranges of the columns that left take the uncovered ones) and
 * the plasma goes into its tiles' ranges; a range that is full passes the
 * rest to the overflow range, and when that fills too particles are lost and
 * PIC_ERR_OVERFLOW is returned.  Every other species takes the compact path:
 * the plasma is appended after its slots (PIC_ERR_OVERFLOW, and nothing
 * changed, if its capacity would be exceeded) and the species is sorted.
 * Needs PIC_BC_OPEN and 1 <= ncells <= nx - 8; the laser source keeps its
 * time profile at the new x = 0.  Synchronous.  The step index is unchanged. */
pic_status_t pic_shift_window(void *ctx, int ncells, const pic_particles_t *inject, void *stream);

/* The co-moving window on the stepping path.  With it on, pic_step makes the
 * move pic_shift_window describes before the step from index n whenever
 *     n >= start_step  and  moved + ncells <= floor((n - start_step) dt speed / dx),
 * moved being the cells the window has moved since this call: the box
 * follows a front that leaves at step start_step with speed `speed` (units of
 * c), lagging it by less than ncells cells.  Each move takes the oldest
 * plasma staged with pic_stage_injection (none staged: vacuum enters) and
 * runs on the device without host synchronisation; a plasma that does not
 * fit is reported by the next synchronising call (PIC_ERR_OVERFLOW).  In the
 * binned 3D3V layout choose ncells a multiple of the tile width along x:
 * other moves sort every species.  ncells = 0 switches the window off;
 * otherwise 1 <= ncells <= nx - 8, speed > 0 and finite, PIC_BC_OPEN (else
 * PIC_ERR_ARG).  pic_push_deposit and pic_field_update never move it. */
pic_status_t pic_set_window(void *ctx, int ncells, int64_t start_step, double speed);

/* Stages the plasma of one future move: inject = nspecies host particle sets
 * (layout of pic_set_particles, cells of the moved box, normally
 * [nx - 2 - ncells, nx - 2)), copied to device memory the context owns and
 * queued behind the ones staged before; the moves of pic_step consume them
 * in order.  Cells outside the particle region give PIC_ERR_ARG, a set larger
 * than the species capacity PIC_ERR_OVERFLOW; nothing is queued then.
 * Synchronous: the host arrays may be reused on return. */
pic_status_t pic_stage_injection(void *ctx, const pic_particles_t *inject, void *stream);

/* Staged plasmas not yet consumed by a move. */
pic_status_t pic_staged_injections(void *ctx, int64_t *count);

/* *binned = 1 when species s is in the binned 3D3V layout now, else 0 (the
 * compact layout: the binned layout is off, the species is immobile, or its
 * capacity cannot hold the binned ranges of its live-particle bound, which
 * counts every particle staged into it since the last completed count). */
pic_status_t pic_get_layout(void *ctx, int species, int *binned);

/* Caller-owned device memory for a context's state (e.g. torch tensors,
 * which then are the state, with no copy).  Per species the two particle
 * buffers the steps and sorts
 * alternate between: the cell words (0xFFFFFFFF = removed), the record
 * arrays in the context's real type (float for precision 32, double for 64;
 * oz in 3D3V only) and the ids, each of at least `capacity` entries; and the
 * mesh: eb = E then B, [6][nz][ny][ld] reals, j = [3][nz][ny][ld] reals (nz = 1
 * in 2D3V; ld and the sizes from pic_buffer_sizes).  A NULL member keeps the
 * context's own array. */
typedef struct {
    uint32_t *cell;
    void *ox, *oy, *oz, *ux, *uy, *uz, *sx, *sy, *sz, *w;
    int32_t *id;
} pic_particle_buffer_t;

typedef struct {
    pic_particle_buffer_t sp[PIC_MAX_SPECIES][2];
    void *eb;
    void *j;
} pic_buffers_t;

/* Sizes a caller needs to allocate pic_buffers_t memory: the mesh row pitch
 * ld (reals; >= nx), the reals of one mesh component (plane = ld ny nz), the
 * bytes of one real (4 or 8), and each species' capacity (slots of every
 * particle array; unused entries 0). */
pic_status_t pic_buffer_sizes(void *ctx, int64_t *ld, int64_t *plane, int *real_bytes,
                              int64_t capacity[PIC_MAX_SPECIES]);

/* Moves the context's state into the caller's memory: each non-NULL member of
 * b receives a copy of the array it replaces, the context frees its own and
 * uses the caller's from then on (the caller keeps ownership: the memory must
 * stay allocated, on the context's device, until pic_destroy).  Every pointer
 * must be device (or managed) memory of the context's device, 16-byte aligned,
 * and no two arrays of the context (bound, or its own) may share a byte once
 * bound (else PIC_ERR_ARG and nothing changes); sizes are the caller's
 * responsibility.  Captured step graphs are dropped and the field window's
 * tensor map is re-encoded.  Synchronous. */
pic_status_t pic_bind_buffers(void *ctx, const pic_buffers_t *b, void *stream);

/* Which of species s's two particle buffers holds its particles now (0 or 1;
 * the other is scratch for the next step or sort). */
pic_status_t pic_current_buffer(void *ctx, int species, int *which);

/* Cells the window has moved since pic_create. */
pic_status_t pic_get_window(void *ctx, int64_t *offset_cells);

/* Waits for the stream and reports device-side error flags. */
pic_status_t pic_sync(void *ctx, void *stream);

/* Number of CUDA kernels this context has launched so far (host counter). */
pic_status_t pic_launch_count(void *ctx, int64_t *count);

/* Eq. (4) moments, as pic_polarization computes them for precision 32, of n
 * particles held in caller-owned device arrays (the layout of the library's
 * own float32 buffers: cell
 * words with 0xFFFFFFFF marking a removed particle, float32 u, s and w), for
 * a species of mass mass_me [m_e] and the kinetic-energy window [emin, emax)
 * MeV.  The result is written to the caller's device memory *out_dev.
 *
 * This entry point allocates no device memory: it is meant for callers that
 * cannot, e.g. code being captured into a CUDA graph, callers whose device
 * memory all comes from their own pool, or loops that cannot afford the
 * device-wide synchronisation of cudaMalloc.  The reduction's per-block
 * partial sums live in one fixed array of about 29 KB that the library
 * declares at file scope; every GPU that loads the library holds it until the
 * process exits.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (every slot is rewritten before it is read, so nothing needs clearing);
 * calls that overlap on the GPU (different streams, or different host
 * threads) race on it and must be ordered by the caller.
 *
 * n must be in [0, PIC_NOALLOC_MAX_PARTICLES] (else PIC_ERR_ARG, with the
 * reason in pic_last_error(NULL); the reduction's loops index with 64 bits, so
 * every n up to that limit is safe); the pointers must be device pointers of
 * the current device.  Asynchronous on `stream`.  No counterpart in the
 * paper: this is an interface variant, not part of the method. */
#define PIC_NOALLOC_MAX_PARTICLES 2147483647LL
pic_status_t pic_moments_noalloc(int64_t n, const uint32_t *cell, const float *ux, const float *uy,
                                 const float *uz, const float *sx, const float *sy, const float *sz,
                                 const float *w, double mass_me, double emin_mev, double emax_mev,
                                 pic_moments_t *out_dev, void *stream);

/* Reason for the last failure on this context (or of pic_create when ctx is NULL). */
const char *pic_last_error(void *ctx);

/* ---- adjoint (2D3V) ----------------------------------------------------------
 * Loss on the final state: over the live particles of one species,
 *   L = sum_i a_i s_i / sum_i a_i,   a_i = w_i e_i sig((e_i - e_cut) / e_width),
 * e_i the kinetic energy [MeV], s_i the spin component `axis`, sig the
 * logistic function: the polarization (Eq. 4) of the energetic part of the
 * beam, weighted by energy. */
typedef struct {
    int species;
    int axis;             /* 0: x, 1: y, 2: z */
    double e_cut_mev;
    double e_width_mev;   /* > 0 */
} pic_loss_t;

/* L of the current state.  Synchronous. */
pic_status_t pic_loss(void *ctx, const pic_loss_t *loss, double *value, void *stream);

/* Runs nsteps steps forward from the current state (fused kernel in FP32,
 * split kernels in FP64; no tile sorts: every slot keeps its particle, no
 * in-step diagnostics) keeping a checkpoint every
 * checkpoint_every steps, evaluates L at the end, and back-propagates: each
 * stretch is recomputed from its checkpoint with every state stored, and the
 * adjoint of every step (the transposes of the Yee stages and the
 * vector-Jacobian products of gather, push, spin, advance and deposit) runs
 * back through it.  Out: L, dL/da0 (laser amplitude); the gradients with
 * respect to each particle's initial state and weight are kept for
 * pic_adjoint_particle_grads.  The context ends in the final forward state.
 * Device memory: (ceil(nsteps / checkpoint_every) + checkpoint_every + 1)
 * copies of the particle state and E, B.  Synchronous.  2D3V only. */
pic_status_t pic_adjoint(void *ctx, int nsteps, int checkpoint_every, const pic_loss_t *loss, double *loss_value,
                         double *dloss_da0, void *stream);

/* Gradients of the last pic_adjoint with respect to the initial state of the
 * slots of species s: ox, oy <- dL/d(offset) (per cell), ux, uy, uz <- dL/du,
 * sx, sy, sz <- dL/ds, w <- dL/dw; ix, iy, id <- the slot's initial cell and
 * identity.  out->n >= the slot count (set to it).  Synchronous. */
pic_status_t pic_adjoint_particle_grads(void *ctx, int s, pic_particles_f64_t *out, void *stream);

/* ---- batches of independent 2D3V runs --------------------------------------
 * A parameter scan (density, a0, mesh size, particles per cell, run length)
 * advanced together: each batch step is one launch of a persistent fused
 * kernel that takes (run, tile) items of every active run from one queue, the
 * batched Yee update over every (run, row), and a step-counter advance; the
 * stretches between tile sorts are captured once as CUDA graphs and replayed.
 * Runs share the tile shape and the sort cadence (taken from cfgs[0], or
 * chosen by pic_batch_tune) and must be 2D3V in precision 32. */

/* Creates nruns contexts (cfgs[r], as pic_create) and the batch around them;
 * run r takes nsteps[r] batch steps, then stays idle.  Synchronous. */
pic_status_t pic_batch_create(const pic_config_t *cfgs, int nruns, const int64_t *nsteps, void *stream,
                              void **batch);
/* Releases the batch and its runs' contexts.  NULL is accepted. */
void pic_batch_destroy(void *batch);
/* The context of run r (owned by the batch): load particles and fields, read
 * results with the single-run calls (pic_set_particles, pic_polarization,
 * pic_get_fields, ...).  Do not call pic_destroy on it. */
pic_status_t pic_batch_run(void *batch, int r, void **ctx);
/* Advances every run that has steps left by up to nsteps steps.  Synchronous
 * at the end (checks every run's error flags). */
pic_status_t pic_batch_step(void *batch, int64_t nsteps, void *stream);
/* done[r] = batch steps run r has taken ([nruns]). */
pic_status_t pic_batch_steps_done(void *batch, int64_t *done);
/* Autotuner: for every candidate tile shape (tiles[2k], tiles[2k+1]) and sort
 * cadence sorts[q] it re-tiles the runs, takes one sort cycle of steps and
 * times probe_steps steps (the steps count toward the runs), then keeps the
 * fastest pair: chosen = {tile_x, tile_y, sort_every}.  Synchronous. */
pic_status_t pic_batch_tune(void *batch, int probe_steps, const int *tiles, int ntiles, const int *sorts,
                            int nsorts, int *chosen, void *stream);
/* Kernels launched for the batch and its runs so far. */
pic_status_t pic_batch_launch_count(void *batch, int64_t *count);
/* One-line reason for the last failure of a batch call (NULL: of pic_batch_create). */
const char *pic_batch_last_error(void *batch);

#ifdef __cplusplus
}
#endif
#endif
