// pic_kernels.h -- launchers of the CUDA kernels, called by the C ABI layer.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "pic_device.cuh"
#include "pic_device3.cuh"

// device-side copy of pic_moments_t (same layout: seven doubles)
struct pic_moments_dev {
    double P[3];
    double sum_w, count, ekin_mean, ekin_var;
};

struct LaserParams {
    int pol;            // 0 none, 1 LP-y, 2 CP
    double a0, w0, tau, t_peak, yc, dy;
};

// batched step of many 2D3V runs (pic_batch.cu): the work queue of the
// persistent fused kernel
template <typename R>
struct BatchFused {
    const StepParams<R> *params;   // [nruns]
    const CUtensorMap *tmaps;      // [nruns], 64-byte aligned
    const int2 *work;              // [nwork] (run, tile)
    int nwork;
    int *counter;                  // queue head, zero before the launch
    const long long *step, *nsteps;  // [nruns]: items of runs with step >= nsteps are skipped
};

// per-run field data of a batch: mesh, left boundary values, laser profile,
// laser time factors (fz, fy) of steps step0, step0 + 1, ..., r = dt/dx, q = dt/dy
template <typename R>
struct BatchField {
    MeshParams<R> m;
    R *bnd;
    const double *prof;
    const double *laser;
    long long step0;
    double r, q;
};
template <typename R>
cudaError_t launch_field_update_batch(const BatchField<R> *runs, const int2 *rows, int nrows, long long *step,
                                      const long long *nsteps, int nruns, int *counter, cudaStream_t st);

// k_particles.cu
bool fused_tile_supported(int tx, int ty);
template <typename R>
cudaError_t launch_step_fused_batch(const BatchFused<R> &W, int tx, int ty, int ctas, cudaStream_t st);
int fused_batch_occupancy(int tx, int ty);
template <typename R>
cudaError_t launch_step_fused(const StepParams<R> &P, const CUtensorMap &tmapEB, cudaStream_t st);
template <typename R>
cudaError_t launch_push_split(const StepParams<R> &P, int s, int n_upper, cudaStream_t st);
template <typename R>
cudaError_t launch_deposit_split(const StepParams<R> &P, int s, int n_upper, cudaStream_t st);

// k_fields.cu
template <typename R>
cudaError_t launch_field_update(const MeshParams<R> &m, R *bnd, const double *prof, const LaserParams &L,
                                double dt, double dx, double dy, long long step, cudaStream_t st,
                                const double *lf_dev = nullptr);
void laser_profile(const LaserParams &L, int ny, double *host);
void laser_time_factors(const LaserParams &L, double t, double *fz, double *fy);

// k_particles3.cu, k_fields3.cu (3D3V)
bool fused3_tile_supported(int tx, int ty, int tz);

template <typename R>
cudaError_t launch_step_fused3(const StepParams3<R> &P, const CUtensorMap &tmapEB, bool binned, cudaStream_t st);
template <typename R>
cudaError_t launch_push_split3(const StepParams3<R> &P, int s, int n_upper, cudaStream_t st);
template <typename R>
cudaError_t launch_deposit_split3(const StepParams3<R> &P, int s, int n_upper, cudaStream_t st);
template <typename R>
cudaError_t launch_field_update3(const MeshParams3<R> &m, R *bnd, const double *prof, const LaserParams &L,
                                 double dt, double dx, double dy, double dz, long long step, cudaStream_t st,
                                 const double *lf_dev = nullptr);
void laser_profile3(const LaserParams &L, int ny, int nz, double dz, double *host);

// k_sort.cu
// the arrays of one particle buffer a sort (or a window move) reads or
// writes: the cell word, the reals of a record (2D3V: ox oy ux uy uz sx sy sz
// w; 3D3V: ox oy oz ux uy uz sx sy sz w) and the id; n the device count
template <typename R>
struct SortArrays {
    uint32_t *cell;
    R *f[10];
    int32_t *id;
    const int32_t *n;
};
// host particle arrays a kernel reads in place (device-mapped pointers),
// records in SortArrays order
template <typename HostT>
struct UploadSrc {
    const int32_t *ix, *iy, *iz, *id;
    const HostT *f[10];
};
template <typename HostT, typename R>
cudaError_t launch_upload(const UploadSrc<HostT> &src, const SortArrays<R> &dst, int n, int xlo, int xhi, int ny,
                          int nz, bool d3, unsigned *err, cudaStream_t st);
// per-tile layout record of a sort (k_layout): the full layers' depth, the
// tile's particle count, the size and start of the tail's rest, the starts
// of the tail's depth layers
constexpr int kTileInfo = 8;
struct SortScratch {
    int32_t *cell_count, *cell_off;  // [ntiles * cells per tile]
    int32_t *tile_info;              // [ntiles * kTileInfo]
    int32_t *tile_total;             // [ntiles + 1]
    int32_t *cursor;                 // [ntiles] scan scratch
    int32_t *rank;                   // [n]
};
// Binned 3D3V layout written by a sort (cnt_to == nullptr: compact layout).
// Range T of tile T gets count + max(extra, count * pct / 100) slots rounded
// up to 8; range ntiles (the overflow range) gets ovf_cap.  tile_start then
// needs ntiles + 2 entries.
struct BinSort {
    int pct = 0, extra = 0, ovf_cap = 0;
    int32_t *cnt_to = nullptr;    // [4 (ntiles + 1)] range counters (Bin3) of the sorted buffer
    int32_t *cnt_from = nullptr;  // [4 (ntiles + 1)] of the source buffer, cleared
    // The source is the layout of the previous sort (its slots unchanged
    // since, particles moved only within them): its tile ranges (relabelled
    // by txo in the binned layout) hold that tile's particles, but for those
    // that drifted, so each tile is gathered by one CTA through shared memory
    // and its new range written in order; old_start ([ntiles + 2] scratch)
    // keeps the source ranges.  src_binned: a sealed binned source, whose
    // overflow range is scattered after the tiles.
    bool src_ordered = false, src_binned = false;
    int txo = 0;
    int32_t *old_start = nullptr;
};
// seal of the binned layout: slots outside each range's two segments ->
// PIC_DEAD, and the other buffer's range counters cleared
struct SealSpecies {
    uint32_t *cell;
    const int32_t *tile_start;
    int32_t *cnt_new;
    int32_t *cnt_zero;
};
struct SealArgs {
    SealSpecies sp[PIC_MAXSP];
    int nsp, nranges;
    bool fill = true;      // write PIC_DEAD into the slots outside the segments
    bool counters = true;  // arrival bases of cnt_new, cnt_zero cleared
    // with counters: set to 1 when an overflow range holds more than half its
    // slots (host-mapped memory the next step reads to re-bin in time)
    volatile int *ovf_alert = nullptr;
};
cudaError_t launch_seal_bins(const SealArgs &a, cudaStream_t st);
cudaError_t launch_pack_cells(const int32_t *ix, const int32_t *iy, uint32_t *cell, int n,
                              int xlo, int xhi, int ny, unsigned *err, cudaStream_t st);
cudaError_t launch_unpack_cells(const uint32_t *cell, int32_t *ix, int32_t *iy, int n,
                                cudaStream_t st);
template <typename R>
cudaError_t launch_tile_sort(const DevSpecies<R> &src, const DevSpecies<R> &dst, const TileGeom &t,
                             const SortScratch &w, int32_t *tile_start, int32_t *n_tmp, int n_upper,
                             const BinSort &order, cudaStream_t st);
cudaError_t launch_pack_cells3(const int32_t *ix, const int32_t *iy, const int32_t *iz, uint32_t *cell, int n,
                               int xlo, int xhi, int ny, int nz, unsigned *err, cudaStream_t st);
cudaError_t launch_unpack_cells3(const uint32_t *cell, int32_t *ix, int32_t *iy, int32_t *iz, int n,
                                 cudaStream_t st);
template <typename R>
cudaError_t launch_tile_sort3(const DevSpecies3<R> &src, const DevSpecies3<R> &dst, const TileGeom3 &t,
                              const SortScratch &w, int32_t *tile_start, int32_t *n_tmp, int n_upper,
                              const BinSort &bins, cudaStream_t st);
template <typename R>
cudaError_t launch_shift_rows(const R *src, R *dst, size_t rows, int nx, int ld, int n, cudaStream_t st);
template <typename R>
cudaError_t launch_ghost_from_column(const R *by, const R *bz, R *bnd, size_t rows, int ld, int n, cudaStream_t st);
cudaError_t launch_shift_cells(uint32_t *cell, const int32_t *n_src, int n_upper, int ncells, bool d3,
                               cudaStream_t st);
// co-moving window on the stepping path: every mesh component moved n
// columns toward x_min in place (rows of ld reals, nx used), the left
// boundary values taken from the old column n - 1 of plane[by], plane[bz]
template <typename R>
struct WindowRows {
    R *plane[10];
    int nplanes;
    int by, bz;  // indices of By, Bz in plane[] (-1: none)
    R *bnd;      // [2][rows] By(-1/2), Bz(-1/2)
    size_t rows;
    int nx, ld, n;
};
template <typename R>
cudaError_t launch_window_rows(const WindowRows<R> &a, cudaStream_t st);
// binned layout: the ranges of the last kt tile columns emptied (txo: the
// column relabelling after the move)
cudaError_t launch_window_vacate(int32_t *cnt, int nr, int ntx, int nyz, int kt, int txo, cudaStream_t st);
// binned layout: staged particles (*src.n of them, at most m_upper) into their
// tiles' ranges of the buffer dst, range counters cnt
template <typename R>
cudaError_t launch_window_inject3(const SortArrays<R> &src, int m_upper, const SortArrays<R> &dst,
                                  const int32_t *tile_start, int32_t *cnt, const TileGeom3 &t, int txo,
                                  unsigned *err, cudaStream_t st);
// compact layout: staged particles appended after the *n_dst slots in use
// (PIC_EF_CAP and nothing appended when they do not fit cap)
template <typename R>
cudaError_t launch_window_append(const SortArrays<R> &src, int m_upper, const SortArrays<R> &dst, int32_t *n_dst,
                                 int cap, bool d3, unsigned *err, cudaStream_t st);
// live particles into host-mapped memory: *n_dev (tile_start == nullptr,
// the compact layout) or the sum of the nr binned ranges' lengths
cudaError_t launch_live_sample(const int32_t *n_dev, const int32_t *tile_start, const int32_t *cnt, int nr,
                               volatile long long *out, cudaStream_t st);
template <typename A, typename B>
cudaError_t launch_convert(const A *src, B *dst, size_t n, cudaStream_t st);

// k_reduce.cu
int reduce_blocks();
template <typename R>
cudaError_t launch_moments(const DevSpecies<R> &S, R m_mev, R emin, R emax, double *partials, double *result,
                           cudaStream_t st);
template <typename R>
cudaError_t launch_rho(const DevSpecies<R> &S, int n_upper, const MeshParams<R> &m, R *rho, cudaStream_t st);
template <typename R>
cudaError_t launch_gauss(const MeshParams<R> &m, const R *rho, const R *rho_bg, double dx, double dy, int i0,
                         int i1, double *partials, double *result, cudaStream_t st);
template <typename R>
cudaError_t launch_negate_copy(const R *src, R *dst, size_t n, cudaStream_t st);
template <typename R>
cudaError_t launch_subtract(R *dst, const R *src, size_t n, cudaStream_t st);
template <typename R>
cudaError_t launch_histogram(const DevSpecies<R> &S, R m_mev, R emin, R emax, int nbins, int log_bins,
                             double *out, cudaStream_t st);
template <typename R>
cudaError_t launch_rho3(const DevSpecies3<R> &S, int n_upper, const MeshParams3<R> &m, R *rho, cudaStream_t st);
template <typename R>
cudaError_t launch_gauss3(const MeshParams3<R> &m, const R *rho, const R *rho_bg, double dx, double dy, double dz,
                          int i0, int i1, double *partials, double *result, cudaStream_t st);
cudaError_t launch_diag_final(const double *rows, int nrows, int nsp, double *shift, pic_moments_dev *out,
                              double *tot, cudaStream_t st);

// k_adjoint.cu: discrete adjoint of the 2D3V step
template <typename R>
struct AdjMesh {
    int nx, ny, ld, bc_x;
    size_t plane;
    R dt, dt_dx, dt_dy, dx_dt, dy_dt;
    double r, q;              // dt/dx, dt/dy of the boundary
    R *LEB;                   // [6][ny][ld] lambda of E, B
    R *LJ;                    // [3][ny][ld] lambda of J (written by the E-step transpose)
    R *Lbnd;                  // [2][ny] lambda of By(-1/2), Bz(-1/2)
};
template <typename R>
struct AdjParticles {
    long long n;              // slots
    const uint32_t *cell;     // stored state at the step (2D3V packing)
    const R *ox, *oy, *ux, *uy, *uz, *sx, *sy, *sz, *w;
    const R *EB;              // stored E, B at the step
    R qm, q, a;
    R *lx, *ly, *lux, *luy, *luz, *lsx, *lsy, *lsz, *lw;  // lambdas, in: step n+1, out: step n
};
struct LossParams {
    double m_mev, ec, de;     // species rest energy, sigmoid centre and width [MeV]
    int axis;                 // spin component of the loss
};
template <typename R>
cudaError_t launch_adjoint_fields(const AdjMesh<R> &A, const double *prof, double phz, double phy, double *dl_da0,
                                  cudaStream_t st);
template <typename R>
cudaError_t launch_adjoint_particles(const AdjMesh<R> &A, const AdjParticles<R> &S, cudaStream_t st);
template <typename R>
cudaError_t launch_loss(const AdjParticles<R> &S, const LossParams &L, double *sums, bool grad, cudaStream_t st);

// pic_api.cu: the message pic_last_error(NULL) returns
void set_global_error(const std::string &msg);
