// k_fields.cu -- a6: Yee FDTD update (Yee 1966) in three stages, B half step,
// E full step with -J (which is then cleared), B half step, with a
// first-order Silver-Mueller boundary at x_min (laser source) and x_max.
#include <cmath>

#include "pic_kernels.h"

namespace {

// B <- B - h curl E at (i, j).  Bx on every column; By, Bz on the columns
// whose x+1 neighbour exists (all of them when x is periodic).
template <typename R>
__device__ __forceinline__ void b_half_cell(const MeshParams<R> &m, int i, int j, R hdx, R hdy) {
    const int jp = j + 1 == m.ny ? 0 : j + 1;
    const size_t P = m.plane;
    R *EB = m.EB;
    const size_t c = (size_t)j * m.ld + i, cjp = (size_t)jp * m.ld + i;
    const R ez = EB[2 * P + c];
    EB[3 * P + c] -= hdy * (EB[2 * P + cjp] - ez);
    const bool periodic = m.bc_x == 1;
    if (i < m.nx - 1 || periodic) {
        const size_t cip = (size_t)j * m.ld + (i + 1 == m.nx ? 0 : i + 1);
        EB[4 * P + c] += hdx * (EB[2 * P + cip] - ez);
        EB[5 * P + c] -= hdx * (EB[1 * P + cip] - EB[1 * P + c]) - hdy * (EB[0 * P + cjp] - EB[0 * P + c]);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_b_half(const MeshParams<R> m, R hdx, R hdy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) b_half_cell(m, i, blockIdx.y, hdx, hdy);
}

// The same for float, four cells of a row per thread with 16-byte loads and
// stores (ld is a multiple of 32; cells past nx keep their values).  The x + 1
// neighbour of the group's last cell is the next group's first, or at the
// row's end the wrapped column 0 (periodic x; By, Bz of the last column are
// left to the boundary stage otherwise).
__global__ void __launch_bounds__(128) k_b_half_f4(const MeshParams<float> m, float hdx, float hdy) {
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y;
    if (i0 >= m.nx) return;
    const int jp = j + 1 == m.ny ? 0 : j + 1;
    const size_t P = m.plane, r0 = (size_t)j * m.ld;
    const size_t c = r0 + i0, cjp = (size_t)jp * m.ld + i0;
    float *EB = m.EB;
    auto ld4 = [&](size_t o) { return *reinterpret_cast<const float4 *>(EB + o); };
    auto arr = [](const float4 v, float a[4]) { a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w; };
    float ex[4], ey[4], ez[4], ezjp[4], exjp[4], bx[4], by[4], bz[4];
    arr(ld4(c), ex);
    arr(ld4(P + c), ey);
    arr(ld4(2 * P + c), ez);
    arr(ld4(2 * P + cjp), ezjp);
    arr(ld4(cjp), exjp);
    arr(ld4(3 * P + c), bx);
    arr(ld4(4 * P + c), by);
    arr(ld4(5 * P + c), bz);
    const bool periodic = m.bc_x == 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + q;
        if (i >= m.nx) break;
        bx[q] -= hdy * (ezjp[q] - ez[q]);
        if (i < m.nx - 1 || periodic) {
            float eyn, ezn;  // Ey, Ez at the x + 1 neighbour
            if (i + 1 < m.nx && q < 3) {
                eyn = ey[q + 1];
                ezn = ez[q + 1];
            } else {
                const size_t cn = r0 + (i + 1 < m.nx ? i + 1 : 0);
                eyn = EB[P + cn];
                ezn = EB[2 * P + cn];
            }
            by[q] += hdx * (ezn - ez[q]);
            bz[q] -= hdx * (eyn - ey[q]) - hdy * (exjp[q] - ex[q]);
        }
    }
    *reinterpret_cast<float4 *>(EB + 3 * P + c) = make_float4(bx[0], bx[1], bx[2], bx[3]);
    *reinterpret_cast<float4 *>(EB + 4 * P + c) = make_float4(by[0], by[1], by[2], by[3]);
    *reinterpret_cast<float4 *>(EB + 5 * P + c) = make_float4(bz[0], bz[1], bz[2], bz[3]);
}

// boundary B at t^{n+1/2}: the incoming characteristic is the laser at x_min
// and zero at x_max, imposed on time-centred values with E^{n+1} from its own
// update including the transverse term dBx = Bx(j+1/2) - Bx(j-1/2) (r = dt/dx,
// q = dt/dy):
//   By(-1/2) = (2 Ez(0) - (1-r) By(1/2) - q dBx(0) - 4 f) / (1+r)
//   Bz(-1/2) = (4 g - 2 Ey(0) - (1-r) Bz(1/2)) / (1+r)
//   By(nx-1/2) = (-2 Ez(nx-1) - (1-r) By(nx-3/2) + q dBx(nx-1)) / (1+r)
//   Bz(nx-1/2) = (2 Ey(nx-1) - (1-r) Bz(nx-3/2)) / (1+r)
template <typename R>
__device__ __forceinline__ void boundary_row(const MeshParams<R> &m, R *bnd, const double *prof, double fz,
                                             double fy, double r, double q, int j) {
    // incident Ez (f) and Ey (g) at t^{n+1/2}: the time factor fz, fy (envelope x
    // carrier, one number per step) times the transverse profile prof[j] at y_j
    // and prof[ny + j] at y_{j+1/2}
    const size_t P = m.plane;
    R *EB = m.EB;
    const size_t c0 = (size_t)j * m.ld, cl = c0 + m.nx - 1;
    const size_t cm = (size_t)(j == 0 ? m.ny - 1 : j - 1) * m.ld;
    const double f = fz * prof[j];
    const double g = fy * prof[m.ny + j];
    const double ir = 1.0 / (1.0 + r), mr = 1.0 - r;
    const double dbx0 = (double)EB[3 * P + c0] - (double)EB[3 * P + cm];
    const double dbxl = (double)EB[3 * P + cl] - (double)EB[3 * P + cm + m.nx - 1];
    bnd[j] = (R)((2.0 * EB[2 * P + c0] - mr * EB[4 * P + c0] - q * dbx0 - 4.0 * f) * ir);
    bnd[m.ny + j] = (R)((4.0 * g - 2.0 * EB[1 * P + c0] - mr * EB[5 * P + c0]) * ir);
    EB[4 * P + cl] = (R)((-2.0 * EB[2 * P + cl] - mr * EB[4 * P + cl - 1] + q * dbxl) * ir);
    EB[5 * P + cl] = (R)((2.0 * EB[1 * P + cl] - mr * EB[5 * P + cl - 1]) * ir);
}

// lf: NULL, or the device address of this step's laser time factors (fz, fy)
// (a step replayed from a CUDA graph reads them from a table the host fills
// before each replay; a launched step passes them by value)
template <typename R>
__global__ void k_boundary(const MeshParams<R> m, R *bnd, const double *prof, double fz, double fy, double r,
                           double q, const double *lf) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (lf) {
        fz = lf[0];
        fy = lf[1];
    }
    if (j < m.ny) boundary_row(m, bnd, prof, fz, fy, r, q, j);
}

// E <- E + dt (curl B - J) at (i, j), then J <- 0
template <typename R>
__device__ __forceinline__ void e_full_cell(const MeshParams<R> &m, const R *bnd, R dt, R dtdx, R dtdy, int i,
                                            int j) {
    const int jm = j == 0 ? m.ny - 1 : j - 1;
    const size_t P = m.plane;
    R *EB = m.EB;
    R *J = m.J;
    const size_t c = (size_t)j * m.ld + i, cjm = (size_t)jm * m.ld + i;
    R by_im, bz_im;
    if (i > 0) {
        by_im = EB[4 * P + c - 1];
        bz_im = EB[5 * P + c - 1];
    } else if (m.bc_x == 1) {
        by_im = EB[4 * P + c + m.nx - 1];
        bz_im = EB[5 * P + c + m.nx - 1];
    } else {
        by_im = bnd[j];
        bz_im = bnd[m.ny + j];
    }
    const R bx = EB[3 * P + c], by = EB[4 * P + c], bz = EB[5 * P + c];
    EB[0 * P + c] += dtdy * (bz - EB[5 * P + cjm]) - dt * J[0 * P + c];
    EB[1 * P + c] += -dtdx * (bz - bz_im) - dt * J[1 * P + c];
    EB[2 * P + c] += dtdx * (by - by_im) - dtdy * (bx - EB[3 * P + cjm]) - dt * J[2 * P + c];
    J[0 * P + c] = R(0);
    J[1 * P + c] = R(0);
    J[2 * P + c] = R(0);
}

template <typename R>
__global__ void __launch_bounds__(256) k_e_full(const MeshParams<R> m, const R *bnd, R dt, R dtdx, R dtdy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m.nx) e_full_cell(m, bnd, dt, dtdx, dtdy, i, blockIdx.y);
}

// ---------------------------------------------------------------------------
// batched field update: one block per (run, row) item, runs past their last
// step skipped; the same cell updates as the single-run kernels, with the
// per-step scalars taken from the run's mesh parameters and laser table
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_b_half_batch(const BatchField<R> *runs, const int2 *rows, int nrows,
                                                      const long long *step, const long long *nsteps) {
    for (int b = blockIdx.x; b < nrows; b += gridDim.x) {
        const int2 rj = rows[b];
        if (step[rj.x] >= nsteps[rj.x]) continue;
        const MeshParams<R> &m = runs[rj.x].m;
        const R hdx = R(0.5) * m.dt_dx, hdy = R(0.5) * m.dt_dy;
        for (int i = threadIdx.x; i < m.nx; i += blockDim.x) b_half_cell(m, i, rj.y, hdx, hdy);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_e_full_batch(const BatchField<R> *runs, const int2 *rows, int nrows,
                                                      const long long *step, const long long *nsteps) {
    for (int b = blockIdx.x; b < nrows; b += gridDim.x) {
        const int2 rj = rows[b];
        if (step[rj.x] >= nsteps[rj.x]) continue;
        const BatchField<R> &F = runs[rj.x];
        for (int i = threadIdx.x; i < F.m.nx; i += blockDim.x)
            e_full_cell(F.m, F.bnd, F.m.dt, F.m.dt_dx, F.m.dt_dy, i, rj.y);
    }
}

template <typename R>
__global__ void k_boundary_batch(const BatchField<R> *runs, const int2 *rows, int nrows, const long long *step,
                                 const long long *nsteps) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nrows; b += gridDim.x * blockDim.x) {
        const int2 rj = rows[b];
        const long long k = step[rj.x];
        if (k >= nsteps[rj.x]) continue;
        const BatchField<R> &F = runs[rj.x];
        if (F.m.bc_x != 0) continue;
        const double *lf = F.laser + 2 * (k - F.step0);
        boundary_row(F.m, F.bnd, F.prof, lf[0], lf[1], F.r, F.q, rj.y);
    }
}

// step counters of the active runs advance; the fused kernel's queue rewinds
__global__ void k_batch_advance(long long *step, const long long *nsteps, int nruns, int *counter) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x)
        if (step[r] < nsteps[r]) step[r] += 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
}

// E <- E + dt (curl B - J), then J <- 0, for float: four cells of a row per
// thread as k_b_half_f4; each cell's x - 1 neighbour is the previous cell of
// the group, the previous group's last, or for column 0 the row's last cell
// (periodic x) or the boundary value.
__global__ void __launch_bounds__(128) k_e_full_f4(const MeshParams<float> m, const float *bnd, float dt,
                                                   float dtdx, float dtdy) {
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y;
    if (i0 >= m.nx) return;
    const int jm = j == 0 ? m.ny - 1 : j - 1;
    const size_t P = m.plane, r0 = (size_t)j * m.ld;
    const size_t c = r0 + i0, cjm = (size_t)jm * m.ld + i0;
    float *EB = m.EB, *J = m.J;
    auto ld4 = [](const float *p) { return *reinterpret_cast<const float4 *>(p); };
    auto arr = [](const float4 v, float a[4]) { a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w; };
    float bx[4], by[4], bz[4], bzjm[4], bxjm[4], ex[4], ey[4], ez[4], jx[4], jy[4], jz[4];
    arr(ld4(EB + 3 * P + c), bx);
    arr(ld4(EB + 4 * P + c), by);
    arr(ld4(EB + 5 * P + c), bz);
    arr(ld4(EB + 5 * P + cjm), bzjm);
    arr(ld4(EB + 3 * P + cjm), bxjm);
    arr(ld4(EB + c), ex);
    arr(ld4(EB + P + c), ey);
    arr(ld4(EB + 2 * P + c), ez);
    arr(ld4(J + c), jx);
    arr(ld4(J + P + c), jy);
    arr(ld4(J + 2 * P + c), jz);
    float by_im, bz_im;  // By, Bz at the x - 1 neighbour of the group's first cell
    if (i0 > 0) {
        by_im = EB[4 * P + c - 1];
        bz_im = EB[5 * P + c - 1];
    } else if (m.bc_x == 1) {
        by_im = EB[4 * P + r0 + m.nx - 1];
        bz_im = EB[5 * P + r0 + m.nx - 1];
    } else {
        by_im = bnd[j];
        bz_im = bnd[m.ny + j];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (i0 + q >= m.nx) break;
        if (q > 0) {
            by_im = by[q - 1];
            bz_im = bz[q - 1];
        }
        ex[q] += dtdy * (bz[q] - bzjm[q]) - dt * jx[q];
        ey[q] += -dtdx * (bz[q] - bz_im) - dt * jy[q];
        ez[q] += dtdx * (by[q] - by_im) - dtdy * (bx[q] - bxjm[q]) - dt * jz[q];
        jx[q] = jy[q] = jz[q] = 0.f;
    }
    *reinterpret_cast<float4 *>(EB + c) = make_float4(ex[0], ex[1], ex[2], ex[3]);
    *reinterpret_cast<float4 *>(EB + P + c) = make_float4(ey[0], ey[1], ey[2], ey[3]);
    *reinterpret_cast<float4 *>(EB + 2 * P + c) = make_float4(ez[0], ez[1], ez[2], ez[3]);
    *reinterpret_cast<float4 *>(J + c) = make_float4(jx[0], jx[1], jx[2], jx[3]);
    *reinterpret_cast<float4 *>(J + P + c) = make_float4(jy[0], jy[1], jy[2], jy[3]);
    *reinterpret_cast<float4 *>(J + 2 * P + c) = make_float4(jz[0], jz[1], jz[2], jz[3]);
}

}  // namespace

template <typename R>
cudaError_t launch_field_update_batch(const BatchField<R> *runs, const int2 *rows, int nrows, long long *step,
                                      const long long *nsteps, int nruns, int *counter, cudaStream_t st) {
    const int g = nrows < 152 * 16 ? nrows : 152 * 16;
    k_b_half_batch<R><<<g, 256, 0, st>>>(runs, rows, nrows, step, nsteps);
    k_boundary_batch<R><<<(nrows + 255) / 256, 256, 0, st>>>(runs, rows, nrows, step, nsteps);
    k_e_full_batch<R><<<g, 256, 0, st>>>(runs, rows, nrows, step, nsteps);
    k_b_half_batch<R><<<g, 256, 0, st>>>(runs, rows, nrows, step, nsteps);
    k_batch_advance<<<(nruns + 255) / 256, 256, 0, st>>>(step, nsteps, nruns, counter);
    return cudaGetLastError();
}
template cudaError_t launch_field_update_batch<float>(const BatchField<float> *, const int2 *, int, long long *,
                                                      const long long *, int, int *, cudaStream_t);

// laser time factors at t: the incident Ez (comp 1) and Ey (comp 0) on the
// axis, i.e. without the transverse profile
void laser_time_factors(const LaserParams &L, double t, double *fz, double *fy) {
    const double e = (t - L.t_peak) / L.tau;
    const double env = std::exp(-e * e);
    const double ph = t - L.t_peak;
    *fz = *fy = 0.0;
    if (L.pol == 1) {
        *fy = L.a0 * env * std::sin(ph);
    } else if (L.pol == 2) {
        *fy = L.a0 * 0.7071067811865476 * env * std::sin(ph);
        *fz = L.a0 * 0.7071067811865476 * env * std::cos(ph);
    }
}

template <typename R>
cudaError_t launch_field_update(const MeshParams<R> &m, R *bnd, const double *prof, const LaserParams &L,
                                double dt, double dx, double dy, long long step, cudaStream_t st,
                                const double *lf_dev) {
    const dim3 blk(256), grd((m.nx + 255) / 256, m.ny);
    const dim3 blk4(128), grd4((m.nx + 4 * 128 - 1) / (4 * 128), m.ny);
    const R hdx = (R)(0.5 * dt / dx), hdy = (R)(0.5 * dt / dy);
    auto b_half = [&]() {
        if constexpr (sizeof(R) == 4)
            k_b_half_f4<<<grd4, blk4, 0, st>>>(m, hdx, hdy);
        else
            k_b_half<R><<<grd, blk, 0, st>>>(m, hdx, hdy);
    };
    b_half();
    if (m.bc_x == 0) {
        double fz, fy;
        laser_time_factors(L, ((double)step + 0.5) * dt, &fz, &fy);
        k_boundary<R><<<(m.ny + 127) / 128, 128, 0, st>>>(m, bnd, prof, fz, fy, dt / dx, dt / dy, lf_dev);
    }
    if constexpr (sizeof(R) == 4)
        k_e_full_f4<<<grd4, blk4, 0, st>>>(m, bnd, (R)dt, (R)(dt / dx), (R)(dt / dy));
    else
        k_e_full<R><<<grd, blk, 0, st>>>(m, bnd, (R)dt, (R)(dt / dx), (R)(dt / dy));
    b_half();
    return cudaGetLastError();
}

template cudaError_t launch_field_update<float>(const MeshParams<float> &, float *, const double *,
                                                const LaserParams &, double, double, double, long long,
                                                cudaStream_t, const double *);
template cudaError_t launch_field_update<double>(const MeshParams<double> &, double *, const double *,
                                                 const LaserParams &, double, double, double, long long,
                                                 cudaStream_t, const double *);

// transverse laser profile exp(-((y - yc)/w0)^2) at y_j (first ny) and y_{j+1/2}
void laser_profile(const LaserParams &L, int ny, double *host) {
    for (int j = 0; j < ny; ++j) {
        const double a = ((double)j * L.dy - L.yc) / L.w0;
        const double b = (((double)j + 0.5) * L.dy - L.yc) / L.w0;
        host[j] = std::exp(-a * a);
        host[ny + j] = std::exp(-b * b);
    }
}
