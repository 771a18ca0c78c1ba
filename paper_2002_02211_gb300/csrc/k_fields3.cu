// k_fields3.cu -- a6 in 3D: Yee FDTD update (Yee 1966) in three stages, B
// half step, E full step with -J (which is then cleared), B half step, with a
// first-order Silver-Mueller boundary at x_min (laser source) and x_max.
// One thread per cell, x fastest (coalesced rows), y and z periodic.
#include <cmath>

#include "pic_device3.cuh"
#include "pic_kernels.h"

namespace {

template <typename R>
struct Idx3 {
    size_t c, cjp, ckp, cjm, ckm;
    int i, j, k;
};

template <typename R>
__device__ __forceinline__ bool cell_of_thread(const MeshParams3<R> &m, Idx3<R> &q) {
    q.i = blockIdx.x * blockDim.x + threadIdx.x;
    q.j = blockIdx.y;
    q.k = blockIdx.z;
    if (q.i >= m.nx) return false;
    const int jp = q.j + 1 == m.ny ? 0 : q.j + 1, jm = q.j == 0 ? m.ny - 1 : q.j - 1;
    const int kp = q.k + 1 == m.nz ? 0 : q.k + 1, km = q.k == 0 ? m.nz - 1 : q.k - 1;
    const size_t row = (size_t)m.ld;
    const size_t slab = (size_t)m.ny * m.ld;
    q.c = q.k * slab + q.j * row + q.i;
    q.cjp = q.k * slab + jp * row + q.i;
    q.cjm = q.k * slab + jm * row + q.i;
    q.ckp = kp * slab + q.j * row + q.i;
    q.ckm = km * slab + q.j * row + q.i;
    return true;
}

// B <- B - h curl E.  Bx on every column; By, Bz where the x+1 neighbour exists
template <typename R>
__global__ void __launch_bounds__(256) k_b_half3(const MeshParams3<R> m, R hdx, R hdy, R hdz) {
    Idx3<R> q;
    if (!cell_of_thread(m, q)) return;
    const size_t P = m.plane;
    R *EB = m.EB;
    const R ex = EB[0 * P + q.c], ey = EB[1 * P + q.c], ez = EB[2 * P + q.c];
    EB[3 * P + q.c] -= hdy * (EB[2 * P + q.cjp] - ez) - hdz * (EB[1 * P + q.ckp] - ey);
    if (q.i < m.nx - 1 || m.bc_x == 1) {
        const size_t cip = q.c - q.i + (q.i + 1 == m.nx ? 0 : q.i + 1);
        EB[4 * P + q.c] -= hdz * (EB[0 * P + q.ckp] - ex) - hdx * (EB[2 * P + cip] - ez);
        EB[5 * P + q.c] -= hdx * (EB[1 * P + cip] - ey) - hdy * (EB[0 * P + q.cjp] - ex);
    }
}

// The same for float, four cells of a row per thread: 16-byte loads and
// stores (rows are padded to a multiple of 32 cells, so a group of four starts
// 16-byte aligned and stays inside its row's storage).  Cells past nx keep
// their values; each cell's x + 1 neighbour is the next cell of the group, the
// next group's first, or column 0 when x is periodic and the cell ends the row.
__global__ void __launch_bounds__(128) k_b_half3_f4(const MeshParams3<float> m, float hdx, float hdy, float hdz) {
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y, k = blockIdx.z;
    if (i0 >= m.nx) return;
    const int jp = j + 1 == m.ny ? 0 : j + 1, kp = k + 1 == m.nz ? 0 : k + 1;
    const size_t row = (size_t)m.ld, slab = (size_t)m.ny * m.ld, P = m.plane;
    const size_t r0 = (size_t)k * slab + (size_t)j * row;  // start of the row
    const size_t c = r0 + i0, cjp = (size_t)k * slab + (size_t)jp * row + i0, ckp = (size_t)kp * slab + (size_t)j * row + i0;
    float *EB = m.EB;
    auto ld4 = [&](size_t o) { return *reinterpret_cast<const float4 *>(EB + o); };
    auto arr = [](const float4 v, float a[4]) { a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w; };
    float ex[4], ey[4], ez[4], ezjp[4], eykp[4], exkp[4], exjp[4], bx[4], by[4], bz[4];
    arr(ld4(c), ex);
    arr(ld4(P + c), ey);
    arr(ld4(2 * P + c), ez);
    arr(ld4(2 * P + cjp), ezjp);
    arr(ld4(P + ckp), eykp);
    arr(ld4(ckp), exkp);
    arr(ld4(cjp), exjp);
    arr(ld4(3 * P + c), bx);
    arr(ld4(4 * P + c), by);
    arr(ld4(5 * P + c), bz);
    const bool periodic = m.bc_x == 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + q;
        if (i >= m.nx) break;
        bx[q] -= hdy * (ezjp[q] - ez[q]) - hdz * (eykp[q] - ey[q]);
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
            by[q] -= hdz * (exkp[q] - ex[q]) - hdx * (ezn - ez[q]);
            bz[q] -= hdx * (eyn - ey[q]) - hdy * (exjp[q] - ex[q]);
        }
    }
    *reinterpret_cast<float4 *>(EB + 3 * P + c) = make_float4(bx[0], bx[1], bx[2], bx[3]);
    *reinterpret_cast<float4 *>(EB + 4 * P + c) = make_float4(by[0], by[1], by[2], by[3]);
    *reinterpret_cast<float4 *>(EB + 5 * P + c) = make_float4(bz[0], bz[1], bz[2], bz[3]);
}

// boundary B at t^{n+1/2}; one thread per (j, k).  With r = dt/dx, qy = dt/dy,
// qz = dt/dz and the incident Ez (f) and Ey (g):
//   By(-1/2) = (2 Ez(0) - (1-r) By(1/2) - qy dyBx - 4 f) / (1+r)
//   Bz(-1/2) = (4 g - 2 Ey(0) - (1-r) Bz(1/2) - qz dzBx) / (1+r)
//   By(nx-1/2) = (-2 Ez - (1-r) By(nx-3/2) + qy dyBx) / (1+r)
//   Bz(nx-1/2) = ( 2 Ey - (1-r) Bz(nx-3/2) + qz dzBx) / (1+r)
// dyBx = Bx(j+1/2) - Bx(j-1/2) and dzBx = Bx(k+1/2) - Bx(k-1/2), taken in the
// boundary column.  bnd holds By(-1/2) [nz][ny] then Bz(-1/2) [nz][ny].
template <typename R>
__global__ void k_boundary3(const MeshParams3<R> m, R *bnd, const double *prof, double fz, double fy, double r,
                            double qy, double qz, const double *lf) {
    if (lf) {  // a step replayed from a CUDA graph: this step's factors from the host-filled table
        fz = lf[0];
        fy = lf[1];
    }
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= m.ny) return;
    const size_t P = m.plane, slab = (size_t)m.ny * m.ld;
    R *EB = m.EB;
    const int jm = j == 0 ? m.ny - 1 : j - 1, km = k == 0 ? m.nz - 1 : k - 1;
    const size_t c0 = k * slab + (size_t)j * m.ld, cl = c0 + m.nx - 1;
    const size_t cy0 = k * slab + (size_t)jm * m.ld, cz0 = km * slab + (size_t)j * m.ld;
    const size_t b = (size_t)k * m.ny + j, nb = (size_t)m.ny * m.nz;
    const double f = fz * prof[b];        // Ez source at (y_j, z_{k+1/2})
    const double g = fy * prof[nb + b];   // Ey source at (y_{j+1/2}, z_k)
    const double ir = 1.0 / (1.0 + r), mr = 1.0 - r;
    const double bx0 = EB[3 * P + c0], bxl = EB[3 * P + cl];
    const double dyb0 = bx0 - (double)EB[3 * P + cy0], dzb0 = bx0 - (double)EB[3 * P + cz0];
    const double dybl = bxl - (double)EB[3 * P + cy0 + m.nx - 1], dzbl = bxl - (double)EB[3 * P + cz0 + m.nx - 1];
    bnd[b] = (R)((2.0 * EB[2 * P + c0] - mr * EB[4 * P + c0] - qy * dyb0 - 4.0 * f) * ir);
    bnd[nb + b] = (R)((4.0 * g - 2.0 * EB[1 * P + c0] - mr * EB[5 * P + c0] - qz * dzb0) * ir);
    EB[4 * P + cl] = (R)((-2.0 * EB[2 * P + cl] - mr * EB[4 * P + cl - 1] + qy * dybl) * ir);
    EB[5 * P + cl] = (R)((2.0 * EB[1 * P + cl] - mr * EB[5 * P + cl - 1] + qz * dzbl) * ir);
}

// E <- E + dt (curl B - J), then J <- 0
template <typename R>
__global__ void __launch_bounds__(256) k_e_full3(const MeshParams3<R> m, const R *bnd, R dt, R dtdx, R dtdy,
                                                 R dtdz) {
    Idx3<R> q;
    if (!cell_of_thread(m, q)) return;
    const size_t P = m.plane;
    R *EB = m.EB;
    R *J = m.J;
    R by_im, bz_im;
    if (q.i > 0) {
        by_im = EB[4 * P + q.c - 1];
        bz_im = EB[5 * P + q.c - 1];
    } else if (m.bc_x == 1) {
        by_im = EB[4 * P + q.c + m.nx - 1];
        bz_im = EB[5 * P + q.c + m.nx - 1];
    } else {
        const size_t b = (size_t)q.k * m.ny + q.j;
        by_im = bnd[b];
        bz_im = bnd[(size_t)m.ny * m.nz + b];
    }
    const R bx = EB[3 * P + q.c], by = EB[4 * P + q.c], bz = EB[5 * P + q.c];
    EB[0 * P + q.c] += dtdy * (bz - EB[5 * P + q.cjm]) - dtdz * (by - EB[4 * P + q.ckm]) - dt * J[0 * P + q.c];
    EB[1 * P + q.c] += dtdz * (bx - EB[3 * P + q.ckm]) - dtdx * (bz - bz_im) - dt * J[1 * P + q.c];
    EB[2 * P + q.c] += dtdx * (by - by_im) - dtdy * (bx - EB[3 * P + q.cjm]) - dt * J[2 * P + q.c];
    J[0 * P + q.c] = R(0);
    J[1 * P + q.c] = R(0);
    J[2 * P + q.c] = R(0);
}

// The same for float, four cells of a row per thread with 16-byte accesses,
// as k_b_half3_f4; cells past nx keep their E and J.  Each cell's x - 1
// neighbour is the previous cell of the group, the previous group's last, or
// for column 0 the row's last cell (periodic x) or the boundary value.
__global__ void __launch_bounds__(128) k_e_full3_f4(const MeshParams3<float> m, const float *bnd, float dt,
                                                    float dtdx, float dtdy, float dtdz) {
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y, k = blockIdx.z;
    if (i0 >= m.nx) return;
    const int jm = j == 0 ? m.ny - 1 : j - 1, km = k == 0 ? m.nz - 1 : k - 1;
    const size_t row = (size_t)m.ld, slab = (size_t)m.ny * m.ld, P = m.plane;
    const size_t r0 = (size_t)k * slab + (size_t)j * row;
    const size_t c = r0 + i0, cjm = (size_t)k * slab + (size_t)jm * row + i0, ckm = (size_t)km * slab + (size_t)j * row + i0;
    float *EB = m.EB, *J = m.J;
    auto ld4 = [](const float *p) { return *reinterpret_cast<const float4 *>(p); };
    auto arr = [](const float4 v, float a[4]) { a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w; };
    float bx[4], by[4], bz[4], bzjm[4], bxjm[4], bykm[4], bxkm[4], ex[4], ey[4], ez[4], jx[4], jy[4], jz[4];
    arr(ld4(EB + 3 * P + c), bx);
    arr(ld4(EB + 4 * P + c), by);
    arr(ld4(EB + 5 * P + c), bz);
    arr(ld4(EB + 5 * P + cjm), bzjm);
    arr(ld4(EB + 3 * P + cjm), bxjm);
    arr(ld4(EB + 4 * P + ckm), bykm);
    arr(ld4(EB + 3 * P + ckm), bxkm);
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
        const size_t b = (size_t)k * m.ny + j;
        by_im = bnd[b];
        bz_im = bnd[(size_t)m.ny * m.nz + b];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (i0 + q >= m.nx) break;
        if (q > 0) {
            by_im = by[q - 1];
            bz_im = bz[q - 1];
        }
        ex[q] += dtdy * (bz[q] - bzjm[q]) - dtdz * (by[q] - bykm[q]) - dt * jx[q];
        ey[q] += dtdz * (bx[q] - bxkm[q]) - dtdx * (bz[q] - bz_im) - dt * jy[q];
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
cudaError_t launch_field_update3(const MeshParams3<R> &m, R *bnd, const double *prof, const LaserParams &L,
                                 double dt, double dx, double dy, double dz, long long step, cudaStream_t st,
                                 const double *lf_dev) {
    const dim3 blk(128), grd((m.nx + 127) / 128, m.ny, m.nz);
    const dim3 grd4((m.nx + 4 * 128 - 1) / (4 * 128), m.ny, m.nz);
    const R hdx = (R)(0.5 * dt / dx), hdy = (R)(0.5 * dt / dy), hdz = (R)(0.5 * dt / dz);
    auto b_half = [&]() {
        if constexpr (sizeof(R) == 4)
            k_b_half3_f4<<<grd4, blk, 0, st>>>(m, hdx, hdy, hdz);
        else
            k_b_half3<R><<<grd, blk, 0, st>>>(m, hdx, hdy, hdz);
    };
    b_half();
    if (m.bc_x == 0) {
        double fz, fy;
        laser_time_factors(L, ((double)step + 0.5) * dt, &fz, &fy);
        k_boundary3<R><<<dim3((m.ny + 127) / 128, m.nz), 128, 0, st>>>(m, bnd, prof, fz, fy, dt / dx, dt / dy,
                                                                       dt / dz, lf_dev);
    }
    if constexpr (sizeof(R) == 4)
        k_e_full3_f4<<<grd4, blk, 0, st>>>(m, bnd, (R)dt, (R)(dt / dx), (R)(dt / dy), (R)(dt / dz));
    else
        k_e_full3<R><<<grd, blk, 0, st>>>(m, bnd, (R)dt, (R)(dt / dx), (R)(dt / dy), (R)(dt / dz));
    b_half();
    return cudaGetLastError();
}

template cudaError_t launch_field_update3<float>(const MeshParams3<float> &, float *, const double *,
                                                 const LaserParams &, double, double, double, double, long long,
                                                 cudaStream_t, const double *);
template cudaError_t launch_field_update3<double>(const MeshParams3<double> &, double *, const double *,
                                                  const LaserParams &, double, double, double, double, long long,
                                                  cudaStream_t, const double *);

// transverse laser profile exp(-((y - yc)^2 + (z - zc)^2) / w0^2): [nz][ny] at
// (y_j, z_{k+1/2}) (the Ez source), then [nz][ny] at (y_{j+1/2}, z_k) (Ey)
void laser_profile3(const LaserParams &L, int ny, int nz, double dz, double *host) {
    const double zc = 0.5 * nz * dz;
    const size_t nb = (size_t)ny * nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            const double ya = (double)j * L.dy - L.yc, za = ((double)k + 0.5) * dz - zc;
            const double yb = ((double)j + 0.5) * L.dy - L.yc, zb = (double)k * dz - zc;
            const size_t b = (size_t)k * ny + j;
            host[b] = std::exp(-(ya * ya + za * za) / (L.w0 * L.w0));
            host[nb + b] = std::exp(-(yb * yb + zb * zb) / (L.w0 * L.w0));
        }
}
