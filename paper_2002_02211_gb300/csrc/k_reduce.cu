// k_reduce.cu -- a8: FP64 reductions.  Eq. (4) polarization moments of one
// species in an energy window (two passes: sums, then the variance about the
// mean), the CIC charge density, and the charge-conservation residual
// div E - rho.  Per-block FP64 partials are summed by one CTA in a fixed
// order, so a result depends only on the particle order, not on timing.
#include "pic_kernels.h"

#define MEC2_MEV 0.51099895

namespace {

constexpr int RB = 152 * 4;  // reduction blocks
constexpr int RT = 256;      // threads per reduction block

// FP64 block reduction of NV values per thread; thread 0 writes the block's row
template <int NV>
__device__ void block_sum(double (&v)[NV], double *row) {
    __shared__ double red[RT / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xFFFFFFFFu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < RT / 32; ++w) s += red[w][k];
            row[k] = s;
        }
    }
}

template <typename R>
__device__ __forceinline__ R ekin(R m_mev, R ux, R uy, R uz) {
    return ekin_mev(m_mev, ux, uy, uz);
}

// pass 1: sum w, sum w s (3), sum w e, count.  Each thread folds float sums of
// at most 16 particles into its double accumulators.
template <typename R>
__global__ void __launch_bounds__(RT) k_mom1(const DevSpecies<R> S, R m_mev, R emin, R emax, double *partials) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    R f[6] = {0, 0, 0, 0, 0, 0};
    int k = 0;
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        if (S.cell[p] == PIC_DEAD) continue;
        const R e = ekin(m_mev, S.ux[p], S.uy[p], S.uz[p]);
        if (!(e >= emin && e < emax)) continue;
        const R w = S.w[p];
        f[0] += w;
        f[1] += w * S.sx[p];
        f[2] += w * S.sy[p];
        f[3] += w * S.sz[p];
        f[4] += w * e;
        f[5] += R(1);
        if (++k == 16) {
            for (int q = 0; q < 6; ++q) {
                acc[q] += (double)f[q];
                f[q] = R(0);
            }
            k = 0;
        }
    }
    for (int q = 0; q < 6; ++q) acc[q] += (double)f[q];
    block_sum<6>(acc, partials + (size_t)blockIdx.x * 6);
}

// fixed-order sum of nb rows of width nv; row 0 of result gets the sums
__global__ void __launch_bounds__(RT) k_final(const double *partials, int nb, int nv, double *result) {
    __shared__ double s[RT];
    for (int q = 0; q < nv; ++q) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) a += partials[(size_t)b * nv + q];
        s[threadIdx.x] = a;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) result[q] = s[0];
        __syncthreads();
    }
}

// max over rows for column 0, sum for column 1
__global__ void __launch_bounds__(RT) k_final_maxsum(const double *partials, int nb, double *result) {
    __shared__ double smax[RT], ssum[RT];
    double a = 0.0, b = 0.0;
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
        a = fmax(a, partials[(size_t)r * 2]);
        b += partials[(size_t)r * 2 + 1];
    }
    smax[threadIdx.x] = a;
    ssum[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        result[0] = smax[0];
        result[1] = ssum[0];
    }
}

// pass 2: sum w (e - mean)^2, the mean read from pass 1's result
template <typename R>
__global__ void __launch_bounds__(RT) k_mom2(const DevSpecies<R> S, R m_mev, R emin, R emax, const double *r1,
                                             double *partials) {
    const double sw = r1[0];
    const R mean = sw > 0.0 ? (R)(r1[4] / sw) : R(0);
    double acc[1] = {0.0};
    R f = R(0);
    int k = 0;
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        if (S.cell[p] == PIC_DEAD) continue;
        const R e = ekin(m_mev, S.ux[p], S.uy[p], S.uz[p]);
        if (!(e >= emin && e < emax)) continue;
        const R d = e - mean;
        f += S.w[p] * d * d;
        if (++k == 16) {
            acc[0] += (double)f;
            f = R(0);
            k = 0;
        }
    }
    acc[0] += (double)f;
    block_sum<1>(acc, partials + blockIdx.x);
}

// CIC charge density of one species at the nodes
template <typename R>
__global__ void k_rho(const DevSpecies<R> S, const MeshParams<R> m, R *rho) {
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[p];
        if (c == PIC_DEAD) continue;
        const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
        const R ox = S.ox[p], oy = S.oy[p], qw = S.q * S.w[p], one = R(1);
        const int ix1 = ix + 1 == m.nx ? 0 : ix + 1;
        const int iy1 = iy + 1 == m.ny ? 0 : iy + 1;
        atomicAdd(&rho[(size_t)iy * m.ld + ix], qw * (one - ox) * (one - oy));
        atomicAdd(&rho[(size_t)iy * m.ld + ix1], qw * ox * (one - oy));
        atomicAdd(&rho[(size_t)iy1 * m.ld + ix], qw * (one - ox) * oy);
        atomicAdd(&rho[(size_t)iy1 * m.ld + ix1], qw * ox * oy);
    }
}

// div E - rho - rho_bg on nodes i in [i0, i1]: block max |r| and sum r^2
template <typename R>
__global__ void __launch_bounds__(RT) k_gauss(const MeshParams<R> m, const R *rho, const R *rho_bg,
                                              double idx, double idy, int i0, int i1, double *partials) {
    double vmax = 0.0, ssq = 0.0;
    const int w = i1 - i0 + 1;
    const long long total = (long long)w * m.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q / w), i = i0 + (int)(q - (long long)j * w);
        const int im = i == 0 ? m.nx - 1 : i - 1, jm = j == 0 ? m.ny - 1 : j - 1;
        const size_t c = (size_t)j * m.ld + i;
        const double div = ((double)m.EB[c] - (double)m.EB[(size_t)j * m.ld + im]) * idx +
                           ((double)m.EB[m.plane + c] - (double)m.EB[m.plane + (size_t)jm * m.ld + i]) * idy;
        const double r = div - (double)rho[c] - (double)rho_bg[c];
        vmax = fmax(vmax, fabs(r));
        ssq += r * r;
    }
    __shared__ double smax[RT], ssum[RT];
    smax[threadIdx.x] = vmax;
    ssum[threadIdx.x] = ssq;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = smax[0];
        partials[2 * blockIdx.x + 1] = ssum[0];
    }
}

// 3D3V: CIC charge density at the nodes (periodic y, z; x wraps when periodic)
template <typename R>
__global__ void k_rho3(const DevSpecies3<R> S, const MeshParams3<R> m, R *rho) {
    const int n = *S.n;
    const size_t slab = (size_t)m.ny * m.ld;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[p];
        if (c == PIC_DEAD) continue;
        int ix, iy, iz;
        unpack_cell3(c, ix, iy, iz);
        const R one = R(1), qw = S.q * S.w[p];
        const R wx[2] = {one - S.ox[p], S.ox[p]}, wy[2] = {one - S.oy[p], S.oy[p]}, wz[2] = {one - S.oz[p], S.oz[p]};
        const int xs[2] = {ix, ix + 1 == m.nx ? 0 : ix + 1};
        const int ys[2] = {iy, iy + 1 == m.ny ? 0 : iy + 1};
        const int zs[2] = {iz, iz + 1 == m.nz ? 0 : iz + 1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int d = 0; d < 2; ++d)
                    atomicAdd(&rho[zs[d] * slab + (size_t)ys[b] * m.ld + xs[a]], qw * wx[a] * wy[b] * wz[d]);
    }
}

// 3D3V div E - rho - rho_bg on nodes with i in [i0, i1]: block max |r| and sum r^2
template <typename R>
__global__ void __launch_bounds__(RT) k_gauss3(const MeshParams3<R> m, const R *rho, const R *rho_bg, double idx,
                                               double idy, double idz, int i0, int i1, double *partials) {
    double vmax = 0.0, ssq = 0.0;
    const int w = i1 - i0 + 1;
    const long long total = (long long)w * m.ny * m.nz;
    const size_t slab = (size_t)m.ny * m.ld;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long jk = q / w;
        const int i = i0 + (int)(q - jk * w);
        const int k = (int)(jk / m.ny), j = (int)(jk - (long long)k * m.ny);
        const int im = i == 0 ? m.nx - 1 : i - 1, jm = j == 0 ? m.ny - 1 : j - 1, km = k == 0 ? m.nz - 1 : k - 1;
        const size_t c = k * slab + (size_t)j * m.ld + i;
        const double div = ((double)m.EB[c] - (double)m.EB[k * slab + (size_t)j * m.ld + im]) * idx +
                           ((double)m.EB[m.plane + c] - (double)m.EB[m.plane + k * slab + (size_t)jm * m.ld + i]) * idy +
                           ((double)m.EB[2 * m.plane + c] -
                            (double)m.EB[2 * m.plane + km * slab + (size_t)j * m.ld + i]) * idz;
        const double r = div - (double)rho[c] - (double)rho_bg[c];
        vmax = fmax(vmax, fabs(r));
        ssq += r * r;
    }
    __shared__ double smax[RT], ssum[RT];
    smax[threadIdx.x] = vmax;
    ssum[threadIdx.x] = ssq;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
            ssum[threadIdx.x] += ssum[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = smax[0];
        partials[2 * blockIdx.x + 1] = ssum[0];
    }
}

template <typename R>
__global__ void k_subtract(R *dst, const R *src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] -= src[i];
}

template <typename R>
__global__ void k_negate(const R *src, R *dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = -src[i];
}

// Fixed-order sum of each column of the per-CTA diagnostic sums
// [PIC_MAXSP][8][nrows]: one block per (species, quantity) column.
__global__ void __launch_bounds__(RT) k_diag_cols(const double *rows, int nrows, double *tot) {
    __shared__ double s[RT];
    const double *col = rows + (size_t)blockIdx.x * nrows;
    double a = 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) a += col[r];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = s[0];
}

// moments of each species from the column sums; the new mean becomes the next shift
__global__ void k_diag_moments(const double *tot, int nsp, double *shift, pic_moments_dev *out) {
    const int sp = threadIdx.x;
    if (sp >= nsp) return;
    const double *t = tot + sp * 8;
    const double sw = t[0], sh = shift[sp];
    pic_moments_dev m;
    for (int k = 0; k < 3; ++k) m.P[k] = sw > 0 ? t[1 + k] / sw : 0.0;
    const double d = sw > 0 ? t[4] / sw : 0.0;
    m.sum_w = sw;
    m.count = t[6];
    m.ekin_mean = sw > 0 ? sh + d : 0.0;
    m.ekin_var = sw > 0 ? fmax(t[5] / sw - d * d, 0.0) : 0.0;
    out[sp] = m;
    if (sw > 0) shift[sp] = sh + d;
}

// Energy spectra: each block bins its particles in shared memory (float, a
// few thousand particles per block), then adds its bins to the FP64
// histogram out[nbins][5] (count, sum w, sum w s) with global atomics.
template <typename R>
__global__ void __launch_bounds__(RT) k_hist(const DevSpecies<R> S, R m_mev, R emin, R emax, int nbins,
                                             int log_bins, double *out) {
    extern __shared__ float sh[];  // [nbins][5]
    for (int i = threadIdx.x; i < 5 * nbins; i += blockDim.x) sh[i] = 0.f;
    __syncthreads();
    const int n = *S.n;
    const R scale = log_bins ? R(1) / log(emax / emin) : R(1) / (emax - emin);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        if (S.cell[p] == PIC_DEAD) continue;
        const R e = ekin(m_mev, S.ux[p], S.uy[p], S.uz[p]);
        if (!(e >= emin && e < emax)) continue;
        const R f = log_bins ? log(e / emin) * scale : (e - emin) * scale;
        int b = (int)floor(f * (R)nbins);
        b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        const float w = (float)S.w[p];
        atomicAdd(&sh[5 * b + 0], 1.f);
        atomicAdd(&sh[5 * b + 1], w);
        atomicAdd(&sh[5 * b + 2], w * (float)S.sx[p]);
        atomicAdd(&sh[5 * b + 3], w * (float)S.sy[p]);
        atomicAdd(&sh[5 * b + 4], w * (float)S.sz[p]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 5 * nbins; i += blockDim.x)
        if (sh[i] != 0.f) atomicAdd(&out[i], (double)sh[i]);
}

}  // namespace

int reduce_blocks() { return RB; }

template <typename R>
cudaError_t launch_histogram(const DevSpecies<R> &S, R m_mev, R emin, R emax, int nbins, int log_bins,
                             double *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 5 * nbins, st);
    if (e != cudaSuccess) return e;
    k_hist<R><<<152 * 32, RT, sizeof(float) * 5 * nbins, st>>>(S, m_mev, emin, emax, nbins, log_bins, out);
    return cudaGetLastError();
}
template cudaError_t launch_histogram<float>(const DevSpecies<float> &, float, float, float, int, int, double *,
                                             cudaStream_t);
template cudaError_t launch_histogram<double>(const DevSpecies<double> &, double, double, double, int, int,
                                              double *, cudaStream_t);

cudaError_t launch_diag_final(const double *rows, int nrows, int nsp, double *shift, pic_moments_dev *out,
                              double *tot, cudaStream_t st) {
    k_diag_cols<<<nsp * 8, RT, 0, st>>>(rows, nrows, tot);
    k_diag_moments<<<1, 32, 0, st>>>(tot, nsp, shift, out);
    return cudaGetLastError();
}


// result[0..5] = sums of pass 1, result[6] = sum w (e - mean)^2
template <typename R>
cudaError_t launch_moments(const DevSpecies<R> &S, R m_mev, R emin, R emax, double *partials, double *result,
                           cudaStream_t st) {
    k_mom1<R><<<RB, RT, 0, st>>>(S, m_mev, emin, emax, partials);
    k_final<<<1, RT, 0, st>>>(partials, RB, 6, result);
    k_mom2<R><<<RB, RT, 0, st>>>(S, m_mev, emin, emax, result, partials);
    k_final<<<1, RT, 0, st>>>(partials, RB, 1, result + 6);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rho(const DevSpecies<R> &S, int n_upper, const MeshParams<R> &m, R *rho, cudaStream_t st) {
    int b = (n_upper + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    k_rho<R><<<b, 256, 0, st>>>(S, m, rho);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gauss(const MeshParams<R> &m, const R *rho, const R *rho_bg, double dx, double dy, int i0,
                         int i1, double *partials, double *result, cudaStream_t st) {
    k_gauss<R><<<RB, RT, 0, st>>>(m, rho, rho_bg, 1.0 / dx, 1.0 / dy, i0, i1, partials);
    k_final_maxsum<<<1, RT, 0, st>>>(partials, RB, result);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rho3(const DevSpecies3<R> &S, int n_upper, const MeshParams3<R> &m, R *rho, cudaStream_t st) {
    int b = (n_upper + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    k_rho3<R><<<b, 256, 0, st>>>(S, m, rho);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gauss3(const MeshParams3<R> &m, const R *rho, const R *rho_bg, double dx, double dy, double dz,
                          int i0, int i1, double *partials, double *result, cudaStream_t st) {
    k_gauss3<R><<<RB, RT, 0, st>>>(m, rho, rho_bg, 1.0 / dx, 1.0 / dy, 1.0 / dz, i0, i1, partials);
    k_final_maxsum<<<1, RT, 0, st>>>(partials, RB, result);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_subtract(R *dst, const R *src, size_t n, cudaStream_t st) {
    k_subtract<R><<<152 * 4, 256, 0, st>>>(dst, src, n);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_negate_copy(const R *src, R *dst, size_t n, cudaStream_t st) {
    k_negate<R><<<152 * 4, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

#define PIC_INST(R)                                                                                        \
    template cudaError_t launch_moments<R>(const DevSpecies<R> &, R, R, R, double *, double *, cudaStream_t); \
    template cudaError_t launch_rho<R>(const DevSpecies<R> &, int, const MeshParams<R> &, R *, cudaStream_t); \
    template cudaError_t launch_gauss<R>(const MeshParams<R> &, const R *, const R *, double, double, int, int,  \
                                         double *, double *, cudaStream_t);                                 \
    template cudaError_t launch_negate_copy<R>(const R *, R *, size_t, cudaStream_t);                    \
    template cudaError_t launch_subtract<R>(R *, const R *, size_t, cudaStream_t);                       \
    template cudaError_t launch_rho3<R>(const DevSpecies3<R> &, int, const MeshParams3<R> &, R *, cudaStream_t); \
    template cudaError_t launch_gauss3<R>(const MeshParams3<R> &, const R *, const R *, double, double, double, \
                                          int, int, double *, double *, cudaStream_t);
PIC_INST(float)
PIC_INST(double)
#undef PIC_INST
