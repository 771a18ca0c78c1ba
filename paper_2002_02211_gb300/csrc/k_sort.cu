// k_sort.cu -- a7: counting sort of the particles of one species by tile,
// laid out in layers inside each tile.  Removed particles are dropped.
//
// With C = TX * TY cells per tile and R = the smallest particle count of any
// cell of the tile, slot r * C + c of the tile holds the r-th particle of
// local cell c for r < R (every cell has at least R, so the layers have no
// holes); the remaining particles follow in a tail, cell by cell.  A CTA of
// C (or a divisor of C) threads walking the tile therefore meets the same
// cell on every pass through the layers, which the fused kernel uses to sum
// the in-cell currents in registers.  Steps: rank of each particle in its
// cell (atomics), per-tile layout (block min and scan over the cells),
// exclusive scan of the tile totals, scatter.
#include "pic_kernels.h"

namespace {

__global__ void k_pack(const int32_t *ix, const int32_t *iy, uint32_t *cell, int n, int xlo, int xhi,
                       int ny, unsigned *err) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int x = ix[p], y = iy[p];
        if (x < xlo || x > xhi || y < 0 || y >= ny) {
            atomicOr(err, PIC_EF_RANGE);
            cell[p] = PIC_DEAD;
        } else {
            cell[p] = ((uint32_t)y << 16) | (uint32_t)x;
        }
    }
}

__global__ void k_unpack(const uint32_t *cell, int32_t *ix, int32_t *iy, int n) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t c = cell[p];
        ix[p] = c == PIC_DEAD ? -1 : (int)(c & 0xFFFFu);
        iy[p] = c == PIC_DEAD ? -1 : (int)(c >> 16);
    }
}

__device__ __forceinline__ int cell_key(uint32_t c, const TileGeom t, int &tile) {
    const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
    const int tx = ix / t.TX, ty = iy / t.TY;
    tile = ty * t.ntx + tx;
    return tile * (t.TX * t.TY) + (iy - ty * t.TY) * t.TX + (ix - tx * t.TX);
}

// per-cell counts and each particle's rank inside its cell (-1: removed)
__global__ void k_rank(const uint32_t *cell, const int32_t *n_src, const TileGeom t, int32_t *cell_count,
                       int32_t *rank) {
    const int n = *n_src;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t c = cell[p];
        int r = -1;
        if (c != PIC_DEAD) {
            int tile;
            r = atomicAdd(&cell_count[cell_key(c, t, tile)], 1);
        }
        rank[p] = r;
    }
}

// one CTA per tile, one thread per cell (C <= 1024): layer depth R (block
// minimum of the counts), tail offset of each cell (exclusive scan of the
// counts above R), tile total
__global__ void __launch_bounds__(1024) k_layout(const int32_t *cell_count, int C, int32_t *cell_off,
                                                 int32_t *tile_R, int32_t *tile_total) {
    __shared__ int32_t wmin[32], wsum[32];
    const int t = blockIdx.x, c = threadIdx.x, lane = c & 31, wid = c >> 5, nw = (C + 31) >> 5;
    const int cnt = cell_count[(size_t)t * C + c];
    int m = cnt;
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if (lane == 0) wmin[wid] = m;
    __syncthreads();
    int R = wmin[0];
    for (int w = 1; w < nw; ++w) R = min(R, wmin[w]);
    const int ex = cnt - R;
    int incl = ex;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; ++w) base += wsum[w];
    cell_off[(size_t)t * C + c] = base + incl - ex;
    if (c == C - 1) {
        tile_R[t] = R;
        tile_total[t] = R * C + base + incl;
    }
}

// exclusive scan of count[0..nt) into start[0..nt], cursor = start; one CTA
__global__ void __launch_bounds__(1024) k_scan(const int32_t *count, int nt, int32_t *start,
                                               int32_t *cursor, int32_t *n_out) {
    __shared__ int32_t part[1024];
    const int per = (nt + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(b + per, nt);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        cursor[i] = run;
        run += count[i];
    }
    if (threadIdx.x == blockDim.x - 1) {
        start[nt] = part[threadIdx.x];
        *n_out = part[threadIdx.x];
    }
}

template <typename R>
__global__ void k_scatter(const DevSpecies<R> src, const DevSpecies<R> dst, const TileGeom t,
                          const int32_t *rank, const int32_t *tile_start, const int32_t *tile_R,
                          const int32_t *cell_off) {
    const int n = *src.n;
    const int C = t.TX * t.TY;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int r = rank[p];
        if (r < 0) continue;
        const uint32_t c = src.cell[p];
        int tile;
        const int key = cell_key(c, t, tile);
        const int lc = key - tile * C, R = tile_R[tile];
        const int pos = tile_start[tile] + (r < R ? r * C + lc : R * C + cell_off[key] + (r - R));
        dst.cell[pos] = c;
        dst.ox[pos] = src.ox[p];
        dst.oy[pos] = src.oy[p];
        dst.ux[pos] = src.ux[p];
        dst.uy[pos] = src.uy[p];
        dst.uz[pos] = src.uz[p];
        dst.sx[pos] = src.sx[p];
        dst.sy[pos] = src.sy[p];
        dst.sz[pos] = src.sz[p];
        dst.w[pos] = src.w[p];
        dst.id[pos] = src.id[p];
    }
}

int grid_for(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b);
}

}  // namespace

cudaError_t launch_pack_cells(const int32_t *ix, const int32_t *iy, uint32_t *cell, int n, int xlo,
                              int xhi, int ny, unsigned *err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_pack<<<grid_for(n), 256, 0, st>>>(ix, iy, cell, n, xlo, xhi, ny, err);
    return cudaGetLastError();
}

cudaError_t launch_unpack_cells(const uint32_t *cell, int32_t *ix, int32_t *iy, int n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_unpack<<<grid_for(n), 256, 0, st>>>(cell, ix, iy, n);
    return cudaGetLastError();
}

// n_upper bounds the source count (sizes the grids); the device counter
// *src.n is read by the kernels and replaced by the sorted count at the end.
// Scratch: cell_count and cell_off [ntiles * C], tile_R and tile_total
// [ntiles], rank [n_upper].
template <typename R>
cudaError_t launch_tile_sort(const DevSpecies<R> &src, const DevSpecies<R> &dst, const TileGeom &t,
                             const SortScratch &w, int32_t *tile_start, int32_t *n_tmp, int n_upper,
                             cudaStream_t st) {
    const int nt = t.ntx * t.nty, C = t.TX * t.TY;
    cudaError_t e = cudaMemsetAsync(w.cell_count, 0, sizeof(int32_t) * (size_t)nt * C, st);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n_upper);
    k_rank<<<g, 256, 0, st>>>(src.cell, src.n, t, w.cell_count, w.rank);
    k_layout<<<nt, C, 0, st>>>(w.cell_count, C, w.cell_off, w.tile_R, w.tile_total);
    k_scan<<<1, 1024, 0, st>>>(w.tile_total, nt, tile_start, w.cursor, n_tmp);
    k_scatter<R><<<g, 256, 0, st>>>(src, dst, t, w.rank, tile_start, w.tile_R, w.cell_off);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(const_cast<int32_t *>(src.n), n_tmp, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
}

template cudaError_t launch_tile_sort<float>(const DevSpecies<float> &, const DevSpecies<float> &,
                                             const TileGeom &, const SortScratch &, int32_t *, int32_t *, int,
                                             cudaStream_t);
template cudaError_t launch_tile_sort<double>(const DevSpecies<double> &, const DevSpecies<double> &,
                                              const TileGeom &, const SortScratch &, int32_t *, int32_t *, int,
                                              cudaStream_t);

// element-wise precision conversion (host transfers of the FP64 instantiation)
namespace {
template <typename A, typename B>
__global__ void k_convert(const A *src, B *dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}
}  // namespace

template <typename A, typename B>
cudaError_t launch_convert(const A *src, B *dst, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_convert<A, B><<<152 * 8, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
template cudaError_t launch_convert<float, double>(const float *, double *, size_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double *, float *, size_t, cudaStream_t);
