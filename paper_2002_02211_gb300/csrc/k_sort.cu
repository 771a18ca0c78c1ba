// k_sort.cu -- a7: counting sort of the particles of one species by tile
// (histogram with warp-aggregated atomics, single-CTA exclusive scan,
// scatter into the second buffer).  Removed particles are dropped.  Within a
// tile the order is that of arrival (warp order preserved), not stable
// across warps.
#include "pic_kernels.h"

namespace {

__device__ __forceinline__ int tile_of(uint32_t c, const TileGeom t) {
    const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
    return (iy / t.TY) * t.ntx + ix / t.TX;
}

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

__global__ void k_count(const uint32_t *cell, const int32_t *n_src, const TileGeom t, int32_t *count) {
    const unsigned lane = threadIdx.x & 31u;
    const int n = *n_src;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int p = base + threadIdx.x;
        const uint32_t c = p < n ? cell[p] : PIC_DEAD;
        const int key = c == PIC_DEAD ? -1 : tile_of(c, t);
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
        const int leader = __ffs(peers) - 1;
        if (key >= 0 && (int)lane == leader) atomicAdd(&count[key], __popc(peers));
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

__global__ void k_scatter(const DevSpecies src, const DevSpecies dst, const TileGeom t,
                          int32_t *cursor) {
    const unsigned lane = threadIdx.x & 31u;
    const int n = *src.n;
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const int p = base + threadIdx.x;
        const uint32_t c = p < n ? src.cell[p] : PIC_DEAD;
        const int key = c == PIC_DEAD ? -1 : tile_of(c, t);
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
        const int leader = __ffs(peers) - 1;
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int pos = 0;
        if (key >= 0 && (int)lane == leader) pos = atomicAdd(&cursor[key], __popc(peers));
        pos = __shfl_sync(peers, pos, leader) + rank;
        if (key < 0) continue;
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
cudaError_t launch_tile_sort(const DevSpecies &src, const DevSpecies &dst, const TileGeom &t,
                             int32_t *count, int32_t *cursor, int32_t *tile_start, int32_t *n_tmp,
                             int n_upper, cudaStream_t st) {
    const int nt = t.ntx * t.nty;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * nt, st);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n_upper);
    k_count<<<g, 256, 0, st>>>(src.cell, src.n, t, count);
    k_scan<<<1, 1024, 0, st>>>(count, nt, tile_start, cursor, n_tmp);
    k_scatter<<<g, 256, 0, st>>>(src, dst, t, cursor);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(const_cast<int32_t *>(src.n), n_tmp, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
}
