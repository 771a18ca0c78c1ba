// k_sort.cu -- a7: counting sort of the particles of one species by tile,
// laid out in layers inside each tile.  Removed particles are dropped.
//
// With C cells per tile and R = the smallest particle count of any cell of
// the tile, slot r * C + c of the tile holds the r-th particle of local cell c
// for r < R (every cell has at least R, so the layers have no holes).  The
// remaining particles follow in a tail: first L depth layers (2D3V: L = 3),
// layer d holding the (R + d)-th particle of every cell that has more than
// R + d, in cell order, so a warp's 32 consecutive slots hold particles of 32
// distinct cells of one or two rows; then the rest, cell by cell, dealt into
// a few interleaved runs, so that a warp's lanes rarely share a cell there
// either (3D3V: the whole tail, L = 0; after some motion most 3D3V tiles have
// an empty cell, R = 0, and the whole tile is tail).  A CTA of C (or a divisor
// of C) threads walking the tile meets the same cell on every pass through
// the full layers, which the 2D3V fused kernel uses to sum the in-cell
// currents in registers.  Steps: rank of each particle in its cell
// (atomics), per-tile layout (block minimum and scans over the cells),
// exclusive scan of the tile totals, scatter.  The 2D3V and 3D3V layouts
// differ in the cell packing, the tile key and the tail.
#include "pic_device3.cuh"
#include "pic_kernels.h"

namespace {

__global__ void k_pack(const int32_t *ix, const int32_t *iy, uint32_t *cell, int n, int xlo, int xhi,
                       int ny, unsigned *err) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
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
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = cell[p];
        ix[p] = c == PIC_DEAD ? -1 : (int)(c & 0xFFFFu);
        iy[p] = c == PIC_DEAD ? -1 : (int)(c >> 16);
    }
}

__global__ void k_pack3(const int32_t *ix, const int32_t *iy, const int32_t *iz, uint32_t *cell, int n, int xlo,
                        int xhi, int ny, int nz, unsigned *err) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int x = ix[p], y = iy[p], z = iz[p];
        if (x < xlo || x > xhi || y < 0 || y >= ny || z < 0 || z >= nz) {
            atomicOr(err, PIC_EF_RANGE);
            cell[p] = PIC_DEAD;
        } else {
            cell[p] = pack_cell3(x, y, z);
        }
    }
}

// Host particle arrays read in place (pinned, device-mapped memory) over the
// host link and written into a particle buffer: cells packed and range
// checked as k_pack / k_pack3 do, records converted to the buffer's real type.
template <typename HostT, typename R, bool D3>
__global__ void k_upload(const UploadSrc<HostT> s, const SortArrays<R> d, int n, int xlo, int xhi, int ny, int nz,
                         unsigned *err) {
    constexpr int NF = D3 ? 10 : 9;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int x = s.ix[p], y = s.iy[p], z = D3 ? s.iz[p] : 0;
        const bool bad = x < xlo || x > xhi || y < 0 || y >= ny || (D3 && (z < 0 || z >= nz));
        if (bad) atomicOr(err, PIC_EF_RANGE);
        d.cell[p] = bad ? PIC_DEAD : (D3 ? pack_cell3(x, y, z) : (((uint32_t)y << 16) | (uint32_t)x));
#pragma unroll
        for (int k = 0; k < NF; ++k) d.f[k][p] = (R)s.f[k][p];
        d.id[p] = s.id[p];
    }
}

__global__ void k_unpack3(const uint32_t *cell, int32_t *ix, int32_t *iy, int32_t *iz, int n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = cell[p];
        int x = -1, y = -1, z = -1;
        if (c != PIC_DEAD) unpack_cell3(c, x, y, z);
        ix[p] = x;
        iy[p] = y;
        iz[p] = z;
    }
}

// sort key of a packed cell: global index of (tile, cell inside the tile).
// Tile sizes are powers of two, so the key is shifts and masks.
__host__ __device__ constexpr int log2i(int v) { return v <= 1 ? 0 : 1 + log2i(v >> 1); }

struct Key2 {
    // the tail: three depth layers (config 3's fused kernel 1.552 -> 1.520 ms
    // against the whole tail dealt, 39.6 -> 40.3 G particle-steps/s; two: the
    // same), then the rest dealt into eight runs
    static constexpr int kTailLayers = 3;
    static constexpr int kTailRuns = 8;
    int sx, sy, ntx, nt;  // log2 of the tile sizes, tiles along x, tiles
    explicit Key2(const TileGeom &t) : sx(log2i(t.TX)), sy(log2i(t.TY)), ntx(t.ntx), nt(t.ntx * t.nty) {}
    __device__ __forceinline__ int operator()(uint32_t c, int &tile) const {
        const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
        tile = (iy >> sy) * ntx + (ix >> sx);
        return (tile << (sx + sy)) | ((iy & ((1 << sy) - 1)) << sx) | (ix & ((1 << sx) - 1));
    }
    int cells() const { return 1 << (sx + sy); }
    int tiles() const { return nt; }
    int ntiles_x() const { return ntx; }
};

struct Key3 {
    // the whole tail dealt into four runs: depth layers left config 2's fused
    // kernel unchanged (3.815 ms with three layers or none) and cost 0.3 ms a sort
    static constexpr int kTailLayers = 0;
    static constexpr int kTailRuns = 4;
    int sx, sy, sz, ntx, nty, nt;
    explicit Key3(const TileGeom3 &t)
        : sx(log2i(t.TX)), sy(log2i(t.TY)), sz(log2i(t.TZ)), ntx(t.ntx), nty(t.nty), nt(t.ntx * t.nty * t.ntz) {}
    __device__ __forceinline__ int operator()(uint32_t c, int &tile) const {
        int ix, iy, iz;
        unpack_cell3(c, ix, iy, iz);
        tile = ((iz >> sz) * nty + (iy >> sy)) * ntx + (ix >> sx);
        int ly = iy & ((1 << sy) - 1);
        // 16-wide tiles: rows in the order 0, 2, 1, 3 (of each group of four),
        // so the two rows a warp's 32 cells span lie 2 rows (48 floats) apart
        // in the field window, 16 banks, and their loads do not collide
        if (sx == 4 && sy >= 2) ly = (ly & ~3) | ((ly & 1) << 1) | ((ly >> 1) & 1);
        const int local = ((((iz & ((1 << sz) - 1)) << sy) | ly) << sx) | (ix & ((1 << sx) - 1));
        return (tile << (sx + sy + sz)) | local;
    }
    int cells() const { return 1 << (sx + sy + sz); }
    int tiles() const { return nt; }
    int ntiles_x() const { return ntx; }
};

// per-cell counts and each particle's rank inside its cell (-1: removed)
template <class K>
__global__ void k_rank(const uint32_t *cell, const int32_t *n_src, const K key, int32_t *cell_count,
                       int32_t *rank) {
    const int n = *n_src;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = cell[p];
        int r = -1;
        if (c != PIC_DEAD) {
            int tile;
            r = atomicAdd(&cell_count[key(c, tile)], 1);
        }
        rank[p] = r;
    }
}

// one CTA per tile, one thread per cell (C <= 1024, a multiple of 32): the
// full layers' depth R (block minimum of the counts); the tail's L depth
// layers (layer d: the cells with more than R + d particles, an exclusive
// scan over the cells each) and the rest (counts above R + L, an exclusive
// scan).  Per cell: its places in the L layers, 10 bits each, written over
// its count in cell_count, and its offset in the rest (cell_off).  Per tile
// (tile_info, kTileInfo entries): R, the tile's particle count, the rest's
// size and start, the layers' starts.
template <int L>
__global__ void __launch_bounds__(1024) k_layout(int32_t *cell_count, int C, int32_t *cell_off, int32_t *tile_info,
                                                 int32_t *tile_total, BinSort bins) {
    static_assert(L >= 0 && L <= 3 && 4 + L <= kTileInfo, "three 10-bit places per cell, kTileInfo entries");
    __shared__ int32_t wmin[32], wsum[L + 1][32];
    const int t = blockIdx.x, c = threadIdx.x, lane = c & 31, wid = c >> 5, nw = (C + 31) >> 5;
    const size_t at = (size_t)t * C + c;
    const int cnt = cell_count[at];
    int m = cnt;
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if (lane == 0) wmin[wid] = m;
    __syncthreads();
    int R = wmin[0];
    for (int w = 1; w < nw; ++w) R = min(R, wmin[w]);
    const int ex = cnt - R;
    // v[q < L]: the cell has a particle in tail layer q; v[L]: its particles after them
    int v[L + 1], incl[L + 1];
#pragma unroll
    for (int q = 0; q <= L; ++q) {
        v[q] = q < L ? (ex > q ? 1 : 0) : max(ex - L, 0);
        incl[q] = v[q];  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xFFFFFFFFu, incl[q], o);
            if (lane >= o) incl[q] += u;
        }
        if (lane == 31) wsum[q][wid] = incl[q];
    }
    __syncthreads();
    int base[L + 1], tot[L + 1];
#pragma unroll
    for (int q = 0; q <= L; ++q) {
        base[q] = tot[q] = 0;
        for (int w = 0; w < nw; ++w) {
            const int ws = wsum[q][w];
            base[q] += w < wid ? ws : 0;
            tot[q] += ws;
        }
    }
    uint32_t places = 0;
#pragma unroll
    for (int q = 0; q < L; ++q) places |= (uint32_t)(base[q] + incl[q] - v[q]) << (10 * q);
    cell_count[at] = (int32_t)places;
    cell_off[at] = base[L] + incl[L] - v[L];
    int lstart = 0;
#pragma unroll
    for (int q = 0; q < L; ++q) lstart += tot[q];
    const int total = R * C + lstart + tot[L];
    if (c == 0) {
        int32_t *ti = tile_info + (size_t)t * kTileInfo;
        ti[0] = R;
        ti[1] = total;
        ti[2] = tot[L];
        ti[3] = lstart;
        int ls = 0;
#pragma unroll
        for (int q = 0; q < L; ++q) {
            ti[4 + q] = ls;
            ls += tot[q];
        }
    }
    if (c == C - 1) {
        if (bins.cnt_to) {
            // binned layout: the range holds the tile's particles (one front
            // segment) and its spare slots; the range after the last tile is
            // the overflow range
            const int nr = gridDim.x + 1;
            bins.cnt_to[t] = total;
            bins.cnt_to[nr + t] = total;
            bins.cnt_to[2 * nr + t] = 0;
            const int spare = max(bins.extra, (int)((long long)total * bins.pct / 100));
            tile_total[t] = (total + spare + 7) / 8 * 8;
            if (t == 0) {
                bins.cnt_to[gridDim.x] = bins.cnt_to[nr + gridDim.x] = bins.cnt_to[2 * nr + gridDim.x] = 0;
                tile_total[gridDim.x] = bins.ovf_cap;
            }
        } else {
            tile_total[t] = total;
        }
    }
}

// exclusive scan of count[0..nt) into start[0..nt] (start[nt] and *n_out =
// the total) in three passes: each block scans a chunk of kScanChunk counts and
// keeps its total, one block scans the totals, each block adds its offset
constexpr int kScanThreads = 1024, kScanPer = 4, kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int &block_total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    block_total = warp_tot[(blockDim.x >> 5) - 1];
    const int base = wid ? warp_tot[wid - 1] : 0;
    __syncthreads();
    return base + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const int32_t *count, int nt, int32_t *start,
                                                             int32_t *chunk_tot) {
    __shared__ int warp_tot[32];
    const int b0 = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = b0 + k < nt ? count[b0 + k] : 0;
        s += v[k];
    }
    int tot;
    int run = block_exclusive_scan(s, warp_tot, tot);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (b0 + k < nt) start[b0 + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) chunk_tot[blockIdx.x] = tot;
}

// exclusive scan of the chunk totals (at most kScanChunk of them), one block
__global__ void __launch_bounds__(kScanThreads) k_scan_totals(int32_t *chunk_tot, int nchunks, int32_t *start, int nt,
                                                             int32_t *n_out) {
    __shared__ int warp_tot[32];
    const int b0 = threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = b0 + k < nchunks ? chunk_tot[b0 + k] : 0;
        s += v[k];
    }
    int tot;
    int run = block_exclusive_scan(s, warp_tot, tot);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (b0 + k < nchunks) chunk_tot[b0 + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) {
        start[nt] = tot;
        *n_out = tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t *start, int nt, const int32_t *chunk_off) {
    const int off = chunk_off[blockIdx.x];
    const int b0 = blockIdx.x * kScanChunk;
    for (int i = threadIdx.x; i < kScanChunk && b0 + i < nt; i += blockDim.x) start[b0 + i] += off;
}

cudaError_t scan_tiles(const int32_t *count, int nt, int32_t *start, int32_t *scratch, int32_t *n_out,
                       cudaStream_t st) {
    const int nchunks = (nt + kScanChunk - 1) / kScanChunk;
    if (nchunks > kScanChunk) return cudaErrorInvalidValue;  // more than 16.7M tiles
    k_scan_chunks<<<nchunks, kScanThreads, 0, st>>>(count, nt, start, scratch);
    k_scan_totals<<<1, kScanThreads, 0, st>>>(scratch, nchunks, start, nt, n_out);
    k_scan_add<<<nchunks, kScanThreads, 0, st>>>(start, nt, scratch);
    return cudaGetLastError();
}

// slot of the r-th particle of cell `key` within its tile's range, from the
// tile's layout (k_layout: tile_info, the cell's places in the tail layers
// in cell_pos, its offset in the rest in cell_off)
template <class K>
__device__ __forceinline__ int slot_in_tile(int key, int tile, int r, const int32_t *tile_info, const int32_t *cell_off,
                                            const int32_t *cell_pos, int C) {
    constexpr int L = K::kTailLayers;
    const int32_t *ti = tile_info + (size_t)tile * kTileInfo;
    const int Rl = ti[0];
    if (r < Rl) return r * C + key - tile * C;
    const int d = r - Rl;
    if (d < L) return Rl * C + ti[4 + d] + (int)(((uint32_t)cell_pos[key] >> (10 * d)) & 1023u);
    int i = cell_off[key] + (d - L);  // place in the rest, cell by cell
    // the rest dealt into S interleaved runs, so that the particles of one
    // cell (consecutive there) land in different warps and a warp's lanes
    // rarely share a cell: their shared-memory atomics then do not collide on
    // one address.  Measured fastest for the whole tail: S = 4 of 2, 3, 4, 6,
    // 8, 16 for 3D3V at 2 per cell, S = 8 of 2, 4, 8 for 2D3V at 8 + 8 per
    // cell (a fifth off its fused kernel)
    constexpr int S = K::kTailRuns;
    const int T = ti[2];
    if (T >= 64 * S) {
        const int m = i % S, q = i / S;
        i = m * (T / S) + min(m, T % S) + q;
    }
    return Rl * C + ti[3] + i;
}

// every particle to its slot; range: nullptr (all *src.n slots) or a device
// pair [range[0], range[1]) of source slots
template <typename R, int NF, class K>
__global__ void k_scatter(const SortArrays<R> src, const SortArrays<R> dst, const K kf, const int32_t *rank,
                          const int32_t *tile_start, const int32_t *tile_info, const int32_t *cell_off,
                          const int32_t *cell_pos, int C, const int32_t *range) {
    const long long p0 = range ? range[0] : 0, n = range ? range[1] : *src.n;
    for (long long p = p0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int r = rank[p];
        if (r < 0) continue;
        const uint32_t c = src.cell[p];
        int tile;
        const int key = kf(c, tile);
        const int pos = tile_start[tile] + slot_in_tile<K>(key, tile, r, tile_info, cell_off, cell_pos, C);
        dst.cell[pos] = c;
#pragma unroll
        for (int k = 0; k < NF; ++k) dst.f[k][pos] = src.f[k][p];
        dst.id[pos] = src.id[p];
    }
}

// Re-bin of a sealed binned source, one CTA per tile t: the particles of its
// source range (old_start, relabelled by txo) go into shared memory at their
// slots, and the tile's new range is written in slot order (coalesced).  A
// tile with more than cap particles, or a particle of another tile (none in
// a sealed binned layout), is written directly.  Slots the CTA did not fill
// (the tile's particles in the overflow range, scattered after this kernel)
// are not written.
// (no cell word takes this value: 3D3V needs nz <= 1020, 2D3V ix, iy < 2^15)
constexpr uint32_t kSlotEmpty = 0xFFFFFFFEu;

template <typename R, int NF, class K>
__global__ void __launch_bounds__(256) k_scatter_tiles(const SortArrays<R> src, const SortArrays<R> dst, const K kf,
                                                       const int32_t *rank, const int32_t *old_start, int txo,
                                                       int ntx, const int32_t *tile_start, const int32_t *tile_info,
                                                       const int32_t *cell_off, const int32_t *cell_pos, int C,
                                                       int cap) {
    extern __shared__ __align__(16) unsigned char sm_rec[];
    uint32_t *scell = reinterpret_cast<uint32_t *>(sm_rec);
    int32_t *sid = reinterpret_cast<int32_t *>(scell + cap);
    R *sf = reinterpret_cast<R *>(sid + cap);  // cap is a multiple of 4: 16-byte aligned
    const int t = blockIdx.x, tx = t % ntx;
    const int r = t - tx + bin_rot_x(tx, ntx, txo);
    const int os = old_start[r], oe = old_start[r + 1];
    const int ns = tile_start[t];
    const int cnt = tile_info[(size_t)t * kTileInfo + 1];
    const bool staged = cnt <= cap;
    if (staged)
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) scell[j] = kSlotEmpty;
    __syncthreads();
    for (int i = os + threadIdx.x; i < oe; i += blockDim.x) {
        const int rk = rank[i];
        if (rk < 0) continue;
        const uint32_t c = src.cell[i];
        int tile;
        const int key = kf(c, tile);
        const int pos = slot_in_tile<K>(key, tile, rk, tile_info, cell_off, cell_pos, C);
        if (staged && tile == t) {
            scell[pos] = c;
            sid[pos] = src.id[i];
#pragma unroll
            for (int k = 0; k < NF; ++k) sf[k * cap + pos] = src.f[k][i];
        } else {
            const int g = tile_start[tile] + pos;
            dst.cell[g] = c;
            dst.id[g] = src.id[i];
#pragma unroll
            for (int k = 0; k < NF; ++k) dst.f[k][g] = src.f[k][i];
        }
    }
    if (!staged) return;
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const uint32_t c = scell[j];
        if (c == kSlotEmpty) continue;
        dst.cell[ns + j] = c;
        dst.id[ns + j] = sid[j];
#pragma unroll
        for (int k = 0; k < NF; ++k) dst.f[k][ns + j] = sf[k * cap + j];
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

cudaError_t launch_pack_cells3(const int32_t *ix, const int32_t *iy, const int32_t *iz, uint32_t *cell, int n,
                               int xlo, int xhi, int ny, int nz, unsigned *err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_pack3<<<grid_for(n), 256, 0, st>>>(ix, iy, iz, cell, n, xlo, xhi, ny, nz, err);
    return cudaGetLastError();
}

cudaError_t launch_unpack_cells3(const uint32_t *cell, int32_t *ix, int32_t *iy, int32_t *iz, int n,
                                 cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_unpack3<<<grid_for(n), 256, 0, st>>>(cell, ix, iy, iz, n);
    return cudaGetLastError();
}

template <typename HostT, typename R>
cudaError_t launch_upload(const UploadSrc<HostT> &src, const SortArrays<R> &dst, int n, int xlo, int xhi, int ny,
                          int nz, bool d3, unsigned *err, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (d3)
        k_upload<HostT, R, true><<<152 * 16, 256, 0, st>>>(src, dst, n, xlo, xhi, ny, nz, err);
    else
        k_upload<HostT, R, false><<<152 * 16, 256, 0, st>>>(src, dst, n, xlo, xhi, ny, nz, err);
    return cudaGetLastError();
}
template cudaError_t launch_upload<float, float>(const UploadSrc<float> &, const SortArrays<float> &, int, int, int,
                                                 int, int, bool, unsigned *, cudaStream_t);
template cudaError_t launch_upload<float, double>(const UploadSrc<float> &, const SortArrays<double> &, int, int, int,
                                                  int, int, bool, unsigned *, cudaStream_t);
template cudaError_t launch_upload<double, float>(const UploadSrc<double> &, const SortArrays<float> &, int, int, int,
                                                  int, int, bool, unsigned *, cudaStream_t);
template cudaError_t launch_upload<double, double>(const UploadSrc<double> &, const SortArrays<double> &, int, int,
                                                   int, int, int, bool, unsigned *, cudaStream_t);

// Binned layout, per range r of each species:
//  - counters: record the range's arrival base for the next step and clear
//    the other buffer's front / split / back counters;
//  - fill: write PIC_DEAD into the slots of the range outside its two
//    segments (slot-wise kernels then read the layout as a compact one with
//    holes; the binned step itself reads only the segments).
__device__ __forceinline__ void bin_counters(const SealSpecies &S, int nr, int r, volatile int *alert) {
    const BinRange b = bin_range(S.tile_start, S.cnt_new, nr, r);
    S.cnt_new[3 * nr + r] = b.beg + b.len;
    if (S.cnt_zero) S.cnt_zero[r] = S.cnt_zero[nr + r] = S.cnt_zero[2 * nr + r] = 0;
    // the overflow range (the last one) past half full: ask for a re-bin
    if (alert && r == nr - 1 && 2 * b.len > S.tile_start[r + 1] - b.beg) *alert = 1;
}

// fill (and counters): one warp per tile range; the overflow range (the last,
// a quarter of the particles or more) shared by the warps of kSealOvfBlocks
// blocks after those of the tile ranges, so that no single warp walks it
constexpr int kSealOvfBlocks = 64;

__global__ void __launch_bounds__(256) k_seal_bins(const SealArgs a) {
    const int nr = a.nranges, lane = threadIdx.x & 31, wb = (nr - 1 + 7) / 8;
    int r, g = 0, G = 1;  // range, this warp's share of it, warps sharing it
    if ((int)blockIdx.x < wb) {
        r = blockIdx.x * 8 + (threadIdx.x >> 5);
        if (r >= nr - 1) return;
    } else {
        r = nr - 1;
        g = (blockIdx.x - wb) * 8 + (threadIdx.x >> 5);
        G = (gridDim.x - wb) * 8;
    }
    const int off = 32 * g + lane, stride = 32 * G;
    for (int s = 0; s < a.nsp; ++s) {
        const SealSpecies &S = a.sp[s];
        const BinRange b = bin_range(S.tile_start, S.cnt_new, nr, r);
        const int end = S.tile_start[r + 1], back_end = b.beg + b.split + (b.len - b.front);
        for (int i = b.beg + b.front + off; i < b.beg + b.split; i += stride) S.cell[i] = PIC_DEAD;
        for (int i = back_end + off; i < end; i += stride) S.cell[i] = PIC_DEAD;
        if (g == 0 && lane == 0 && a.counters) bin_counters(S, nr, r, a.ovf_alert);
    }
}

// counters alone: one thread per range
__global__ void __launch_bounds__(256) k_bin_counters(const SealArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.nranges) return;
    for (int s = 0; s < a.nsp; ++s) bin_counters(a.sp[s], a.nranges, r, a.ovf_alert);
}

cudaError_t launch_seal_bins(const SealArgs &a, cudaStream_t st) {
    if (a.nranges <= 0 || a.nsp <= 0 || !(a.fill || a.counters)) return cudaSuccess;
    if (a.fill)
        k_seal_bins<<<(a.nranges - 1 + 7) / 8 + kSealOvfBlocks, 256, 0, st>>>(a);
    else
        k_bin_counters<<<(a.nranges + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

namespace {
template <typename R, int NF, class K>
cudaError_t tile_sort(const SortArrays<R> &src, const SortArrays<R> &dst, const K &key, const SortScratch &w,
                      int32_t *tile_start, int32_t *n_tmp, int n_upper, const BinSort &bins, cudaStream_t st) {
    const int nt = key.tiles(), C = key.cells();
    cudaError_t e = cudaMemsetAsync(w.cell_count, 0, sizeof(int32_t) * (size_t)nt * C, st);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n_upper);
    // (one CTA a tile: a mesh of few tiles scatters faster over all slots,
    // e.g. the small runs of a batch)
    const bool tiled = bins.src_ordered && bins.old_start && nt >= 4 * 152;
    if (tiled) {
        // the source ranges, before the scan below replaces them
        e = cudaMemcpyAsync(bins.old_start, tile_start, sizeof(int32_t) * (size_t)(nt + 2), cudaMemcpyDeviceToDevice,
                            st);
        if (e != cudaSuccess) return e;
    }
    k_rank<K><<<g, 256, 0, st>>>(src.cell, src.n, key, w.cell_count, w.rank);
    k_layout<K::kTailLayers><<<nt, C, 0, st>>>(w.cell_count, C, w.cell_off, w.tile_info, w.tile_total, bins);
    e = scan_tiles(w.tile_total, bins.cnt_to ? nt + 1 : nt, tile_start, w.cursor, n_tmp, st);
    if (e != cudaSuccess) return e;
    if (tiled) {
        // tiles through shared memory (96 KB: 2 CTAs per SM), then a binned
        // source's overflow range directly
        constexpr int kRecBytes = 8 + NF * (int)sizeof(R);
        const int cap = (96 * 1024 / kRecBytes) / 4 * 4;
        const size_t smem = (size_t)cap * kRecBytes;
        static bool attr_set = false;
        if (!attr_set) {
            e = cudaFuncSetAttribute(k_scatter_tiles<R, NF, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        k_scatter_tiles<R, NF, K><<<nt, 256, smem, st>>>(src, dst, key, w.rank, bins.old_start, bins.txo,
                                                         key.ntiles_x(), tile_start, w.tile_info, w.cell_off,
                                                         w.cell_count, C, cap);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (bins.src_binned)
            k_scatter<R, NF, K><<<g, 256, 0, st>>>(src, dst, key, w.rank, tile_start, w.tile_info, w.cell_off,
                                                   w.cell_count, C, bins.old_start + nt);
    } else {
        k_scatter<R, NF, K><<<g, 256, 0, st>>>(src, dst, key, w.rank, tile_start, w.tile_info, w.cell_off,
                                               w.cell_count, C, nullptr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (bins.cnt_to) {
        // spare slots of every range -> PIC_DEAD; the source buffer's counts
        // cleared for the next binned step to count into
        SealArgs a{};
        a.nsp = 1;
        a.nranges = nt + 1;
        a.sp[0] = SealSpecies{dst.cell, tile_start, bins.cnt_to, bins.cnt_from};
        e = launch_seal_bins(a, st);
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(const_cast<int32_t *>(src.n), n_tmp, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
}

template <typename R>
SortArrays<R> arrays2(const DevSpecies<R> &S) {
    return SortArrays<R>{S.cell, {S.ox, S.oy, S.ux, S.uy, S.uz, S.sx, S.sy, S.sz, S.w, nullptr}, S.id, S.n};
}

template <typename R>
SortArrays<R> arrays3(const DevSpecies3<R> &S) {
    return SortArrays<R>{S.cell, {S.ox, S.oy, S.oz, S.ux, S.uy, S.uz, S.sx, S.sy, S.sz, S.w}, S.id, S.n};
}
}  // namespace

// n_upper bounds the source count (sizes the grids); the device counter
// *src.n is read by the kernels and replaced by the sorted count at the end.
// Scratch: cell_count and cell_off [ntiles * C], tile_info [ntiles *
// kTileInfo], tile_total [ntiles + 1], rank [n_upper].
template <typename R>
cudaError_t launch_tile_sort(const DevSpecies<R> &src, const DevSpecies<R> &dst, const TileGeom &t,
                             const SortScratch &w, int32_t *tile_start, int32_t *n_tmp, int n_upper,
                             const BinSort &order, cudaStream_t st) {
    return tile_sort<R, 9>(arrays2(src), arrays2(dst), Key2(t), w, tile_start, n_tmp, n_upper, order, st);
}

template <typename R>
cudaError_t launch_tile_sort3(const DevSpecies3<R> &src, const DevSpecies3<R> &dst, const TileGeom3 &t,
                              const SortScratch &w, int32_t *tile_start, int32_t *n_tmp, int n_upper,
                              const BinSort &bins, cudaStream_t st) {
    return tile_sort<R, 10>(arrays3(src), arrays3(dst), Key3(t), w, tile_start, n_tmp, n_upper, bins, st);
}

template cudaError_t launch_tile_sort3<float>(const DevSpecies3<float> &, const DevSpecies3<float> &,
                                              const TileGeom3 &, const SortScratch &, int32_t *, int32_t *, int,
                                              const BinSort &, cudaStream_t);
template cudaError_t launch_tile_sort3<double>(const DevSpecies3<double> &, const DevSpecies3<double> &,
                                               const TileGeom3 &, const SortScratch &, int32_t *, int32_t *, int,
                                               const BinSort &, cudaStream_t);

template cudaError_t launch_tile_sort<float>(const DevSpecies<float> &, const DevSpecies<float> &,
                                             const TileGeom &, const SortScratch &, int32_t *, int32_t *, int,
                                             const BinSort &, cudaStream_t);
template cudaError_t launch_tile_sort<double>(const DevSpecies<double> &, const DevSpecies<double> &,
                                              const TileGeom &, const SortScratch &, int32_t *, int32_t *, int,
                                              const BinSort &, cudaStream_t);

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

// ---------------------------------------------------------------------------
// co-moving window: mesh rows and particle cells slide ncells toward x_min
// ---------------------------------------------------------------------------
namespace {

// dst row r = src row r moved n columns toward x_min, zero in the uncovered
// columns (rows of ld reals, nx of them used)
template <typename R>
__global__ void k_shift_rows(const R *src, R *dst, size_t rows, int nx, int ld, int n) {
    const size_t total = rows * (size_t)ld;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % ld);
        dst[q] = i + n < nx ? src[q + n] : R(0);
    }
}

// left boundary values By(-1/2), Bz(-1/2) of the moved box: the old column n-1
template <typename R>
__global__ void k_ghost_from_column(const R *by, const R *bz, R *bnd, size_t rows, int ld, int n) {
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < rows; r += (size_t)gridDim.x * blockDim.x) {
        bnd[r] = by[r * ld + n - 1];
        bnd[rows + r] = bz[r * ld + n - 1];
    }
}

// particle cells move n cells toward x_min; cells below x = 2 are removed
template <bool D3>
__global__ void k_shift_cells(uint32_t *cell, const int32_t *n_src, int n) {
    const int np = *n_src;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = cell[p];
        if (c == PIC_DEAD) continue;
        if (D3) {
            int ix, iy, iz;
            unpack_cell3(c, ix, iy, iz);
            cell[p] = ix - n < 2 ? PIC_DEAD : pack_cell3(ix - n, iy, iz);
        } else {
            const int ix = (int)(c & 0xFFFFu) - n;
            cell[p] = ix < 2 ? PIC_DEAD : ((c & 0xFFFF0000u) | (uint32_t)ix);
        }
    }
}

}  // namespace

template <typename R>
cudaError_t launch_shift_rows(const R *src, R *dst, size_t rows, int nx, int ld, int n, cudaStream_t st) {
    k_shift_rows<R><<<152 * 8, 256, 0, st>>>(src, dst, rows, nx, ld, n);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ghost_from_column(const R *by, const R *bz, R *bnd, size_t rows, int ld, int n, cudaStream_t st) {
    k_ghost_from_column<R><<<(int)((rows + 255) / 256), 256, 0, st>>>(by, bz, bnd, rows, ld, n);
    return cudaGetLastError();
}

cudaError_t launch_shift_cells(uint32_t *cell, const int32_t *n_src, int n_upper, int ncells, bool d3,
                               cudaStream_t st) {
    if (n_upper == 0) return cudaSuccess;
    if (d3)
        k_shift_cells<true><<<grid_for(n_upper), 256, 0, st>>>(cell, n_src, ncells);
    else
        k_shift_cells<false><<<grid_for(n_upper), 256, 0, st>>>(cell, n_src, ncells);
    return cudaGetLastError();
}

template cudaError_t launch_shift_rows<float>(const float *, float *, size_t, int, int, int, cudaStream_t);
template cudaError_t launch_shift_rows<double>(const double *, double *, size_t, int, int, int, cudaStream_t);
template cudaError_t launch_ghost_from_column<float>(const float *, const float *, float *, size_t, int, int,
                                                     cudaStream_t);
template cudaError_t launch_ghost_from_column<double>(const double *, const double *, double *, size_t, int, int,
                                                      cudaStream_t);

// ---------------------------------------------------------------------------
// co-moving window on the stepping path (no host synchronisation)
// ---------------------------------------------------------------------------
namespace {

// Every mesh row moved n columns toward x_min in place, the uncovered columns
// zero; one warp per row.  The warp reads a group of 256 columns into
// registers before it writes them n columns lower, and the groups run in
// increasing x, so every column is read before anything overwrites it.  The
// left boundary values By(-1/2), Bz(-1/2) become the old column n - 1 of By
// and Bz (read before the row moves).
constexpr int kRowGroup = 8;  // columns a lane moves per group (256 a warp)

template <typename R>
__global__ void __launch_bounds__(256) k_window_rows(const WindowRows<R> a) {
    const int lane = threadIdx.x & 31;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    const size_t total = a.rows * (size_t)a.nplanes;
    for (size_t wq = blockIdx.x * (size_t)(blockDim.x >> 5) + (threadIdx.x >> 5); wq < total; wq += warps) {
        const int pl = (int)(wq / a.rows);
        const size_t r = wq - (size_t)pl * a.rows;
        R *row = a.plane[pl] + r * a.ld;
        if (lane == 0 && a.bnd && (pl == a.by || pl == a.bz)) a.bnd[(pl == a.by ? 0 : a.rows) + r] = row[a.n - 1];
        __syncwarp();
        for (int x0 = 0; x0 < a.nx; x0 += 32 * kRowGroup) {
            R v[kRowGroup];
#pragma unroll
            for (int k = 0; k < kRowGroup; ++k) {
                const int x = x0 + 32 * k + lane;
                v[k] = x + a.n < a.nx ? row[x + a.n] : R(0);
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < kRowGroup; ++k) {
                const int x = x0 + 32 * k + lane;
                if (x < a.nx) row[x] = v[k];
            }
            __syncwarp();
        }
    }
}

// Binned layout: the ranges of the tile columns the move uncovered at x_max
// (the last kt columns; the particles they held have all left the box) are
// emptied: front, split and back zero in the current buffer's counters.
// txo is the relabelling after the move (range of tile (tx, ty, tz) = that of
// tile ((tx + txo) mod ntx, ty, tz)).
__global__ void k_window_vacate(int32_t *cnt, int nr, int ntx, int nyz, int kt, int txo) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kt * nyz) return;
    const int yz = j / kt, tx = ntx - kt + (j - yz * kt);
    const int r = yz * ntx + bin_rot_x(tx, ntx, txo);
    cnt[r] = cnt[nr + r] = cnt[2 * nr + r] = 0;
}

// Binned layout: each staged particle is appended to the arrival segment of
// its tile's range (slot beg + split + back, back counted up), or, when that
// range is full, to the overflow range's; with both full it is dropped and
// PIC_EF_BINS raised.  The arrival bases are recomputed afterwards.
template <typename R>
__global__ void k_window_inject3(const SortArrays<R> src, const SortArrays<R> dst, const int32_t *tile_start,
                                 int32_t *cnt, const TileGeom3 t, int txo, unsigned *err) {
    const int m = *src.n;
    const int nt = t.ntx * t.nty * t.ntz, nr = nt + 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = src.cell[i];
        if (c == PIC_DEAD) continue;
        int ix, iy, iz;
        unpack_cell3(c, ix, iy, iz);
        const int r = ((iz / t.TZ) * t.nty + iy / t.TY) * t.ntx + bin_rot_x(ix / t.TX, t.ntx, txo);
        int slot = tile_start[r] + cnt[nr + r] + atomicAdd(&cnt[2 * nr + r], 1);
        if (slot >= tile_start[r + 1]) {
            slot = tile_start[nt] + cnt[nr + nt] + atomicAdd(&cnt[2 * nr + nt], 1);
            if (slot >= tile_start[nt + 1]) {
                atomicOr(err, PIC_EF_BINS);
                continue;
            }
        }
        dst.cell[slot] = c;
#pragma unroll
        for (int k = 0; k < 10; ++k) dst.f[k][slot] = src.f[k][i];
        dst.id[slot] = src.id[i];
    }
}

// Compact layout: the staged particles appended after the *n_dst slots in use
// (nf reals a record), or, when they do not fit the capacity, nothing and
// PIC_EF_CAP; k_window_count then adds the count.
template <typename R, int NF>
__global__ void k_window_append(const SortArrays<R> src, const SortArrays<R> dst, const int32_t *n_dst, int cap,
                                unsigned *err) {
    const int m = *src.n, n0 = *n_dst;
    if ((long long)n0 + m > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, PIC_EF_CAP);
        return;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const long long slot = n0 + i;
        dst.cell[slot] = src.cell[i];
#pragma unroll
        for (int k = 0; k < NF; ++k) dst.f[k][slot] = src.f[k][i];
        dst.id[slot] = src.id[i];
    }
}

__global__ void k_window_count(int32_t *n_dst, const int32_t *m_src, int cap) {
    const long long n = (long long)*n_dst + *m_src;
    if (n <= cap) *n_dst = (int32_t)n;
}

// Live particles into host-mapped memory: the compact layout's count
// (*n_dev), or the sum of the binned ranges' lengths (tile ranges and the
// overflow range; removed particles still inside a segment count too, so it
// is a bound).  One block.
__global__ void __launch_bounds__(1024) k_live_sample(const int32_t *n_dev, const int32_t *tile_start,
                                                      const int32_t *cnt, int nr, volatile long long *out) {
    __shared__ long long part[32];
    long long s = 0;
    if (tile_start)
        for (int r = threadIdx.x; r < nr; r += blockDim.x) s += bin_range(tile_start, cnt, nr, r).len;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        *out = tile_start ? tot : (long long)*n_dev;
        __threadfence_system();
    }
}

}  // namespace

template <typename R>
cudaError_t launch_window_rows(const WindowRows<R> &a, cudaStream_t st) {
    if (a.rows == 0 || a.nplanes <= 0) return cudaSuccess;
    if (a.n < 1 || a.n > a.nx) return cudaErrorInvalidValue;
    k_window_rows<R><<<152 * 16, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_window_vacate(int32_t *cnt, int nr, int ntx, int nyz, int kt, int txo, cudaStream_t st) {
    const int n = kt * nyz;
    if (n <= 0) return cudaSuccess;
    k_window_vacate<<<(n + 255) / 256, 256, 0, st>>>(cnt, nr, ntx, nyz, kt, txo);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_window_inject3(const SortArrays<R> &src, int m_upper, const SortArrays<R> &dst,
                                  const int32_t *tile_start, int32_t *cnt, const TileGeom3 &t, int txo,
                                  unsigned *err, cudaStream_t st) {
    if (m_upper <= 0) return cudaSuccess;
    k_window_inject3<R><<<grid_for(m_upper), 256, 0, st>>>(src, dst, tile_start, cnt, t, txo, err);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_window_append(const SortArrays<R> &src, int m_upper, const SortArrays<R> &dst, int32_t *n_dst,
                                 int cap, bool d3, unsigned *err, cudaStream_t st) {
    if (m_upper <= 0) return cudaSuccess;
    if (d3)
        k_window_append<R, 10><<<grid_for(m_upper), 256, 0, st>>>(src, dst, n_dst, cap, err);
    else
        k_window_append<R, 9><<<grid_for(m_upper), 256, 0, st>>>(src, dst, n_dst, cap, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_window_count<<<1, 1, 0, st>>>(n_dst, src.n, cap);
    return cudaGetLastError();
}

cudaError_t launch_live_sample(const int32_t *n_dev, const int32_t *tile_start, const int32_t *cnt, int nr,
                               volatile long long *out, cudaStream_t st) {
    k_live_sample<<<1, 1024, 0, st>>>(n_dev, tile_start, cnt, nr, out);
    return cudaGetLastError();
}

template cudaError_t launch_window_rows<float>(const WindowRows<float> &, cudaStream_t);
template cudaError_t launch_window_rows<double>(const WindowRows<double> &, cudaStream_t);
template cudaError_t launch_window_inject3<float>(const SortArrays<float> &, int, const SortArrays<float> &,
                                                  const int32_t *, int32_t *, const TileGeom3 &, int, unsigned *,
                                                  cudaStream_t);
template cudaError_t launch_window_inject3<double>(const SortArrays<double> &, int, const SortArrays<double> &,
                                                   const int32_t *, int32_t *, const TileGeom3 &, int, unsigned *,
                                                   cudaStream_t);
template cudaError_t launch_window_append<float>(const SortArrays<float> &, int, const SortArrays<float> &, int32_t *,
                                                 int, bool, unsigned *, cudaStream_t);
template cudaError_t launch_window_append<double>(const SortArrays<double> &, int, const SortArrays<double> &,
                                                  int32_t *, int, bool, unsigned *, cudaStream_t);
