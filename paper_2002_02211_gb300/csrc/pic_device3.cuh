// pic_device3.cuh -- device-side layout and per-particle arithmetic of the
// 3D3V step.  The Boris push and the Thomas-BMT rotation (Eqs. 1-3) are the
// ones of pic_device.cuh (push_spin); this header adds the 3D mesh, the
// trilinear gather at the 3D Yee positions and the 3D Esirkepov current.
//
// Particle state per species (structure of arrays, sorted by tile):
//   cell  uint32  (iz << 22) | (iy << 11) | ix, or PIC_DEAD
//   ox,oy,oz R    offsets inside the cell, [0, 1)
//   ux..w, id     as in 2D3V
// Mesh: one [6][nz][ny][ld] block of R for Ex Ey Ez Bx By Bz and one
// [3][nz][ny][ld] block for Jx Jy Jz; element (c, k, j, i) of
//   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
//   Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
#pragma once
#include "pic_device.cuh"

#define PIC3_XBITS 11
#define PIC3_YBITS 11
// largest mesh the packing holds with room for the +1 shift of the split path
#define PIC3_MAX_NX 2044
#define PIC3_MAX_NY 2044
#define PIC3_MAX_NZ 1020

__host__ __device__ __forceinline__ uint32_t pack_cell3(int ix, int iy, int iz) {
    return ((uint32_t)iz << (PIC3_XBITS + PIC3_YBITS)) | ((uint32_t)iy << PIC3_XBITS) | (uint32_t)ix;
}
__host__ __device__ __forceinline__ void unpack_cell3(uint32_t c, int &ix, int &iy, int &iz) {
    ix = (int)(c & ((1u << PIC3_XBITS) - 1));
    iy = (int)((c >> PIC3_XBITS) & ((1u << PIC3_YBITS) - 1));
    iz = (int)(c >> (PIC3_XBITS + PIC3_YBITS));
}

template <typename R>
struct DevSpecies3 {
    uint32_t *cell;
    R *ox, *oy, *oz, *ux, *uy, *uz, *sx, *sy, *sz, *w;
    int32_t *id;
    int32_t *tile_start;
    uint32_t *cell_old;            // split path: x^n kept for pic_deposit
    R *ox_old, *oy_old, *oz_old;
    R qm, q, a;
    int mobile;
    const int32_t *n;
};

template <typename R>
struct MeshParams3 {
    int nx, ny, nz, ld, bc_x;
    R dt;
    R dt_dx, dt_dy, dt_dz;         // cell units per unit velocity
    R dx_dt, dy_dt, dz_dt;         // Esirkepov current scales
    R *EB;                         // [6][nz][ny][ld]
    R *J;                          // [3][nz][ny][ld]
    size_t plane;                  // nz * ny * ld
};

struct TileGeom3 {
    int TX, TY, TZ;                // tile size in cells
    int WX, WY, WZ;                // current-window extents
    int FX;                        // field-window row pitch (TMA box width; rows WY, planes WZ)
    int HX, HY, HZ;                // window margins before the tile
    int ntx, nty, ntz;
};

// The window holds every node a particle touches ([cell-1, cell+2] along each
// axis) while its cell lies in the tile grown by PIC3_MARGIN cells along y and
// z.  Along x the margin is 4 cells before the tile (TMA: a 16-byte aligned
// start) and the row is rounded up to 16 bytes.
#ifndef PIC3_MARGIN
#define PIC3_MARGIN 0
#endif
template <typename R>
__host__ __device__ constexpr int window3_wx(int tx) {
    return (tx + 4 + 2 + (int)(16 / sizeof(R)) - 1) / (int)(16 / sizeof(R)) * (int)(16 / sizeof(R));
}
// Row pitch of the staged field window (the TMA box width): the current-window
// width, except in float with 8-cell tiles, where 24 (8 mod 32 banks apart per
// row) puts the four y rows a warp's 32 cells span in distinct bank groups.
template <typename R>
__host__ __device__ constexpr int window3_fx(int tx) {
    return sizeof(R) == 4 && tx == 8 ? 24 : window3_wx<R>(tx);
}
__host__ __device__ constexpr int window3_hx() { return 4; }
__host__ __device__ constexpr int window3_w(int t) { return t + 3 + 2 * PIC3_MARGIN; }
__host__ __device__ constexpr int window3_h() { return 1 + PIC3_MARGIN; }

// Binned layout.  Tile T owns slots [tile_start[T], tile_start[T + 1]) in
// both particle buffers; range nt (after the last tile) is the overflow range.
// In one buffer a range holds two segments: the particles that stayed in the
// tile, [beg, beg + front), and the ones that arrived from other tiles,
// [beg + split, beg + split + back), split being the range's particle count
// in the buffer it was stepped from.  Counters per buffer, nr = nt + 1
// ranges: cnt[r] front, cnt[nr + r] split, cnt[2 nr + r] back, and
// cnt[3 nr + r] = beg + front + back, the first slot a step reading this
// buffer gives to arrivals (written by the seal).  back may exceed the room
// after split (the excess went to the overflow range): readers clamp it.
template <typename R>
struct Bin3 {
    uint32_t *cell;         // destination buffer
    R *f[10];               // ox oy oz ux uy uz sx sy sz w
    int32_t *id;
    const int32_t *cnt_in;  // [4 nr] counters of the source buffer
    int32_t *cnt_out;       // [4 nr] of the destination buffer, front / split / back zero on entry
    int txo;                // tile-column relabelling of the co-moving window (bin_rot_x)
};

// The co-moving window moves the box by whole tile columns without moving a
// particle between ranges: after moves of kt columns in total since the last
// sort, tile column tx uses the ranges of column (tx + txo) mod ntx, txo = kt
// mod ntx (the columns that left the box lend their ranges to the uncovered
// ones).  txo in [0, ntx).
__host__ __device__ __forceinline__ int bin_rot_x(int tx, int ntx, int txo) {
    const int r = tx + txo;
    return r >= ntx ? r - ntx : r;
}

struct BinRange {
    int beg, front, split, len;
};

__device__ __forceinline__ BinRange bin_range(const int32_t *tile_start, const int32_t *cnt, int nr, int r) {
    BinRange b;
    b.beg = tile_start[r];
    const int cap = tile_start[r + 1] - b.beg;
    b.front = cnt[r];
    b.split = cnt[nr + r];
    b.len = b.front + max(0, min(cnt[2 * nr + r], cap - b.split));
    return b;
}

// slot of the k-th particle of a range (k < len)
__device__ __forceinline__ int bin_slot(const BinRange &b, int k) {
    return k < b.front ? b.beg + k : b.beg + b.split + (k - b.front);
}

template <typename R>
struct StepParams3 {
    MeshParams3<R> m;
    TileGeom3 t;
    int nsp;
    DevSpecies3<R> sp[PIC_MAXSP];
    unsigned *err;
    DiagParams diag;
    Bin3<R> bin[PIC_MAXSP];  // binned layout only
    int nextra;              // binned layout: CTAs of the overflow-range kernel
    int diag_cols0;          // diagnostic columns of the fused kernel's CTAs (the overflow CTAs' follow)
};

// Global-memory access to the 4 x 4 x 4 nodes [cell-1, cell+2] of one
// particle, in local coordinates 0..3: the wrapped row offsets are formed once,
// so the gather's 48 loads carry no branches between them and issue back to
// back.  A stencil that leaves the mesh (only a corrupt cell can do that) is
// flagged and clamped.
template <typename R>
struct NodeBlock3 {
    const R *EB;
    R *J;
    size_t plane;
    int ld;
    int xs[4];       // wrapped x of nodes cell-1 .. cell+2
    unsigned rs[16]; // row index z * ny + y of the 4 x 4 (y, z) node rows, [z][y]
    __device__ __forceinline__ NodeBlock3(const MeshParams3<R> &m, int ix, int iy, int iz, unsigned *err)
        : EB(m.EB), J(m.J), plane(m.plane), ld(m.ld) {
        bool bad = false;
        int ys[4], zs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int x = ix - 1 + k, y = iy - 1 + k, z = iz - 1 + k;
            if (m.bc_x == 1) x = x < 0 ? x + m.nx : (x >= m.nx ? x - m.nx : x);
            y = y < 0 ? y + m.ny : (y >= m.ny ? y - m.ny : y);
            z = z < 0 ? z + m.nz : (z >= m.nz ? z - m.nz : z);
            bad |= x < 0 || x >= m.nx || y < 0 || y >= m.ny || z < 0 || z >= m.nz;
            xs[k] = min(max(x, 0), m.nx - 1);
            ys[k] = min(max(y, 0), m.ny - 1);
            zs[k] = min(max(z, 0), m.nz - 1);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) rs[a * 4 + b] = (unsigned)zs[a] * (unsigned)m.ny + (unsigned)ys[b];
        if (bad) atomicOr(err, PIC_EF_RANGE);
    }
    __device__ __forceinline__ size_t at(int x, int y, int z) const {
        return (size_t)rs[z * 4 + y] * ld + xs[x];
    }
    __device__ __forceinline__ R f(int c, int x, int y, int z) const { return __ldg(&EB[c * plane + at(x, y, z)]); }
    __device__ __forceinline__ void j(int c, int x, int y, int z, R v) const { atomicAdd(&J[c * plane + at(x, y, z)], v); }
};

// a1 in 3D: trilinear interpolation of each component at its own Yee position
template <typename R, class M>
__device__ __forceinline__ void gather_eb3(const M &m, int ix, int iy, int iz, R ox, R oy, R oz, R E[3], R B[3]) {
    const R half = R(0.5), one = R(1);
    const bool rx = ox >= half, ry = oy >= half, rz = oz >= half;
    const int hx = rx ? ix : ix - 1, hy = ry ? iy : iy - 1, hz = rz ? iz : iz - 1;
    const R ohx = rx ? ox - half : ox + half, ohy = ry ? oy - half : oy + half, ohz = rz ? oz - half : oz + half;
    // weights: n = node-centred, h = half-shifted
    const R xn[2] = {one - ox, ox}, yn[2] = {one - oy, oy}, zn[2] = {one - oz, oz};
    const R xh[2] = {one - ohx, ohx}, yh[2] = {one - ohy, ohy}, zh[2] = {one - ohz, ohz};
    auto tri = [&](int c, int x, int y, int z, const R *a, const R *b, const R *g) {
        const R s00 = a[0] * m.f(c, x, y, z) + a[1] * m.f(c, x + 1, y, z);
        const R s10 = a[0] * m.f(c, x, y + 1, z) + a[1] * m.f(c, x + 1, y + 1, z);
        const R s01 = a[0] * m.f(c, x, y, z + 1) + a[1] * m.f(c, x + 1, y, z + 1);
        const R s11 = a[0] * m.f(c, x, y + 1, z + 1) + a[1] * m.f(c, x + 1, y + 1, z + 1);
        return g[0] * (b[0] * s00 + b[1] * s10) + g[1] * (b[0] * s01 + b[1] * s11);
    };
    E[0] = tri(0, hx, iy, iz, xh, yn, zn);   // Ex (i+1/2, j, k)
    E[1] = tri(1, ix, hy, iz, xn, yh, zn);   // Ey (i, j+1/2, k)
    E[2] = tri(2, ix, iy, hz, xn, yn, zh);   // Ez (i, j, k+1/2)
    B[0] = tri(3, ix, hy, hz, xn, yh, zh);   // Bx (i, j+1/2, k+1/2)
    B[1] = tri(4, hx, iy, hz, xh, yn, zh);   // By (i+1/2, j, k+1/2)
    B[2] = tri(5, hx, hy, iz, xh, yh, zn);   // Bz (i+1/2, j+1/2, k)
}

// ---------------------------------------------------------------------------
// a5 in 3D (Esirkepov, Comput. Phys. Commun. 135, 144, 2001):
//   Wx = dSx (S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3), Wy, Wz cyclic,
//   Jx(org+i+1/2, ., .) = -q w dx/dt sum_{i'<=i} Wx(i', ., .), likewise Jy, Jz.
// A move inside its cell, with offsets (d, e, f) and midpoint (xm, ym, zm),
// reduces to four values per component:
//   Jx(i+1/2, j+b, k+c) = q w dx/dt d F(ym, zm, e f)(b, c),
//   F(0,0) = (1-ym)(1-zm) + ef/12,  F(1,0) = ym (1-zm) - ef/12,
//   F(0,1) = (1-ym) zm - ef/12,     F(1,1) = ym zm + ef/12,
// and cyclically for Jy (x, z) and Jz (x, y).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void in_cell_weights3(R ox, R oy, R oz, R ox1, R oy1, R oz1, R qw, R dx_dt, R dy_dt,
                                                 R dz_dt, R v[12]) {
    const R one = R(1), half = R(0.5), k12 = R(1) / R(12);
    const R d = ox1 - ox, e = oy1 - oy, f = oz1 - oz;
    const R xm = ox + half * d, ym = oy + half * e, zm = oz + half * f;
    const R jx = qw * dx_dt * d, jy = qw * dy_dt * e, jz = qw * dz_dt * f;
    const R ef = e * f * k12, df = d * f * k12, de = d * e * k12;
    v[0] = jx * ((one - ym) * (one - zm) + ef);   // Jx (i+1/2, j,   k)
    v[1] = jx * (ym * (one - zm) - ef);           // Jx (i+1/2, j+1, k)
    v[2] = jx * ((one - ym) * zm - ef);           // Jx (i+1/2, j,   k+1)
    v[3] = jx * (ym * zm + ef);                   // Jx (i+1/2, j+1, k+1)
    v[4] = jy * ((one - xm) * (one - zm) + df);   // Jy (i,   j+1/2, k)
    v[5] = jy * (xm * (one - zm) - df);           // Jy (i+1, j+1/2, k)
    v[6] = jy * ((one - xm) * zm - df);           // Jy (i,   j+1/2, k+1)
    v[7] = jy * (xm * zm + df);                   // Jy (i+1, j+1/2, k+1)
    v[8] = jz * ((one - xm) * (one - ym) + de);   // Jz (i,   j,   k+1/2)
    v[9] = jz * (xm * (one - ym) - de);           // Jz (i+1, j,   k+1/2)
    v[10] = jz * ((one - xm) * ym - de);          // Jz (i,   j+1, k+1/2)
    v[11] = jz * (xm * ym + de);                  // Jz (i+1, j+1, k+1/2)
}

template <typename R, class M>
__device__ __forceinline__ void deposit_in_cell3(const M &m, int ix, int iy, int iz, const R v[12]) {
    m.j(0, ix, iy, iz, v[0]);
    m.j(0, ix, iy + 1, iz, v[1]);
    m.j(0, ix, iy, iz + 1, v[2]);
    m.j(0, ix, iy + 1, iz + 1, v[3]);
    m.j(1, ix, iy, iz, v[4]);
    m.j(1, ix + 1, iy, iz, v[5]);
    m.j(1, ix, iy, iz + 1, v[6]);
    m.j(1, ix + 1, iy, iz + 1, v[7]);
    m.j(2, ix, iy, iz, v[8]);
    m.j(2, ix + 1, iy, iz, v[9]);
    m.j(2, ix, iy + 1, iz, v[10]);
    m.j(2, ix + 1, iy + 1, iz, v[11]);
}

// general move (crosses at least one cell boundary): 3-node shapes per axis
// from shape3 (org = min(old, new) cell); planes that only hold zeros when an
// axis is not crossed are skipped.  The Esirkepov weight factors through the
// midpoint shapes M = S0 + dS/2:
//   S0y S0z + (dSy S0z + S0y dSz)/2 + dSy dSz/3 = My Mz + dSy dSz / 12,
// and the prefix sums of dSx along x are formed once, so each current value
// is one product of a prefix and a factor.
template <typename R, class M>
__device__ __forceinline__ void deposit_esirkepov3(const M &m, int ix, int iy, int iz, R ox, R oy, R oz, int ix1,
                                                   int iy1, int iz1, R ox1, R oy1, R oz1, R qw, R dx_dt, R dy_dt,
                                                   R dz_dt) {
    const R half = R(0.5), k12 = R(1) / R(12);
    R S0x[3], dSx[3], S0y[3], dSy[3], S0z[3], dSz[3];
    const int gx = shape3(ix, ox, ix1, ox1, S0x, dSx);
    const int gy = shape3(iy, oy, iy1, oy1, S0y, dSy);
    const int gz = shape3(iz, oz, iz1, oz1, S0z, dSz);
    const int nx = ix1 != ix ? 3 : 2, ny = iy1 != iy ? 3 : 2, nz = iz1 != iz ? 3 : 2;
    R Mx[3], My[3], Mz[3], Ex[3], Ey[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Mx[a] = S0x[a] + half * dSx[a];
        My[a] = S0y[a] + half * dSy[a];
        Mz[a] = S0z[a] + half * dSz[a];
        Ex[a] = k12 * dSx[a];
        Ey[a] = k12 * dSy[a];
    }
    // prefixes -q w (dx/dt) sum_{i' <= i} dSx(i'); the last one is zero
    const R cx = -qw * dx_dt, cy = -qw * dy_dt, cz = -qw * dz_dt;
    const R Px[2] = {cx * dSx[0], cx * (dSx[0] + dSx[1])};
    const R Py[2] = {cy * dSy[0], cy * (dSy[0] + dSy[1])};
    const R Pz[2] = {cz * dSz[0], cz * (dSz[0] + dSz[1])};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= nz) break;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (j >= ny) break;
            const R F = My[j] * Mz[k] + Ey[j] * dSz[k];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i >= nx - 1) break;
                m.j(0, gx + i, gy + j, gz + k, Px[i] * F);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= nz) break;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= nx) break;
            const R F = Mx[i] * Mz[k] + Ex[i] * dSz[k];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (j >= ny - 1) break;
                m.j(1, gx + i, gy + j, gz + k, Py[j] * F);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j >= ny) break;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= nx) break;
            const R F = Mx[i] * My[j] + Ex[i] * dSy[j];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (k >= nz - 1) break;
                m.j(2, gx + i, gy + j, gz + k, Pz[k] * F);
            }
        }
    }
}

// Binned layout: warp-collective store of one particle per lane into the
// range of its destination tile `dest` (-1: nothing to store).  Stayers (dest
// == tile, the storing CTA's own tile) take the next slots of the range's front
// through the CTA's shared-memory counter *s_front; arrivals take slots from
// the range's arrival base on, lanes with one destination reserving them with
// one global atomic (all destinations of the warp in one round trip).  An
// arrival past the range's end goes to the overflow range; when that is full
// too the particle is dropped and PIC_EF_BINS raised.  tile = -1 (the
// overflow-range kernel): every particle is an arrival.  front_base: the first
// slot of the tile's range when the caller holds it (else it is read from
// tile_start).  All 32 lanes of the warp must call it together.
template <typename R>
__device__ __forceinline__ void bin_store3(const Bin3<R> &B, const int32_t *tile_start, int nt, int tile,
                                           int *s_front, int dest, uint32_t cell, const R v[10], int32_t id,
                                           unsigned *err, int front_base = -1) {
    constexpr unsigned kAll = 0xFFFFFFFFu;
    const int nr = nt + 1, lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const bool stayer = dest >= 0 && dest == tile;
    int slot = -1;
    const unsigned stay = __ballot_sync(kAll, stayer);
    if (stay) {
        const int leader = __ffs(stay) - 1;
        int b = 0;
        if (lane == leader) b = atomicAdd(s_front, __popc(stay));
        b = __shfl_sync(kAll, b, leader);
        if (stayer) slot = (front_base >= 0 ? front_base : tile_start[tile]) + b + __popc(stay & below);
    }
    const int arr = dest >= 0 && !stayer ? dest : -1;
    if (__any_sync(kAll, arr >= 0)) {
        const unsigned peers = __match_any_sync(kAll, arr);
        const int leader = __ffs(peers) - 1;
        int b = 0;
        int base = 0, end = 0;
        if (arr >= 0) {
            base = B.cnt_in[3 * nr + arr];
            end = tile_start[arr + 1];
            if (lane == leader) b = atomicAdd(&B.cnt_out[2 * nr + arr], __popc(peers));
        }
        b = __shfl_sync(kAll, b, leader);
        if (arr >= 0) {
            const int s = base + b + __popc(peers & below);
            if (s < end) {
                slot = s;
            } else {
                const int ob = tile_start[nt], ocap = tile_start[nt + 1] - ob;
                const int op = atomicAdd(&B.cnt_out[2 * nr + nt], 1);
                if (op < ocap)
                    slot = ob + op;
                else
                    atomicOr(err, PIC_EF_BINS);
            }
        }
    }
    if (slot < 0) return;
    B.cell[slot] = cell;
#pragma unroll
    for (int k = 0; k < 10; ++k) B.f[k][slot] = v[k];
    B.id[slot] = id;
}
