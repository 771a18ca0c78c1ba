// pic_step3.cuh -- pieces of the 3D3V fused step kernels (k_particles3.cu):
// window geometry, the shared-memory mesh accessor, the a4 boundary rule, tile
// and bin destinations, the in-step Eq. (4) sums.
#pragma once
#include "pic_device3.cuh"

namespace {

// a4 boundary rule: removal at the open x ends, periodic wraps
template <typename R>
__device__ __forceinline__ bool finish_move3(const MeshParams3<R> &m, int &ix1, int &iy1, int &iz1) {
    bool alive = true;
    if (m.bc_x == 0) {
        alive = ix1 >= 2 && ix1 <= m.nx - 3;
    } else {
        if (ix1 < 0) ix1 += m.nx;
        else if (ix1 >= m.nx) ix1 -= m.nx;
    }
    if (iy1 < 0) iy1 += m.ny;
    else if (iy1 >= m.ny) iy1 -= m.ny;
    if (iz1 < 0) iz1 += m.nz;
    else if (iz1 >= m.nz) iz1 -= m.nz;
    return alive;
}

// Window geometry of a TX x TY x TZ tile: current window [3][WZ][WY][WX],
// field window [6][WZ][WY][FX], margins (HX, HY, HZ) before the tile.
template <int TX, int TY, int TZ, typename R>
struct WinConst3 {
    static constexpr int WX = window3_wx<R>(TX), WY = window3_w(TY), WZ = window3_w(TZ);
    static constexpr int WA = WX * WY * WZ;
    static constexpr int FX = window3_fx<R>(TX);
    static constexpr int FA = FX * WY * WZ;
    static constexpr int HX = window3_hx(), HY = window3_h(), HZ = window3_h();
};

template <typename R, int WX, int WY, int WA, int FX, int FA>
struct SmemMesh3T {
    const R *F;
    R *Jw;
    __device__ __forceinline__ R f(int c, int x, int y, int z) const { return F[c * FA + (z * WY + y) * FX + x]; }
    __device__ __forceinline__ void j(int c, int x, int y, int z, R v) const {
        atomicAdd(&Jw[c * WA + (z * WY + y) * WX + x], v);
    }
};

// range of the tile of cell (ix, iy, iz), tile columns relabelled by txo
// (bin_rot_x; txo = 0: the tile's own index)
template <int TX, int TY, int TZ>
__device__ __forceinline__ int tile_of3(const TileGeom3 &t, int ix, int iy, int iz, int txo = 0) {
    return ((iz / TZ) * t.nty + iy / TY) * t.ntx + bin_rot_x(ix / TX, t.ntx, txo);
}

// destination range of a particle that survived the move (-1 and PIC_EF_RANGE
// for a cell outside the mesh, which only a corrupt input cell can produce)
template <int TX, int TY, int TZ, typename R>
__device__ __forceinline__ int bin_dest3(const MeshParams3<R> &m, const TileGeom3 &t, int ix, int iy, int iz,
                                         unsigned *err, int txo) {
    if (ix < 0 || ix >= m.nx || iy < 0 || iy >= m.ny || iz < 0 || iz >= m.nz) {
        atomicOr(err, PIC_EF_RANGE);
        return -1;
    }
    return tile_of3<TX, TY, TZ>(t, ix, iy, iz, txo);
}

// Eq. (4) sums of the particles in the window [dlo, dhi) MeV
template <typename R>
__device__ __forceinline__ void diag_add3(R dacc[7], R dm, R dlo, R dhi, R dshift, R w, const R u[3],
                                          const R spn[3]) {
    const R e = ekin_mev(dm, u[0], u[1], u[2]);
    if (e >= dlo && e < dhi) {
        const R ep = e - dshift;
        dacc[0] += w;
        dacc[1] += w * spn[0];
        dacc[2] += w * spn[1];
        dacc[3] += w * spn[2];
        dacc[4] += w * ep;
        dacc[5] += w * ep * ep;
        dacc[6] += R(1);
    }
}

// Fused kernel, steps with the Eq. (4) sums: one record per lane, summed
// over the warp at once (float shuffles) and added to the warp's FP64 row of
// sdiag, so no accumulator stays live across the particle loop.  All 32 lanes
// of the warp call it together.
template <typename R>
__device__ __forceinline__ void diag_warp3(const DiagParams &D, int sp, bool has, R w, const R u[3], const R spn[3],
                                           double *row) {
    constexpr unsigned kAll = 0xFFFFFFFFu;
    R c[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    if (has) diag_add3(c, (R)D.m_mev[sp], (R)D.lo[sp], (R)D.hi[sp], (R)D.shift[sp], w, u, spn);
    if (!__any_sync(kAll, c[6] != R(0))) return;
    // the 8 slots (7 sums and a zero) over the warp in 9 shuffles: across lane
    // bits 4, 3 and 2 each lane keeps the half of its slots that bit selects
    // and adds its partner's copy of that half; then bits 1 and 0 sum the one
    // slot left, which lane 4 q ends up holding for slot q
    const int lane = threadIdx.x & 31;
    const bool h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1, h2 = (lane >> 2) & 1;
    R c4[4], c2[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R keep = h4 ? c[4 + k] : c[k], give = h4 ? c[k] : c[4 + k];
        c4[k] = keep + __shfl_xor_sync(kAll, give, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const R keep = h3 ? c4[2 + k] : c4[k], give = h3 ? c4[k] : c4[2 + k];
        c2[k] = keep + __shfl_xor_sync(kAll, give, 8);
    }
    R v = (h2 ? c2[1] : c2[0]) + __shfl_xor_sync(kAll, h2 ? c2[0] : c2[1], 4);
    v += __shfl_xor_sync(kAll, v, 2);
    v += __shfl_xor_sync(kAll, v, 1);
    const int q = lane >> 2;  // = 4 h4 + 2 h3 + h2
    if ((lane & 3) == 0 && q < 7) row[q] += (double)v;
}

}  // namespace
