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

}  // namespace
