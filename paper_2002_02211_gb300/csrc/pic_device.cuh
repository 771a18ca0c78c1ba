// pic_device.cuh -- device-side data layout and per-particle arithmetic of the
// 2D3V PIC + Thomas-BMT step, templated on the real type R (float: the
// production path; double: the FP64 instantiation for the precision study).
//
// Particle state is a structure of arrays per species, sorted by tile:
//   cell  uint32  (iy << 16) | ix, or PIC_DEAD for a removed particle
//   ox,oy R       offset inside the cell, [0, 1)
//   ux,uy,uz R    u = p / (m c) at the half step
//   sx,sy,sz R    spin at the half step
//   w     R       density carried by the macro-particle
//   id    int32   caller's identity (moved only by the sort)
// The mesh is one [6][ny][ld] block of R for Ex Ey Ez Bx By Bz and one
// [3][ny][ld] block for Jx Jy Jz (ld = nx rounded up to 32).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PIC_DEAD 0xFFFFFFFFu

// device-side error flags (bit set), read by the host at synchronising calls
#define PIC_EF_NAN 1u
#define PIC_EF_CFL 2u
#define PIC_EF_TIMEOUT 4u
#define PIC_EF_RANGE 8u
#define PIC_EF_BINS 16u   // binned layout: a tile range and the overflow range were full
#define PIC_EF_CAP 32u    // a window move's plasma did not fit the species capacity

#define PIC_MAXSP 4
#define PIC_HALO 4     // least window margin around a tile along x, in cells
#define PIC_HALO_Y 4   // window margin along y, in cells

// precision-specific intrinsics
template <typename R>
struct Real;

template <>
struct Real<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
    // below this th^2 the rotation factors use their Taylor series (truncation < 1e-9)
    static constexpr float kTaylor = 9e-4f;
};

template <>
struct Real<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double sqrt_(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ void sincos_(double x, double *s, double *c) { ::sincos(x, s, c); }
    // truncation of the second-order series below th^2 = 1e-10: th^4/120 < 1e-22
    static constexpr double kTaylor = 1e-10;
};

template <typename R>
struct DevSpecies {
    uint32_t *cell;
    R *ox, *oy, *ux, *uy, *uz, *sx, *sy, *sz, *w;
    int32_t *id;
    int32_t *tile_start;           // [ntiles + 1] slot range of each tile
    uint32_t *cell_old;            // split path: x^n kept for pic_deposit
    R *ox_old, *oy_old, *vz;
    R qm, q, a;                    // q/m, q, anomaly
    int mobile;
    const int32_t *n;              // slots in use (device counter)
};

template <typename R>
struct MeshParams {
    int nx, ny, ld, bc_x;          // bc_x: 0 open, 1 periodic
    R dt;
    R dt_dx, dt_dy;                // dt/dx, dt/dy (cell units per unit velocity)
    R dx_dt, dy_dt;                // dx/dt, dy/dt (Esirkepov current scale)
    R *EB;                         // [6][ny][ld]
    R *J;                          // [3][ny][ld]
    size_t plane;                  // ny * ld
};

struct TileGeom {
    int TX, TY;                    // tile size in cells
    int WX, WY;                    // window: x row stride (tile + 2 * PIC_HALO rounded up to
                                   // 128 bytes, so a row shift never changes a bank), y rows
    int HX, HY;                    // window margins before the tile (the window starts at
                                   // tile origin - (HX, HY)); HX is a multiple of 4 (TMA)
    int ntx, nty;                  // tiles along x and y
};

template <typename R>
__host__ __device__ constexpr int window_wx(int tx) {
    return (tx + 2 * PIC_HALO + (int)(128 / sizeof(R)) - 1) / (int)(128 / sizeof(R)) * (int)(128 / sizeof(R));
}
// the row padding is split evenly between the two sides of the tile
template <typename R>
__host__ __device__ constexpr int window_hx(int tx) { return (window_wx<R>(tx) - tx) / 2 / 4 * 4; }
__host__ __device__ constexpr int window_wy(int ty) { return ty + 2 * PIC_HALO_Y; }
__host__ __device__ constexpr int window_hy() { return PIC_HALO_Y; }

// Eq. (4) moments accumulated inside the fused kernel on diagnostic steps:
// per species and CTA the sums w, w s (3), w e', w e'^2, count over live
// particles with kinetic energy e in [lo, hi), where e' = e - shift and shift
// is the mean of the previous diagnostic (a one-pass variance that stays
// well conditioned).
struct DiagParams {
    int on;
    double lo[PIC_MAXSP], hi[PIC_MAXSP], m_mev[PIC_MAXSP];
    const double *shift;           // [PIC_MAXSP] device
    double *rows;                  // [PIC_MAXSP][8][gridDim] per-CTA sums (columns contiguous)
};

template <typename R>
struct StepParams {
    MeshParams<R> m;
    TileGeom t;
    int nsp;
    DevSpecies<R> sp[PIC_MAXSP];
    unsigned *err;
    DiagParams diag;
};

// kinetic energy (gamma - 1) m c^2 = m c^2 u^2 / (1 + gamma), no cancellation
template <typename R>
__device__ __forceinline__ R ekin_mev(R m_mev, R ux, R uy, R uz) {
    const R u2 = ux * ux + uy * uy + uz * uz;
    return m_mev * u2 / (R(1) + Real<R>::sqrt_(R(1) + u2));
}

// ---------------------------------------------------------------------------
// mesh accessors: a window staged in shared memory (local coordinates) or the
// global mesh (periodic wrap in y, and in x when periodic)
// ---------------------------------------------------------------------------
template <typename R>
struct SmemMesh {
    const R *F;   // [6][WY][WX]
    R *Jw;        // [3][WY][WX]
    int WX, WY;
    __device__ __forceinline__ R f(int c, int x, int y) const { return F[(c * WY + y) * WX + x]; }
    __device__ __forceinline__ void j(int c, int x, int y, R v) const {
        atomicAdd(&Jw[(c * WY + y) * WX + x], v);
    }
};

template <typename R>
struct GlobalMesh {
    const R *EB;
    R *J;
    int nx, ny, ld, periodic_x;
    size_t plane;
    unsigned *err;
    __device__ __forceinline__ int wx(int x) const {
        if (periodic_x) {
            if (x < 0) x += nx;
            else if (x >= nx) x -= nx;
        }
        return x;
    }
    __device__ __forceinline__ int wy(int y) const {
        if (y < 0) y += ny;
        else if (y >= ny) y -= ny;
        return y;
    }
    __device__ __forceinline__ bool ok(int x, int y) const {
        return x >= 0 && x < nx && y >= 0 && y < ny;
    }
    __device__ __forceinline__ R f(int c, int x, int y) const {
        x = wx(x);
        y = wy(y);
        if (!ok(x, y)) {
            atomicOr(err, PIC_EF_RANGE);
            return R(0);
        }
        return __ldg(&EB[c * plane + (size_t)y * ld + x]);
    }
    __device__ __forceinline__ void j(int c, int x, int y, R v) const {
        x = wx(x);
        y = wy(y);
        if (!ok(x, y)) {
            atomicOr(err, PIC_EF_RANGE);
            return;
        }
        atomicAdd(&J[c * plane + (size_t)y * ld + x], v);
    }
};

// ---------------------------------------------------------------------------
// a1: first-order (CIC) gather of the six Yee components at their staggered
// positions; (ix, iy) in the accessor's frame, (ox, oy) in [0, 1)
// ---------------------------------------------------------------------------
template <typename R, class M>
__device__ __forceinline__ void gather_eb(const M &m, int ix, int iy, R ox, R oy, R E[3], R B[3]) {
    const R half = R(0.5), one = R(1);
    const R xn0 = one - ox, xn1 = ox, yn0 = one - oy, yn1 = oy;
    const bool rx = ox >= half, ry = oy >= half;
    const int hx = rx ? ix : ix - 1, hy = ry ? iy : iy - 1;
    const R ohx = rx ? ox - half : ox + half, ohy = ry ? oy - half : oy + half;
    const R xh0 = one - ohx, xh1 = ohx, yh0 = one - ohy, yh1 = ohy;
    auto bil = [&](int c, int x, int y, R a0, R a1, R b0, R b1) {
        return b0 * (a0 * m.f(c, x, y) + a1 * m.f(c, x + 1, y)) +
               b1 * (a0 * m.f(c, x, y + 1) + a1 * m.f(c, x + 1, y + 1));
    };
    E[0] = bil(0, hx, iy, xh0, xh1, yn0, yn1);   // Ex (i+1/2, j)
    E[1] = bil(1, ix, hy, xn0, xn1, yh0, yh1);   // Ey (i, j+1/2)
    E[2] = bil(2, ix, iy, xn0, xn1, yn0, yn1);   // Ez (i, j)
    B[0] = bil(3, ix, hy, xn0, xn1, yh0, yh1);   // Bx (i, j+1/2)
    B[1] = bil(4, hx, iy, xh0, xh1, yn0, yn1);   // By (i+1/2, j)
    B[2] = bil(5, hx, hy, xh0, xh1, yh0, yh1);   // Bz (i+1/2, j+1/2)
}

// ---------------------------------------------------------------------------
// a2 + a3: Boris push of u and the Thomas-BMT rotation of s.
// Omega (Eq. 2, c = 1) with the coefficients of Eq. (3) is evaluated at
// E^n, B^n and the mean momentum ubar = (u^{n-1/2} + u^{n+1/2}) / 2; Eq. (1),
// ds/dt = -Omega x s, is a rotation by the vector w = -Omega dt:
//   s' = s + (sin th / th) w x s + ((1 - cos th) / th^2) w x (w x s),  th = |w|.
// Below Real<R>::kTaylor (th^2) the two factors use their Taylor series to
// second order; above, sincos of th/2.  In float the divisions use the fast
// reciprocal (2 ulp), well inside the 1e-5 budget.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void push_spin(R qm, R a, R dt, const R E[3], const R B[3], R u[3], R s[3]) {
    using M = Real<R>;
    const R one = R(1), half = R(0.5);
    const R h = half * qm * dt;
    const R umx = u[0] + h * E[0], umy = u[1] + h * E[1], umz = u[2] + h * E[2];
    const R gi = M::rsqrt(one + umx * umx + umy * umy + umz * umz);
    const R tx = h * B[0] * gi, ty = h * B[1] * gi, tz = h * B[2] * gi;
    const R f = M::div(R(2), one + tx * tx + ty * ty + tz * tz);
    const R upx = umx + (umy * tz - umz * ty);
    const R upy = umy + (umz * tx - umx * tz);
    const R upz = umz + (umx * ty - umy * tx);
    const R sx_ = f * tx, sy_ = f * ty, sz_ = f * tz;
    const R nx = umx + (upy * sz_ - upz * sy_) + h * E[0];
    const R ny = umy + (upz * sx_ - upx * sz_) + h * E[1];
    const R nz = umz + (upx * sy_ - upy * sx_) + h * E[2];

    // spin: Omega at the mean momentum
    const R bx = half * (u[0] + nx), by = half * (u[1] + ny), bz = half * (u[2] + nz);
    const R g2 = one + bx * bx + by * by + bz * bz;
    const R gbi = M::rsqrt(g2);
    const R gb = g2 * gbi;
    const R vx = bx * gbi, vy = by * gbi, vz = bz * gbi;
    const R ip1 = M::div(one, one + gb);
    const R omB = a + gbi;               // Eq. (3)
    const R omv = a * gb * ip1;          // Eq. (3)
    const R omE = a + ip1;               // Eq. (3)
    const R vB = vx * B[0] + vy * B[1] + vz * B[2];
    const R cxE = vy * E[2] - vz * E[1];
    const R cyE = vz * E[0] - vx * E[2];
    const R czE = vx * E[1] - vy * E[0];
    // w = -Omega dt
    const R k = -qm * dt;
    const R wx = k * (omB * B[0] - omv * vB * vx - omE * cxE);
    const R wy = k * (omB * B[1] - omv * vB * vy - omE * cyE);
    const R wz = k * (omB * B[2] - omv * vB * vz - omE * czE);
    const R th2 = wx * wx + wy * wy + wz * wz;
    R A, C;
    if (th2 < M::kTaylor) {
        A = one - th2 * (one / R(6));
        C = half - th2 * (one / R(24));
    } else {
        const R rth = M::rsqrt(th2);
        R sh, ch;
        M::sincos_(half * th2 * rth, &sh, &ch);
        A = R(2) * sh * ch * rth;
        C = R(2) * sh * sh * rth * rth;
    }
    const R s0 = s[0], s1 = s[1], s2 = s[2];
    const R c0 = wy * s2 - wz * s1, c1 = wz * s0 - wx * s2, c2 = wx * s1 - wy * s0;  // w x s
    const R d0 = wy * c2 - wz * c1, d1 = wz * c0 - wx * c2, d2 = wx * c1 - wy * c0;  // w x (w x s)
    s[0] = s0 + A * c0 + C * d0;
    s[1] = s1 + A * c1 + C * d1;
    s[2] = s2 + A * c2 + C * d2;
    u[0] = nx;
    u[1] = ny;
    u[2] = nz;
}

// a4 along one axis: offset o in [0, 1) of cell i moves by d (|d| < 1 cell)
template <typename R>
__device__ __forceinline__ void advance_axis(int &i, R &o, R d) {
    R o1 = o + d;
    if (o1 < R(0)) {
        o1 += R(1);
        i -= 1;
    } else if (o1 >= R(1)) {
        o1 -= R(1);
        i += 1;
    }
    if (o1 >= R(1)) {  // o1 + 1 rounded up to 1
        o1 -= R(1);
        i += 1;
    }
    o = o1;
}

// First-order shape factors of the old position and their change, on the
// three nodes org, org+1, org+2 (org = min(i, i1)).  Differences are formed
// from the offsets directly so a small move keeps its relative precision.
template <typename R>
__device__ __forceinline__ int shape3(int i, R o, int i1, R o1, R S0[3], R dS[3]) {
    const int d = i1 - i;
    if (d == 0) {
        const R dd = o1 - o;
        S0[0] = R(1) - o; S0[1] = o; S0[2] = R(0);
        dS[0] = -dd; dS[1] = dd; dS[2] = R(0);
        return i;
    }
    if (d > 0) {
        const R q = R(1) - o;
        S0[0] = q; S0[1] = o; S0[2] = R(0);
        dS[0] = -q; dS[1] = q - o1; dS[2] = o1;
        return i;
    }
    const R q1 = R(1) - o1;
    S0[0] = R(0); S0[1] = R(1) - o; S0[2] = o;
    dS[0] = q1; dS[1] = o - q1; dS[2] = -o;
    return i - 1;
}

// ---------------------------------------------------------------------------
// a5: Esirkepov current of one move (old cell (ix, iy) offsets (ox, oy) to
// (ix1, iy1) (ox1, oy1), unwrapped, in the accessor's frame):
//   Wx = dSx (S0y + dSy/2),  Wy = dSy (S0x + dSx/2),
//   Wz = S0x S0y + (dSx S0y + S0x dSy)/2 + dSx dSy/3,
//   Jx(org+i+1/2) = -q w dx/dt sum_{i'<=i} Wx(i'),  Jy likewise,  Jz = q w vz Wz.
// Rows / columns that only hold zeros when the particle stays in its cell
// are skipped.
// ---------------------------------------------------------------------------
// Move that stays inside its cell (the common case): with the offsets d, e
// of the move and the midpoint (xm, ym) = (ox + d/2, oy + e/2) the weights
// above reduce to
//   Jx(i+1/2, j) = q w d dx/dt (1 - ym),  Jx(i+1/2, j+1) = q w d dx/dt ym,
//   Jy(i, j+1/2) = q w e dy/dt (1 - xm),  Jy(i+1, j+1/2) = q w e dy/dt xm,
//   Jz = q w vz [(1-xm)(1-ym) + de/12, xm(1-ym) - de/12, (1-xm) ym - de/12, xm ym + de/12].
template <typename R>
__device__ __forceinline__ void in_cell_weights(R ox, R oy, R ox1, R oy1, R qw, R vz, R dx_dt, R dy_dt,
                                                R v[8]) {
    const R one = R(1), half = R(0.5);
    const R d = ox1 - ox, e = oy1 - oy;
    const R xm = ox + half * d, ym = oy + half * e;
    const R jx = qw * dx_dt * d, jy = qw * dy_dt * e, cz = qw * vz;
    const R de = d * e * (one / R(12));
    v[0] = jx * (one - ym);                      // Jx (i+1/2, j)
    v[1] = jx * ym;                              // Jx (i+1/2, j+1)
    v[2] = jy * (one - xm);                      // Jy (i, j+1/2)
    v[3] = jy * xm;                              // Jy (i+1, j+1/2)
    v[4] = cz * ((one - xm) * (one - ym) + de);  // Jz (i, j)
    v[5] = cz * (xm * (one - ym) - de);          // Jz (i+1, j)
    v[6] = cz * ((one - xm) * ym - de);          // Jz (i, j+1)
    v[7] = cz * (xm * ym + de);                  // Jz (i+1, j+1)
}

template <typename R, class M>
__device__ __forceinline__ void deposit_in_cell(const M &m, int ix, int iy, R ox, R oy, R ox1, R oy1, R qw,
                                                R vz, R dx_dt, R dy_dt) {
    R v[8];
    in_cell_weights(ox, oy, ox1, oy1, qw, vz, dx_dt, dy_dt, v);
    m.j(0, ix, iy, v[0]);
    m.j(0, ix, iy + 1, v[1]);
    m.j(1, ix, iy, v[2]);
    m.j(1, ix + 1, iy, v[3]);
    m.j(2, ix, iy, v[4]);
    m.j(2, ix + 1, iy, v[5]);
    m.j(2, ix, iy + 1, v[6]);
    m.j(2, ix + 1, iy + 1, v[7]);
}

template <typename R, class M>
__device__ __forceinline__ void deposit_esirkepov(const M &m, int ix, int iy, R ox, R oy, int ix1, int iy1,
                                                  R ox1, R oy1, R qw, R vz, R dx_dt, R dy_dt) {
    if (ix1 == ix && iy1 == iy) {
        deposit_in_cell(m, ix, iy, ox, oy, ox1, oy1, qw, vz, dx_dt, dy_dt);
        return;
    }
    const R half = R(0.5);
    R S0x[3], dSx[3], S0y[3], dSy[3];
    const int gx = shape3(ix, ox, ix1, ox1, S0x, dSx);
    const int gy = shape3(iy, oy, iy1, oy1, S0y, dSy);
    const bool crx = ix1 != ix, cry = iy1 != iy;
    const R cx = -qw * dx_dt, cy = -qw * dy_dt, cz = qw * vz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j == 2 && !cry) break;
        const R fy = S0y[j] + half * dSy[j];
        const R a0 = dSx[0] * fy;
        m.j(0, gx, gy + j, cx * a0);
        if (crx) m.j(0, gx + 1, gy + j, cx * (a0 + dSx[1] * fy));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i == 2 && !crx) break;
        const R fx = S0x[i] + half * dSx[i];
        const R b0 = dSy[0] * fx;
        m.j(1, gx + i, gy, cy * b0);
        if (cry) m.j(1, gx + i, gy + 1, cy * (b0 + dSy[1] * fx));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j == 2 && !cry) break;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i == 2 && !crx) break;
            const R wz = S0x[i] * S0y[j] + half * (dSx[i] * S0y[j] + S0x[i] * dSy[j]) +
                         (R(1) / R(3)) * dSx[i] * dSy[j];
            m.j(2, gx + i, gy + j, cz * wz);
        }
    }
}

template <typename R>
__device__ __forceinline__ bool finite3(const R v[3]) {
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

__device__ __forceinline__ uint32_t pack_cell(int ix, int iy) {
    return ((uint32_t)iy << 16) | (uint32_t)ix;
}

// Eq. (4) sums of the particles in the window [dlo, dhi) MeV
template <typename R>
__device__ __forceinline__ void diag_add(R dacc[7], R dm, R dlo, R dhi, R dshift, R w, const R u[3],
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
__device__ __forceinline__ void diag_warp(const DiagParams &D, int sp, bool has, R w, const R u[3], const R spn[3],
                                           double *row) {
    constexpr unsigned kAll = 0xFFFFFFFFu;
    R c[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    if (has) diag_add(c, (R)D.m_mev[sp], (R)D.lo[sp], (R)D.hi[sp], (R)D.shift[sp], w, u, spn);
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

// column `col` of the CTA's FP64 sums of species sp, kept per warp in sdiag
// (nwarps rows, ncols columns per output row); the whole CTA calls it
__device__ __forceinline__ void store_diag_sums(const DiagParams &D, int sp, double (*sdiag)[8], int nwarps, int col,
                                                int ncols) {
    __syncthreads();
    const int tid = threadIdx.x;
    if (tid < 7) {
        double t = 0.0;
        for (int w8 = 0; w8 < nwarps; ++w8) t += sdiag[w8][tid];
        D.rows[((size_t)sp * 8 + tid) * ncols + col] = t;
    }
    __syncthreads();
}
