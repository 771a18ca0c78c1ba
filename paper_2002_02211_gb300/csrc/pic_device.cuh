// pic_device.cuh -- device-side data layout and per-particle arithmetic of the
// 2D3V PIC + Thomas-BMT step (FP32 bulk math).
//
// Particle state is a structure of arrays per species, sorted by tile:
//   cell  uint32  (iy << 16) | ix, or PIC_DEAD for a removed particle
//   ox,oy float   offset inside the cell, [0, 1)
//   ux,uy,uz      u = p / (m c) at the half step
//   sx,sy,sz      spin at the half step
//   w             density carried by the macro-particle
//   id    int32   caller's identity (moved only by the sort)
// The mesh is one [6][ny][ld] float block for Ex Ey Ez Bx By Bz and one
// [3][ny][ld] block for Jx Jy Jz (ld = nx rounded up to 32 floats).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PIC_DEAD 0xFFFFFFFFu

// device-side error flags (bit set), read by the host at synchronising calls
#define PIC_EF_NAN 1u
#define PIC_EF_CFL 2u
#define PIC_EF_TIMEOUT 4u
#define PIC_EF_RANGE 8u

#define PIC_MAXSP 4
#define PIC_HALO 4   // window margin around a tile, in cells, on every side

struct DevSpecies {
    uint32_t *cell;
    float *ox, *oy, *ux, *uy, *uz, *sx, *sy, *sz, *w;
    int32_t *id;
    int32_t *tile_start;           // [ntiles + 1] slot range of each tile
    uint32_t *cell_old;            // split path: x^n kept for pic_deposit
    float *ox_old, *oy_old, *vz;
    float qm, q, a;                // q/m, q, anomaly
    int mobile;
    const int32_t *n;              // slots in use (device counter)
};

struct MeshParams {
    int nx, ny, ld, bc_x;          // bc_x: 0 open, 1 periodic
    float dt;
    float dt_dx, dt_dy;            // dt/dx, dt/dy (cell units per unit velocity)
    float dx_dt, dy_dt;            // dx/dt, dy/dt (Esirkepov current scale)
    float *EB;                     // [6][ny][ld]
    float *J;                      // [3][ny][ld]
    size_t plane;                  // ny * ld
};

struct TileGeom {
    int TX, TY;                    // tile size in cells
    int WX, WY;                    // window: x row stride (tile + 2 * PIC_HALO rounded up to
                                   // 32 floats, so a row shift never changes a bank), y rows
    int ntx, nty;                  // tiles along x and y
};

__host__ __device__ constexpr int window_wx(int tx) { return (tx + 2 * PIC_HALO + 31) / 32 * 32; }
__host__ __device__ constexpr int window_wy(int ty) { return ty + 2 * PIC_HALO; }

// Eq. (4) moments accumulated inside the fused kernel on diagnostic steps:
// per species and CTA the sums w, w s (3), w e', w e'^2, count over live
// particles with kinetic energy e in [lo, hi), where e' = e - shift and shift
// is the mean of the previous diagnostic (a one-pass variance that stays
// well conditioned).
struct DiagParams {
    int on;
    float lo[PIC_MAXSP], hi[PIC_MAXSP], m_mev[PIC_MAXSP];
    const double *shift;           // [PIC_MAXSP] device
    double *rows;                  // [PIC_MAXSP][8][gridDim] per-CTA sums (columns contiguous)
};

struct StepParams {
    MeshParams m;
    TileGeom t;
    int nsp;
    DevSpecies sp[PIC_MAXSP];
    unsigned *err;
    DiagParams diag;
};

// kinetic energy (gamma - 1) m c^2 = m c^2 u^2 / (1 + gamma), no cancellation
__device__ __forceinline__ float ekin_mev(float m_mev, float ux, float uy, float uz) {
    const float u2 = ux * ux + uy * uy + uz * uz;
    return m_mev * u2 / (1.f + sqrtf(1.f + u2));
}

// ---------------------------------------------------------------------------
// mesh accessors: a window staged in shared memory (local coordinates) or the
// global mesh (periodic wrap in y, and in x when periodic)
// ---------------------------------------------------------------------------
struct SmemMesh {
    const float *F;   // [6][WY][WX]
    float *Jw;        // [3][WY][WX]
    int WX, WY;
    __device__ __forceinline__ float f(int c, int x, int y) const { return F[(c * WY + y) * WX + x]; }
    __device__ __forceinline__ void j(int c, int x, int y, float v) const {
        atomicAdd(&Jw[(c * WY + y) * WX + x], v);
    }
};

struct GlobalMesh {
    const float *EB;
    float *J;
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
    __device__ __forceinline__ float f(int c, int x, int y) const {
        x = wx(x);
        y = wy(y);
        if (!ok(x, y)) {
            atomicOr(err, PIC_EF_RANGE);
            return 0.f;
        }
        return __ldg(&EB[c * plane + (size_t)y * ld + x]);
    }
    __device__ __forceinline__ void j(int c, int x, int y, float v) const {
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
template <class M>
__device__ __forceinline__ void gather_eb(const M &m, int ix, int iy, float ox, float oy,
                                          float E[3], float B[3]) {
    const float xn0 = 1.f - ox, xn1 = ox, yn0 = 1.f - oy, yn1 = oy;
    const bool rx = ox >= 0.5f, ry = oy >= 0.5f;
    const int hx = rx ? ix : ix - 1, hy = ry ? iy : iy - 1;
    const float ohx = rx ? ox - 0.5f : ox + 0.5f, ohy = ry ? oy - 0.5f : oy + 0.5f;
    const float xh0 = 1.f - ohx, xh1 = ohx, yh0 = 1.f - ohy, yh1 = ohy;
    auto bil = [&](int c, int x, int y, float a0, float a1, float b0, float b1) {
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
// Below th = 0.03 the two factors use their Taylor series to second order
// (truncation below 1e-9, under float rounding); above, sincosf of th/2.
// Divisions use the fast reciprocal (2 ulp), well inside the 1e-5 budget.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void push_spin(float qm, float a, float dt, const float E[3],
                                          const float B[3], float u[3], float s[3]) {
    const float h = 0.5f * qm * dt;
    const float umx = u[0] + h * E[0], umy = u[1] + h * E[1], umz = u[2] + h * E[2];
    const float gi = rsqrtf(1.f + umx * umx + umy * umy + umz * umz);
    const float tx = h * B[0] * gi, ty = h * B[1] * gi, tz = h * B[2] * gi;
    const float f = __fdividef(2.f, 1.f + tx * tx + ty * ty + tz * tz);
    const float upx = umx + (umy * tz - umz * ty);
    const float upy = umy + (umz * tx - umx * tz);
    const float upz = umz + (umx * ty - umy * tx);
    const float sx_ = f * tx, sy_ = f * ty, sz_ = f * tz;
    const float nx = umx + (upy * sz_ - upz * sy_) + h * E[0];
    const float ny = umy + (upz * sx_ - upx * sz_) + h * E[1];
    const float nz = umz + (upx * sy_ - upy * sx_) + h * E[2];

    // spin: Omega at the mean momentum
    const float bx = 0.5f * (u[0] + nx), by = 0.5f * (u[1] + ny), bz = 0.5f * (u[2] + nz);
    const float g2 = 1.f + bx * bx + by * by + bz * bz;
    const float gbi = rsqrtf(g2);
    const float gb = g2 * gbi;
    const float vx = bx * gbi, vy = by * gbi, vz = bz * gbi;
    const float ip1 = __fdividef(1.f, 1.f + gb);
    const float omB = a + gbi;               // Eq. (3)
    const float omv = a * gb * ip1;          // Eq. (3)
    const float omE = a + ip1;               // Eq. (3)
    const float vB = vx * B[0] + vy * B[1] + vz * B[2];
    const float cxE = vy * E[2] - vz * E[1];
    const float cyE = vz * E[0] - vx * E[2];
    const float czE = vx * E[1] - vy * E[0];
    // w = -Omega dt
    const float k = -qm * dt;
    const float wx = k * (omB * B[0] - omv * vB * vx - omE * cxE);
    const float wy = k * (omB * B[1] - omv * vB * vy - omE * cyE);
    const float wz = k * (omB * B[2] - omv * vB * vz - omE * czE);
    const float th2 = wx * wx + wy * wy + wz * wz;
    float A, C;
    if (th2 < 9e-4f) {
        A = 1.f - th2 * (1.f / 6.f);
        C = 0.5f - th2 * (1.f / 24.f);
    } else {
        const float rth = rsqrtf(th2);
        float sh, ch;
        sincosf(0.5f * th2 * rth, &sh, &ch);
        A = 2.f * sh * ch * rth;
        C = 2.f * sh * sh * rth * rth;
    }
    const float s0 = s[0], s1 = s[1], s2 = s[2];
    const float c0 = wy * s2 - wz * s1, c1 = wz * s0 - wx * s2, c2 = wx * s1 - wy * s0;  // w x s
    const float d0 = wy * c2 - wz * c1, d1 = wz * c0 - wx * c2, d2 = wx * c1 - wy * c0;  // w x (w x s)
    s[0] = s0 + A * c0 + C * d0;
    s[1] = s1 + A * c1 + C * d1;
    s[2] = s2 + A * c2 + C * d2;
    u[0] = nx;
    u[1] = ny;
    u[2] = nz;
}

// a4 along one axis: offset o in [0, 1) of cell i moves by d (|d| < 1 cell)
__device__ __forceinline__ void advance_axis(int &i, float &o, float d) {
    float o1 = o + d;
    if (o1 < 0.f) {
        o1 += 1.f;
        i -= 1;
    } else if (o1 >= 1.f) {
        o1 -= 1.f;
        i += 1;
    }
    if (o1 >= 1.f) {  // o1 + 1 rounded up to 1
        o1 -= 1.f;
        i += 1;
    }
    o = o1;
}

// First-order shape factors of the old position and their change, on the
// three nodes org, org+1, org+2 (org = min(i, i1)).  Differences are formed
// from the offsets directly so a small move keeps its relative precision.
__device__ __forceinline__ int shape3(int i, float o, int i1, float o1, float S0[3], float dS[3]) {
    const int d = i1 - i;
    if (d == 0) {
        const float dd = o1 - o;
        S0[0] = 1.f - o; S0[1] = o; S0[2] = 0.f;
        dS[0] = -dd; dS[1] = dd; dS[2] = 0.f;
        return i;
    }
    if (d > 0) {
        const float q = 1.f - o;
        S0[0] = q; S0[1] = o; S0[2] = 0.f;
        dS[0] = -q; dS[1] = q - o1; dS[2] = o1;
        return i;
    }
    const float q1 = 1.f - o1;
    S0[0] = 0.f; S0[1] = 1.f - o; S0[2] = o;
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
template <class M>
__device__ __forceinline__ void deposit_in_cell(const M &m, int ix, int iy, float ox, float oy,
                                                float ox1, float oy1, float qw, float vz,
                                                float dx_dt, float dy_dt) {
    const float d = ox1 - ox, e = oy1 - oy;
    const float xm = ox + 0.5f * d, ym = oy + 0.5f * e;
    const float jx = qw * dx_dt * d, jy = qw * dy_dt * e, cz = qw * vz;
    const float de = d * e * (1.f / 12.f);
    m.j(0, ix, iy, jx * (1.f - ym));
    m.j(0, ix, iy + 1, jx * ym);
    m.j(1, ix, iy, jy * (1.f - xm));
    m.j(1, ix + 1, iy, jy * xm);
    m.j(2, ix, iy, cz * ((1.f - xm) * (1.f - ym) + de));
    m.j(2, ix + 1, iy, cz * (xm * (1.f - ym) - de));
    m.j(2, ix, iy + 1, cz * ((1.f - xm) * ym - de));
    m.j(2, ix + 1, iy + 1, cz * (xm * ym + de));
}

template <class M>
__device__ __forceinline__ void deposit_esirkepov(const M &m, int ix, int iy, float ox, float oy,
                                                  int ix1, int iy1, float ox1, float oy1,
                                                  float qw, float vz, float dx_dt, float dy_dt) {
    if (ix1 == ix && iy1 == iy) {
        deposit_in_cell(m, ix, iy, ox, oy, ox1, oy1, qw, vz, dx_dt, dy_dt);
        return;
    }
    float S0x[3], dSx[3], S0y[3], dSy[3];
    const int gx = shape3(ix, ox, ix1, ox1, S0x, dSx);
    const int gy = shape3(iy, oy, iy1, oy1, S0y, dSy);
    const bool crx = ix1 != ix, cry = iy1 != iy;
    const float cx = -qw * dx_dt, cy = -qw * dy_dt, cz = qw * vz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j == 2 && !cry) break;
        const float fy = S0y[j] + 0.5f * dSy[j];
        const float a0 = dSx[0] * fy;
        m.j(0, gx, gy + j, cx * a0);
        if (crx) m.j(0, gx + 1, gy + j, cx * (a0 + dSx[1] * fy));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i == 2 && !crx) break;
        const float fx = S0x[i] + 0.5f * dSx[i];
        const float b0 = dSy[0] * fx;
        m.j(1, gx + i, gy, cy * b0);
        if (cry) m.j(1, gx + i, gy + 1, cy * (b0 + dSy[1] * fx));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j == 2 && !cry) break;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i == 2 && !crx) break;
            const float wz = S0x[i] * S0y[j] + 0.5f * (dSx[i] * S0y[j] + S0x[i] * dSy[j]) +
                             (1.f / 3.f) * dSx[i] * dSy[j];
            m.j(2, gx + i, gy + j, cz * wz);
        }
    }
}

__device__ __forceinline__ bool finite3(const float v[3]) {
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

__device__ __forceinline__ uint32_t pack_cell(int ix, int iy) {
    return ((uint32_t)iy << 16) | (uint32_t)ix;
}
