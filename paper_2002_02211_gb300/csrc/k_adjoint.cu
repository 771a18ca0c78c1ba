// k_adjoint.cu -- discrete adjoint of the 2D3V step (gather, Boris push,
// Thomas-BMT rotation, position advance, Esirkepov current, three-stage Yee
// update with the Silver-Mueller boundary and laser source), for the gradient
// of a loss on the final particle state with respect to the initial particle
// state, the particle weights and the laser amplitude a0.
//
// The step is linear in the mesh fields except through the particles, so the
// mesh part of the adjoint is the transpose of each field stage; the particle
// part is, per particle, the vector-Jacobian product of the forward arithmetic
// (the gather, push_spin and the deposit swept in reverse by hand, each with
// the derivatives of the branch the forward step takes).  Adjoint kernels run
// in the reverse order of the forward stages:
//   b_half^T, e_full^T (-> lambda_J), boundary^T (-> dL/da0), b_half^T, particles^T.
#include <algorithm>

#include "pic_device.cuh"
#include "pic_kernels.h"

namespace {

// ---------------------------------------------------------------------------
// mesh transposes (the same validity rules as the forward stages)
// ---------------------------------------------------------------------------
// forward: Bx(j,i) -= hdy (Ez(j+1,i) - Ez(j,i));  By(j,i) += hdx (Ez(j,i+1) - Ez(j,i));
//          Bz(j,i) -= hdx (Ey(j,i+1) - Ey(j,i)) - hdy (Ex(j+1,i) - Ex(j,i)),
// By, Bz only where column i+1 exists.  Transpose: lambda_E += C^T lambda_B.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_b_half(const AdjMesh<R> A, R hdx, R hdy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    const int nx = A.nx, ny = A.ny, ld = A.ld;
    if (i >= nx) return;
    const bool per = A.bc_x == 1;
    const size_t P = A.plane;
    R *L = A.LEB;
    const int jm = j == 0 ? ny - 1 : j - 1;
    const int im = i == 0 ? (per ? nx - 1 : -1) : i - 1;
    auto valid = [&](int k) { return k >= 0 && (per || k < nx - 1); };
    const size_t c = (size_t)j * ld + i, cjm = (size_t)jm * ld + i;
    R lez = hdy * (L[3 * P + c] - L[3 * P + cjm]) - (valid(i) ? hdx * L[4 * P + c] : R(0));
    R ley = valid(i) ? hdx * L[5 * P + c] : R(0);
    R lex = valid(i) ? hdy * (L[5 * P + cjm] - L[5 * P + c]) : R(0);
    if (valid(im)) {
        const size_t cim = (size_t)j * ld + im;
        lez += hdx * L[4 * P + cim];
        ley -= hdx * L[5 * P + cim];
    }
    L[0 * P + c] += lex;
    L[1 * P + c] += ley;
    L[2 * P + c] += lez;
}

// forward: Ex(j,i) += dtdy (Bz(j,i) - Bz(j-1,i)) - dt Jx;  Ey(j,i) -= dtdx (Bz(j,i) - Bz(j,i-1)) + dt Jy;
//          Ez(j,i) += dtdx (By(j,i) - By(j,i-1)) - dtdy (Bx(j,i) - Bx(j-1,i)) - dt Jz,
// with the left boundary values byL, bzL in place of column -1 when x is open.
// Transpose: lambda_B += C^T lambda_E, lambda_ghost, lambda_J = -dt lambda_E.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_e_full(const AdjMesh<R> A, R dt, R dtdx, R dtdy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    const int nx = A.nx, ny = A.ny, ld = A.ld;
    if (i >= nx) return;
    const bool per = A.bc_x == 1;
    const size_t P = A.plane;
    R *L = A.LEB;
    const int jp = j + 1 == ny ? 0 : j + 1;
    const int ip = i + 1 == nx ? (per ? 0 : -1) : i + 1;
    const size_t c = (size_t)j * ld + i, cjp = (size_t)jp * ld + i;
    const R lex = L[c], ley = L[P + c], lez = L[2 * P + c];
    R lbz = dtdy * (lex - L[cjp]) - dtdx * ley;
    R lby = dtdx * lez;
    const R lbx = dtdy * (L[2 * P + cjp] - lez);
    if (ip >= 0) {
        const size_t cip = (size_t)j * ld + ip;
        lbz += dtdx * L[P + cip];
        lby -= dtdx * L[2 * P + cip];
    }
    L[3 * P + c] += lbx;
    L[4 * P + c] += lby;
    L[5 * P + c] += lbz;
    A.LJ[c] = -dt * lex;
    A.LJ[P + c] = -dt * ley;
    A.LJ[2 * P + c] = -dt * lez;
    if (i == 0 && !per) {
        A.Lbnd[j] = -dtdx * lez;       // By(-1/2)
        A.Lbnd[ny + j] = dtdx * ley;   // Bz(-1/2)
    }
}

// forward (open x): byL = (2 Ez(0) - (1-r) By(0) - q (Bx(j,0) - Bx(j-1,0)) - 4 a0 phz prof_j) / (1+r)
//                   bzL = (4 a0 phy prof'_j - 2 Ey(0) - (1-r) Bz(0)) / (1+r)
//                   By(nx-1) = (-2 Ez(nx-1) - (1-r) By(nx-2) + q (Bx(j,nx-1) - Bx(j-1,nx-1))) / (1+r)
//                   Bz(nx-1) = (2 Ey(nx-1) - (1-r) Bz(nx-2)) / (1+r)
// (assignments: the adjoints of the overwritten values are consumed).
template <typename R>
__global__ void k_adj_boundary(const AdjMesh<R> A, const double *prof, double phz, double phy, double r, double q,
                               double *dl_da0) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int ny = A.ny, nx = A.nx, ld = A.ld;
    double acc = 0.0;
    if (j < ny) {
        const size_t P = A.plane;
        R *L = A.LEB;
        const int jm = j == 0 ? ny - 1 : j - 1;
        const double ir = 1.0 / (1.0 + r), mr = 1.0 - r;
        const size_t c0 = (size_t)j * ld, cm0 = (size_t)jm * ld;
        const double lyl = A.Lbnd[j], lzl = A.Lbnd[ny + j];
        L[2 * P + c0] += (R)(2.0 * ir * lyl);
        L[4 * P + c0] += (R)(-mr * ir * lyl);
        atomicAdd(&L[3 * P + c0], (R)(-q * ir * lyl));
        atomicAdd(&L[3 * P + cm0], (R)(q * ir * lyl));
        L[1 * P + c0] += (R)(-2.0 * ir * lzl);
        L[5 * P + c0] += (R)(-mr * ir * lzl);
        acc = (-4.0 * phz * prof[j] * lyl + 4.0 * phy * prof[ny + j] * lzl) * ir;
        A.Lbnd[j] = R(0);
        A.Lbnd[ny + j] = R(0);
        const size_t cl = c0 + nx - 1, cml = cm0 + nx - 1;
        const double lyr = L[4 * P + cl], lzr = L[5 * P + cl];
        L[4 * P + cl] = R(0);
        L[5 * P + cl] = R(0);
        L[2 * P + cl] += (R)(-2.0 * ir * lyr);
        atomicAdd(&L[4 * P + cl - 1], (R)(-mr * ir * lyr));
        atomicAdd(&L[3 * P + cl], (R)(q * ir * lyr));
        atomicAdd(&L[3 * P + cml], (R)(-q * ir * lyr));
        L[1 * P + cl] += (R)(2.0 * ir * lzr);
        atomicAdd(&L[5 * P + cl - 1], (R)(-mr * ir * lzr));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(dl_da0, acc);
}

// ---------------------------------------------------------------------------
// particles
// ---------------------------------------------------------------------------
// wrapped global node index (periodic y, and x when periodic); -1 outside
template <typename R>
__device__ __forceinline__ long long node(const AdjMesh<R> &A, int x, int y) {
    if (A.bc_x == 1) x = x < 0 ? x + A.nx : (x >= A.nx ? x - A.nx : x);
    y = y < 0 ? y + A.ny : (y >= A.ny ? y - A.ny : y);
    if (x < 0 || x >= A.nx || y < 0 || y >= A.ny) return -1;
    return (long long)y * A.ld + x;
}

// field values of the stored state for the forward gather
template <typename R>
struct StoredMesh {
    const AdjMesh<R> *A;
    const R *EB;
    __device__ __forceinline__ R f(int c, int x, int y) const {
        const long long k = node(*A, x, y);
        return k < 0 ? R(0) : EB[c * A->plane + k];
    }
};

// Reverse of the 2D3V Esirkepov deposit (a5), by hand: val = <lambda_J, J>
// of one move, and its derivatives g in (ox, oy, ox1, oy1, vz), for the same
// nodes and the same branch (in-cell closed form, or the general form over the
// shape3 factors) as deposit_esirkepov; lambda_J outside the mesh counts zero.
template <typename R>
__device__ __forceinline__ void deposit_vjp(const AdjMesh<R> &A, int ix, int iy, R ox, R oy, int ix1, int iy1,
                                            R ox1, R oy1, R qw, R vz, R dx_dt, R dy_dt, R &val, R g[5]) {
    const R one = R(1), half = R(0.5), third = R(1) / R(3);
    auto lam = [&](int c, int x, int y) {
        const long long k = node(A, x, y);
        return k < 0 ? R(0) : A.LJ[c * A.plane + k];
    };
    if (ix1 == ix && iy1 == iy) {
        const R d = ox1 - ox, e = oy1 - oy;
        const R xm = ox + half * d, ym = oy + half * e;
        const R jx = qw * dx_dt * d, jy = qw * dy_dt * e, cz = qw * vz;
        const R de = d * e * (one / R(12));
        const R lx0 = lam(0, ix, iy), lx1 = lam(0, ix, iy + 1);
        const R ly0 = lam(1, ix, iy), ly1 = lam(1, ix + 1, iy);
        const R z00 = lam(2, ix, iy), z10 = lam(2, ix + 1, iy), z01 = lam(2, ix, iy + 1), z11 = lam(2, ix + 1, iy + 1);
        const R Lx = lx0 * (one - ym) + lx1 * ym;
        const R Ly = ly0 * (one - xm) + ly1 * xm;
        const R K = z00 - z10 - z01 + z11;
        const R Z = z00 * (one - xm) * (one - ym) + z10 * xm * (one - ym) + z01 * (one - xm) * ym + z11 * xm * ym + de * K;
        val = jx * Lx + jy * Ly + cz * Z;
        const R gd = qw * dx_dt * Lx + cz * e * (one / R(12)) * K;
        const R ge = qw * dy_dt * Ly + cz * d * (one / R(12)) * K;
        const R gxm = jy * (ly1 - ly0) + cz * ((z10 - z00) * (one - ym) + (z11 - z01) * ym);
        const R gym = jx * (lx1 - lx0) + cz * ((z01 - z00) * (one - xm) + (z11 - z10) * xm);
        // d = ox1 - ox, xm = ox + d / 2 (likewise e, ym)
        g[0] = -gd + half * gxm;
        g[2] = gd + half * gxm;
        g[1] = -ge + half * gym;
        g[3] = ge + half * gym;
        g[4] = qw * Z;
        return;
    }
    R S0x[3], dSx[3], S0y[3], dSy[3];
    const int gx = shape3(ix, ox, ix1, ox1, S0x, dSx);
    const int gy = shape3(iy, oy, iy1, oy1, S0y, dSy);
    const bool crx = ix1 != ix, cry = iy1 != iy;
    const int ni = crx ? 3 : 2, nj = cry ? 3 : 2;
    const R cx = -qw * dx_dt, cy = -qw * dy_dt, cz = qw * vz;
    R gS0x[3] = {R(0), R(0), R(0)}, gdSx[3] = {R(0), R(0), R(0)};
    R gS0y[3] = {R(0), R(0), R(0)}, gdSy[3] = {R(0), R(0), R(0)};
    R vx = R(0), vy = R(0), vzs = R(0);
    // Jx(gx, gy+j) = cx dSx0 fy_j, Jx(gx+1, gy+j) = cx (dSx0 + dSx1) fy_j (crossing x)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j >= nj) break;
        const R fy = S0y[j] + half * dSy[j];
        const R l1 = crx ? lam(0, gx + 1, gy + j) : R(0);
        const R P = lam(0, gx, gy + j) + l1, Q = l1;
        vx += fy * (dSx[0] * P + dSx[1] * Q);
        gdSx[0] += cx * fy * P;
        gdSx[1] += cx * fy * Q;
        const R gf = cx * (dSx[0] * P + dSx[1] * Q);
        gS0y[j] += gf;
        gdSy[j] += half * gf;
    }
    // Jy(gx+i, gy) = cy dSy0 fx_i, Jy(gx+i, gy+1) = cy (dSy0 + dSy1) fx_i (crossing y)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i >= ni) break;
        const R fx = S0x[i] + half * dSx[i];
        const R l1 = cry ? lam(1, gx + i, gy + 1) : R(0);
        const R P = lam(1, gx + i, gy) + l1, Q = l1;
        vy += fx * (dSy[0] * P + dSy[1] * Q);
        gdSy[0] += cy * fx * P;
        gdSy[1] += cy * fx * Q;
        const R gf = cy * (dSy[0] * P + dSy[1] * Q);
        gS0x[i] += gf;
        gdSx[i] += half * gf;
    }
    // Jz(gx+i, gy+j) = cz wz(i, j)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j >= nj) break;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= ni) break;
            const R l = lam(2, gx + i, gy + j);
            vzs += l * (S0x[i] * S0y[j] + half * (dSx[i] * S0y[j] + S0x[i] * dSy[j]) + third * dSx[i] * dSy[j]);
            const R cl = cz * l;
            gS0x[i] += cl * (S0y[j] + half * dSy[j]);
            gdSx[i] += cl * (half * S0y[j] + third * dSy[j]);
            gS0y[j] += cl * (S0x[i] + half * dSx[i]);
            gdSy[j] += cl * (half * S0x[i] + third * dSx[i]);
        }
    }
    val = cx * vx + cy * vy + cz * vzs;
    g[4] = qw * vzs;
    // shape3 in reverse: S0, dS as functions of (o, o1) in each of its branches
    auto shape_back = [&](int d, const R gS0[3], const R gdS[3], R &go, R &go1) {
        if (d == 0) {
            go = -gS0[0] + gS0[1] + gdS[0] - gdS[1];
            go1 = -gdS[0] + gdS[1];
        } else if (d > 0) {
            go = -gS0[0] + gS0[1] + gdS[0] - gdS[1];
            go1 = -gdS[1] + gdS[2];
        } else {
            go = -gS0[1] + gS0[2] + gdS[1] - gdS[2];
            go1 = -gdS[0] + gdS[1];
        }
    };
    shape_back(ix1 - ix, gS0x, gdSx, g[0], g[2]);
    shape_back(iy1 - iy, gS0y, gdSy, g[1], g[3]);
}

// Reverse of the gather (a1), by hand, one pass over the 24 stencil nodes:
// lambda of each staggered node += weight x lambda of the gathered value (the
// transpose into lambda_EB), and the derivatives of <lE, E> + <lB, B> in the
// offsets, whose bilinear weights move as (-1, +1) with ox (x weights) and
// with oy (y weights), within the stencil branch the forward gather takes.
template <typename R>
__device__ __forceinline__ void gather_vjp(const AdjMesh<R> &A, const R *EB, int ix, int iy, R ox, R oy,
                                           const R lE[3], const R lB[3], R &lox, R &loy) {
    const R half = R(0.5), one = R(1);
    const R xn0 = one - ox, xn1 = ox, yn0 = one - oy, yn1 = oy;
    const bool rx = ox >= half, ry = oy >= half;
    const int hx = rx ? ix : ix - 1, hy = ry ? iy : iy - 1;
    const R ohx = rx ? ox - half : ox + half, ohy = ry ? oy - half : oy + half;
    const R xh0 = one - ohx, xh1 = ohx, yh0 = one - ohy, yh1 = ohy;
    auto bil = [&](int c, int x, int y, R a0, R a1, R b0, R b1, R lam) {
        if (lam == R(0)) return;
        const long long n00 = node(A, x, y), n10 = node(A, x + 1, y);
        const long long n01 = node(A, x, y + 1), n11 = node(A, x + 1, y + 1);
        const R *F = EB + c * A.plane;
        const R f00 = n00 < 0 ? R(0) : F[n00], f10 = n10 < 0 ? R(0) : F[n10];
        const R f01 = n01 < 0 ? R(0) : F[n01], f11 = n11 < 0 ? R(0) : F[n11];
        lox += lam * (b0 * (f10 - f00) + b1 * (f11 - f01));
        loy += lam * ((a0 * f01 + a1 * f11) - (a0 * f00 + a1 * f10));
        R *L = A.LEB + c * A.plane;
        if (n00 >= 0) atomicAdd(&L[n00], b0 * a0 * lam);
        if (n10 >= 0) atomicAdd(&L[n10], b0 * a1 * lam);
        if (n01 >= 0) atomicAdd(&L[n01], b1 * a0 * lam);
        if (n11 >= 0) atomicAdd(&L[n11], b1 * a1 * lam);
    };
    bil(0, hx, iy, xh0, xh1, yn0, yn1, lE[0]);
    bil(1, ix, hy, xn0, xn1, yh0, yh1, lE[1]);
    bil(2, ix, iy, xn0, xn1, yn0, yn1, lE[2]);
    bil(3, ix, hy, xn0, xn1, yh0, yh1, lB[0]);
    bil(4, hx, iy, xh0, xh1, yn0, yn1, lB[1]);
    bil(5, hx, hy, xh0, xh1, yh0, yh1, lB[2]);
}

// Vector-Jacobian product of push_spin (a2 + a3), by hand: the forward
// arithmetic is recomputed with its intermediates kept, then swept in reverse
// with the derivatives of each formula of the branch the forward step takes
// (Taylor series or sincos of the rotation angle).  In: the step's inputs and
// the lambdas lun, lsn of the new u and s; out: the lambdas of u, s, E, B.
// For a cross product c = p x q the sweep adds q x lc to lp and lc x p to lq.
template <typename R>
__device__ __forceinline__ void push_spin_vjp(R qm, R a, R dt, const R E[3], const R B[3], const R u[3],
                                              const R s[3], const R lun[3], const R lsn[3], R lu[3], R ls[3],
                                              R lE[3], R lB[3]) {
    using M = Real<R>;
    const R one = R(1), half = R(0.5), two = R(2);
    auto cross = [](const R p[3], const R q[3], R c[3]) {
        c[0] = p[1] * q[2] - p[2] * q[1];
        c[1] = p[2] * q[0] - p[0] * q[2];
        c[2] = p[0] * q[1] - p[1] * q[0];
    };
    auto dot = [](const R p[3], const R q[3]) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; };
    // ---- forward, as push_spin computes it
    const R h = half * qm * dt;
    const R um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
    const R gm = M::rsqrt(one + dot(um, um));
    const R t[3] = {h * B[0] * gm, h * B[1] * gm, h * B[2] * gm};
    const R T2 = one + dot(t, t);
    const R f = M::div(two, T2);
    R ut[3];
    cross(um, t, ut);
    const R up[3] = {um[0] + ut[0], um[1] + ut[1], um[2] + ut[2]};
    const R sv[3] = {f * t[0], f * t[1], f * t[2]};
    R us[3];
    cross(up, sv, us);
    const R un[3] = {um[0] + us[0] + h * E[0], um[1] + us[1] + h * E[1], um[2] + us[2] + h * E[2]};
    const R b[3] = {half * (u[0] + un[0]), half * (u[1] + un[1]), half * (u[2] + un[2])};
    const R g2 = one + dot(b, b);
    const R gbi = M::rsqrt(g2);
    const R gb = g2 * gbi;
    const R v[3] = {b[0] * gbi, b[1] * gbi, b[2] * gbi};
    const R ip1 = M::div(one, one + gb);
    const R omB = a + gbi, omv = a * gb * ip1, omE = a + ip1;  // Eq. (3)
    const R vB = dot(v, B);
    R cE[3];
    cross(v, E, cE);
    const R k = -qm * dt;
    const R w[3] = {k * (omB * B[0] - omv * vB * v[0] - omE * cE[0]),
                    k * (omB * B[1] - omv * vB * v[1] - omE * cE[1]),
                    k * (omB * B[2] - omv * vB * v[2] - omE * cE[2])};
    const R th2 = dot(w, w);
    R A, C, dA, dC;  // rotation factors and their derivatives in th2
    if (th2 < M::kTaylor) {
        A = one - th2 * (one / R(6));
        C = half - th2 * (one / R(24));
        dA = -(one / R(6));
        dC = -(one / R(24));
    } else {
        const R rth = M::rsqrt(th2);  // 1 / theta
        R sh, ch;
        M::sincos_(half * th2 * rth, &sh, &ch);
        const R sn = two * sh * ch, omc = two * sh * sh, cs = one - omc;  // sin, 1 - cos, cos of theta
        A = sn * rth;
        C = omc * rth * rth;
        const R th = th2 * rth;
        // dA/dth2 = (theta cos - sin) / (2 theta^3), dC/dth2 = (theta sin - 2 (1 - cos)) / (2 theta^4)
        dA = half * (th * cs - sn) * rth * rth * rth;
        dC = half * (th * sn - two * omc) * rth * rth * rth * rth;
    }
    R c[3], d[3];
    cross(w, s, c);
    cross(w, c, d);
    // ---- reverse: s_new = s + A c + C d, c = w x s, d = w x c
    const R lA = dot(lsn, c), lC = dot(lsn, d);
    R ld[3] = {C * lsn[0], C * lsn[1], C * lsn[2]};
    R lc[3], lw[3], tmp[3];
    cross(ld, w, tmp);  // from d = w x c: lc += ld x w, lw += c x ld
    lc[0] = A * lsn[0] + tmp[0], lc[1] = A * lsn[1] + tmp[1], lc[2] = A * lsn[2] + tmp[2];
    cross(c, ld, lw);
    cross(s, lc, tmp);  // from c = w x s: lw += s x lc, ls += lc x w
    lw[0] += tmp[0], lw[1] += tmp[1], lw[2] += tmp[2];
    cross(lc, w, tmp);
    ls[0] = lsn[0] + tmp[0], ls[1] = lsn[1] + tmp[1], ls[2] = lsn[2] + tmp[2];
    const R lth2 = lA * dA + lC * dC;
    lw[0] += two * w[0] * lth2, lw[1] += two * w[1] * lth2, lw[2] += two * w[2] * lth2;
    // w = k (omB B - omv vB v - omE cE)
    const R lwv = dot(lw, v);
    const R lomB = k * dot(lw, B), lomv = -k * vB * lwv, lvB = -k * omv * lwv, lomE = -k * dot(lw, cE);
    R lv[3], lcE[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lB[i] = k * omB * lw[i] + lvB * v[i];
        lv[i] = -k * omv * vB * lw[i] + lvB * B[i];
        lcE[i] = -k * omE * lw[i];
    }
    cross(E, lcE, tmp);  // cE = v x E: lv += E x lcE, lE += lcE x v
    lv[0] += tmp[0], lv[1] += tmp[1], lv[2] += tmp[2];
    cross(lcE, v, lE);
    // omB = a + gbi, omv = a gb ip1, omE = a + ip1, ip1 = 1 / (1 + gb)
    const R lip1 = a * gb * lomv + lomE;
    const R lgb = a * ip1 * lomv - ip1 * ip1 * lip1;
    // v = b gbi, gb = g2 gbi, gbi = g2^(-1/2), g2 = 1 + b.b
    const R lgbi = lomB + dot(lv, b) + g2 * lgb;
    const R lg2 = gbi * lgb - half * gbi * gbi * gbi * lgbi;
    R lb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) lb[i] = gbi * lv[i] + two * b[i] * lg2;
    // b = (u + un) / 2
    R lunt[3] = {lun[0] + half * lb[0], lun[1] + half * lb[1], lun[2] + half * lb[2]};
    // un = um + up x sv + h E
    R lum[3] = {lunt[0], lunt[1], lunt[2]};
    R lup[3], lsv[3];
    cross(sv, lunt, lup);   // lup = sv x lun
    cross(lunt, up, lsv);   // lsv = lun x up
    // sv = f t
    const R lf = dot(lsv, t);
    R lt[3] = {f * lsv[0], f * lsv[1], f * lsv[2]};
    // up = um + um x t
    lum[0] += lup[0], lum[1] += lup[1], lum[2] += lup[2];
    cross(t, lup, tmp);  // lum += t x lup
    lum[0] += tmp[0], lum[1] += tmp[1], lum[2] += tmp[2];
    cross(lup, um, tmp);  // lt += lup x um
    lt[0] += tmp[0], lt[1] += tmp[1], lt[2] += tmp[2];
    // f = 2 / T2, T2 = 1 + t.t
    const R lT2 = -half * f * f * lf;
    lt[0] += two * t[0] * lT2, lt[1] += two * t[1] * lT2, lt[2] += two * t[2] * lT2;
    // t = h B gm, gm = (1 + um.um)^(-1/2)
    const R lgm = h * dot(lt, B);
    const R gm3 = gm * gm * gm;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lB[i] += h * gm * lt[i];
        lum[i] -= gm3 * um[i] * lgm;
    }
    // um = u + h E; un's own h E term
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lu[i] = half * lb[i] + lum[i];
        lE[i] += h * (lum[i] + lunt[i]);
    }
}

// One adjoint particle step.  In: the particle state at step n (stored), the
// fields E^n, B^n (stored), lambda_J of the step, and the particle lambdas of
// step n+1; out: the particle lambdas of step n, lambda_w accumulated, the
// gather's transpose added to the mesh lambdas.
template <typename R>
// (FP32: at most 64 registers, 8 CTAs of 128 threads per SM; this
// latency-bound kernel ran 5% faster so than at 118 registers and 4 CTAs)
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 8 : 1) k_adj_particles(const AdjMesh<R> A, const AdjParticles<R> S) {
    const StoredMesh<R> sm{&A, S.EB};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < S.n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[p];
        if (c == PIC_DEAD) continue;
        const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
        const R ox = S.ox[p], oy = S.oy[p], w = S.w[p];
        const R u0[3] = {S.ux[p], S.uy[p], S.uz[p]};
        const R s0[3] = {S.sx[p], S.sy[p], S.sz[p]};
        // forward of this step, as the split path computes it
        R E[3], B[3];
        gather_eb(sm, ix, iy, ox, oy, E, B);
        R un[3] = {u0[0], u0[1], u0[2]}, sn[3] = {s0[0], s0[1], s0[2]};
        push_spin(S.qm, S.a, A.dt, E, B, un, sn);
        const R gi = Real<R>::rsqrt(R(1) + un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
        int ix1 = ix, iy1 = iy;
        R ox1 = ox, oy1 = oy;
        advance_axis(ix1, ox1, un[0] * gi * A.dt_dx);
        advance_axis(iy1, oy1, un[1] * gi * A.dt_dy);
        const R vz = un[2] * gi;
        // lambdas of step n+1 (zero for a particle removed in this step)
        R lx1 = S.lx[p], ly1 = S.ly[p];
        R lu[3] = {S.lux[p], S.luy[p], S.luz[p]}, ls[3] = {S.lsx[p], S.lsy[p], S.lsz[p]};
        // a5: <lambda_J, J> of the move and its derivatives in (ox, oy, ox1, oy1, vz)
        R dval, dg[5];
        deposit_vjp(A, ix, iy, ox, oy, ix1, iy1, ox1, oy1, S.q * w, vz, A.dx_dt, A.dy_dt, dval, dg);
        if (w != R(0)) S.lw[p] += dval / w;
        lx1 += dg[2];
        ly1 += dg[3];
        // a4: ox1 = ox + dt/dx ux gi, oy1 = oy + dt/dy uy gi, vz = uz gi
        const R cv[3] = {lx1 * A.dt_dx, ly1 * A.dt_dy, dg[4]};
        const R cu = cv[0] * un[0] + cv[1] * un[1] + cv[2] * un[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) lu[k] += gi * cv[k] - un[k] * cu * gi * gi * gi;
        R lox = lx1 + dg[0], loy = ly1 + dg[1];
        // a2 + a3: vector-Jacobian product of push_spin over (u, s, E, B)
        R lin[12];
        push_spin_vjp(S.qm, S.a, A.dt, E, B, u0, s0, lu, ls, lin, lin + 3, lin + 6, lin + 9);
        // a1: the gathered values depend on the mesh (transpose into lambda_EB)
        // and on the offsets
        gather_vjp(A, S.EB, ix, iy, ox, oy, lin + 6, lin + 9, lox, loy);
        S.lx[p] = lox;
        S.ly[p] = loy;
        S.lux[p] = lin[0];
        S.luy[p] = lin[1];
        S.luz[p] = lin[2];
        S.lsx[p] = lin[3];
        S.lsy[p] = lin[4];
        S.lsz[p] = lin[5];
    }
}

// ---------------------------------------------------------------------------
// loss: L = sum a_i s_i / sum a_i over the live particles of a species, with
// a_i = w_i e_i sig((e_i - ec)/de), e_i the kinetic energy [MeV] and s_i the
// chosen spin component (the energy-weighted polarization above ec)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_loss_sums(const AdjParticles<R> S, LossParams L, double *sums) {
    double a = 0.0, as = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < S.n; p += (long long)gridDim.x * blockDim.x) {
        if (S.cell[p] == PIC_DEAD) continue;
        const double ux = S.ux[p], uy = S.uy[p], uz = S.uz[p];
        const double u2 = ux * ux + uy * uy + uz * uz;
        const double e = L.m_mev * u2 / (1.0 + sqrt(1.0 + u2));
        const double sg = 1.0 / (1.0 + exp(-(e - L.ec) / L.de));
        const double ai = (double)S.w[p] * e * sg;
        const double sp = L.axis == 0 ? S.sx[p] : (L.axis == 1 ? S.sy[p] : S.sz[p]);
        a += ai;
        as += ai * sp;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        as += __shfl_down_sync(0xFFFFFFFFu, as, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, a);
        atomicAdd(sums + 1, as);
    }
}

// lambdas of the final state: dL/du, dL/ds, dL/dw (positions: zero)
template <typename R>
__global__ void __launch_bounds__(256) k_loss_grad(const AdjParticles<R> S, LossParams L, const double *sums) {
    const double A = sums[0], Lv = A > 0 ? sums[1] / A : 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < S.n; p += (long long)gridDim.x * blockDim.x) {
        S.lx[p] = R(0);
        S.ly[p] = R(0);
        S.lux[p] = S.luy[p] = S.luz[p] = R(0);
        S.lsx[p] = S.lsy[p] = S.lsz[p] = R(0);
        S.lw[p] = R(0);
        if (S.cell[p] == PIC_DEAD || !(A > 0)) continue;
        const double ux = S.ux[p], uy = S.uy[p], uz = S.uz[p];
        const double u2 = ux * ux + uy * uy + uz * uz;
        const double g = sqrt(1.0 + u2);
        const double e = L.m_mev * u2 / (1.0 + g);
        const double sg = 1.0 / (1.0 + exp(-(e - L.ec) / L.de));
        const double w = S.w[p];
        const double sp = L.axis == 0 ? S.sx[p] : (L.axis == 1 ? S.sy[p] : S.sz[p]);
        const double dla = (sp - Lv) / A;                    // dL/da_i
        const double dade = w * (sg + e * sg * (1.0 - sg) / L.de);
        const double k = dla * dade * L.m_mev / g;          // dL/du = k u  (de/du = m u / g)
        S.lux[p] = (R)(k * ux);
        S.luy[p] = (R)(k * uy);
        S.luz[p] = (R)(k * uz);
        const double ai = w * e * sg;
        (L.axis == 0 ? S.lsx : (L.axis == 1 ? S.lsy : S.lsz))[p] = (R)(ai / A);
        S.lw[p] = (R)(dla * e * sg);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename R>
cudaError_t launch_adjoint_fields(const AdjMesh<R> &A, const double *prof, double phz, double phy, double *dl_da0,
                                  cudaStream_t st) {
    const dim3 blk(256), grd((A.nx + 255) / 256, A.ny);
    const R hdx = R(0.5) * A.dt_dx, hdy = R(0.5) * A.dt_dy;
    k_adj_b_half<R><<<grd, blk, 0, st>>>(A, hdx, hdy);
    k_adj_e_full<R><<<grd, blk, 0, st>>>(A, A.dt, A.dt_dx, A.dt_dy);
    if (A.bc_x == 0)
        k_adj_boundary<R><<<(A.ny + 127) / 128, 128, 0, st>>>(A, prof, phz, phy, A.r, A.q, dl_da0);
    k_adj_b_half<R><<<grd, blk, 0, st>>>(A, hdx, hdy);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adjoint_particles(const AdjMesh<R> &A, const AdjParticles<R> &S, cudaStream_t st) {
    if (S.n == 0) return cudaSuccess;
    long long b = (S.n + 127) / 128;
    if (b > 152 * 32) b = 152 * 32;
    k_adj_particles<R><<<(int)b, 128, 0, st>>>(A, S);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_loss(const AdjParticles<R> &S, const LossParams &L, double *sums, bool grad, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int b = S.n > 0 ? (int)std::min<long long>((S.n + 255) / 256, 152 * 8) : 1;
    k_loss_sums<R><<<b, 256, 0, st>>>(S, L, sums);
    if (grad) k_loss_grad<R><<<b, 256, 0, st>>>(S, L, sums);
    return cudaGetLastError();
}

#define PIC_ADJ_INST(R)                                                                                     \
    template cudaError_t launch_adjoint_fields<R>(const AdjMesh<R> &, const double *, double, double, double *, \
                                                  cudaStream_t);                                          \
    template cudaError_t launch_adjoint_particles<R>(const AdjMesh<R> &, const AdjParticles<R> &, cudaStream_t); \
    template cudaError_t launch_loss<R>(const AdjParticles<R> &, const LossParams &, double *, bool, cudaStream_t);
PIC_ADJ_INST(float)
PIC_ADJ_INST(double)
#undef PIC_ADJ_INST
