// k_particles3.cu -- 3D3V particle kernels: the fused a1-a5 step kernel (one
// CTA per tile of TX x TY x TZ cells, 4D TMA-staged field window, shared-memory
// current window) and the split a1-a4 / a5 kernels.
#include <cuda.h>

#include "pic_device3.cuh"
#include "pic_step3.cuh"
#include "pic_kernels.h"
#include "pic_ptx.cuh"

using namespace pic_ptx;

namespace {

constexpr int kThreads3 = 256;
#ifndef PIC3_MINB
#define PIC3_MINB 4  // most resident CTAs per SM the register budget of the FP32 kernel is sized for
#endif
constexpr int kRec3 = 10;  // staged reals per particle: ox oy oz ux uy uz sx sy sz w (plus the cell word)

template <int TX, int TY, int TZ, typename R>
struct TileConst3 : WinConst3<TX, TY, TZ, R> {
    using W = WinConst3<TX, TY, TZ, R>;
    // field window, current window, one record stage per thread (cell word,
    // kRec3 reals, and the id the binned layout moves with the particle, staged
    // and kept)
    static constexpr size_t smem_bytes =
        (size_t)(6 * W::FA + 3 * W::WA) * sizeof(R) + kThreads3 * (3 * sizeof(uint32_t) + kRec3 * sizeof(R));
    // resident CTAs per SM the register budget is sized for: as many as fit
    // in the SM's 228 KB of shared memory (1 KB reserved per CTA, plus the
    // static arrays), at most PIC3_MINB, at least two; the FP64 instantiation
    // takes one.  At 2 particles per cell the kernel is latency bound, and a
    // fourth CTA (64 registers, a few spilled) beats three (80 registers).
    static constexpr int smem_ctas = (int)(228 * 1024 / (smem_bytes + 2048));
    static constexpr int minb =
        sizeof(R) == 8 ? 1 : (smem_ctas >= PIC3_MINB ? PIC3_MINB : (smem_ctas >= 3 ? 3 : 2));
};

// column `col` of the per-CTA sums of species sp (FP64 warp shuffles), ncols
// columns per row; the whole CTA calls it
template <typename R>
__device__ __forceinline__ void store_diag_rows3(const DiagParams &D, int sp, const R dacc[7], double (*sdiag)[8],
                                                 int col, int ncols) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int qd = 0; qd < 7; ++qd) {
        double v = (double)dacc[qd];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) sdiag[wid][qd] = v;
    }
    __syncthreads();
    if (tid < 7) {
        double t = 0.0;
        for (int w8 = 0; w8 < kThreads3 / 32; ++w8) t += sdiag[w8][tid];
        D.rows[((size_t)sp * 8 + tid) * ncols + col] = t;
    }
    __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
// Binned layout, the overflow range: its particles take the whole step against
// global memory (NodeBlock3) and are binned like every other particle; P.nextra
// CTAs, Eq. (4) sums in the diagnostic columns after the tiles'.  The range is
// empty unless a tile range filled since the last sort.
// ---------------------------------------------------------------------------
template <int TX, int TY, int TZ, typename R>
__global__ void __launch_bounds__(kThreads3) k_overflow3(const StepParams3<R> P) {
    __shared__ double sdiag[kThreads3 / 32][8];
    const MeshParams3<R> &m = P.m;
    const int nt = P.t.ntx * P.t.nty * P.t.ntz;
    const int tid = threadIdx.x;
    const bool diag = P.diag.on != 0;
    bool bad = false;
    for (int sp = 0; sp < P.nsp; ++sp) {
        const DevSpecies3<R> &S = P.sp[sp];
        if (!S.mobile) continue;
        const BinRange rg = bin_range(S.tile_start, P.bin[sp].cnt_in, nt + 1, nt);
        const int len = rg.len;
        R dacc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
        const R dlo = (R)P.diag.lo[sp], dhi = (R)P.diag.hi[sp], dm = (R)P.diag.m_mev[sp];
        const R dshift = diag ? (R)P.diag.shift[sp] : R(0);
        for (int k0 = blockIdx.x * kThreads3; k0 < len; k0 += P.nextra * kThreads3) {
            const int k = k0 + tid;
            int dest = -1;
            uint32_t cw = PIC_DEAD;
            R v[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) v[q] = R(0);
            int32_t id = 0;
            const int slot = k < len ? bin_slot(rg, k) : 0;
            const uint32_t c = k < len ? S.cell[slot] : PIC_DEAD;
            if (c != PIC_DEAD) {
                int ix, iy, iz;
                unpack_cell3(c, ix, iy, iz);
                const R ox = S.ox[slot], oy = S.oy[slot], oz = S.oz[slot], w = S.w[slot];
                R u[3] = {S.ux[slot], S.uy[slot], S.uz[slot]};
                R spn[3] = {S.sx[slot], S.sy[slot], S.sz[slot]};
                const NodeBlock3<R> nb(m, ix, iy, iz, P.err);
                R E[3], B[3];
                gather_eb3(nb, 1, 1, 1, ox, oy, oz, E, B);
                push_spin(S.qm, S.a, m.dt, E, B, u, spn);
                const R gi = Real<R>::rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                int ix1 = ix, iy1 = iy, iz1 = iz;
                R ox1 = ox, oy1 = oy, oz1 = oz;
                advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
                advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
                advance_axis(iz1, oz1, u[2] * gi * m.dt_dz);
                const R qw = S.q * w;
                if (ix1 == ix && iy1 == iy && iz1 == iz) {
                    R jv[12];
                    in_cell_weights3(ox, oy, oz, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt, jv);
                    deposit_in_cell3(nb, 1, 1, 1, jv);
                } else {
                    deposit_esirkepov3(nb, 1, 1, 1, ox, oy, oz, ix1 - ix + 1, iy1 - iy + 1, iz1 - iz + 1, ox1, oy1,
                                       oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt);
                }
                bad |= !finite3(u) || !finite3(spn);
                if (finish_move3(m, ix1, iy1, iz1)) {
                    if (diag) diag_add(dacc, dm, dlo, dhi, dshift, w, u, spn);
                    dest = bin_dest3<TX, TY, TZ>(m, P.t, ix1, iy1, iz1, P.err, P.bin[sp].txo);
                    cw = pack_cell3(ix1, iy1, iz1);
                    v[0] = ox1, v[1] = oy1, v[2] = oz1, v[3] = u[0], v[4] = u[1], v[5] = u[2];
                    v[6] = spn[0], v[7] = spn[1], v[8] = spn[2], v[9] = w;
                    id = S.id[slot];
                }
            }
            bin_store3(P.bin[sp], S.tile_start, nt, -1, nullptr, dest, cw, v, id, P.err);
        }
        if (diag) store_diag_rows3(P.diag, sp, dacc, sdiag, P.diag_cols0 + blockIdx.x, P.diag_cols0 + P.nextra);
    }
    if (bad) atomicOr(P.err, PIC_EF_NAN);
}

// ---------------------------------------------------------------------------
// Fused 3D step kernel.  Thread 0 stages the 6-component field window (x
// margin 4 cells before the tile, row rounded up to 16 bytes; along y and z
// the tile plus 1 + PIC3_MARGIN cells before and 2 + PIC3_MARGIN after) with
// one 4D TMA load, zero-filled outside the mesh, and alone waits for it (the
// others wait at the block barrier).  Each thread owns one record slot in
// shared memory: it copies the record it is about to process into registers
// and at once requests its next record into the same slot (cp.async), so one
// record is always in flight while it computes.  The current window is added
// to J at the end (16-byte vector atomics in float), rows outside the mesh
// wrapped onto the periodic rows.
//
// BIN = false (compact layout, periodic tile sorts, records rewritten in
// place): a particle may have drifted out of its tile since the last sort; it
// runs a1-a5 against shared memory when its stencil [cell-1, cell+2]^3 lies
// in the window and in the mesh (no wrap), else against global memory through
// a NodeBlock3 (wrapped offsets formed once, loads without branches).
//
// BIN = true (binned layout): tile T reads its two segments and every
// surviving particle is stored into the range of the tile its new cell lies
// in, in the other buffer (bin_store3); k_overflow3 runs the overflow range.
// The binned layout keeps every particle in its tile, so every stencil lies in
// the window: the window of a tile at a periodic edge (y, z, and x when
// periodic) is completed from the wrapped rows after the TMA load (which
// fills rows outside the mesh with zeros), and there is no global-memory
// path.  A warp whose lanes all stay in their cells deposits with the in-cell
// closed form; once any lane crosses a cell face the whole warp takes the
// general Esirkepov form, which gives the in-cell lanes the same values, so
// the two forms never run one after the other in a warp.
//
// DIAG: the step accumulates the Eq. (4) sums (the instantiation without them
// keeps their registers free).
// ---------------------------------------------------------------------------
// g mod n in [0, n): one compare each way for a window row next to the mesh,
// the remainder only when a window spans more than a short mesh axis
static __device__ __forceinline__ int wrap3(int g, int n) {
    g = g < 0 ? g + n : (g >= n ? g - n : g);
    if (g < 0 || g >= n) {
        g %= n;
        if (g < 0) g += n;
    }
    return g;
}

template <int TX, int TY, int TZ, typename R, bool BIN, bool DIAG>
__global__ void __launch_bounds__(kThreads3, (TileConst3<TX, TY, TZ, R>::minb))
    k_step_fused3(const StepParams3<R> P, const __grid_constant__ CUtensorMap tmapEB) {
    using TC = TileConst3<TX, TY, TZ, R>;
    constexpr int WX = TC::WX, WY = TC::WY, WZ = TC::WZ, WA = TC::WA, FX = TC::FX, FA = TC::FA;
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double sdiag[kThreads3 / 32][8];
    __shared__ int s_front[PIC_MAXSP];  // binned layout: stayers stored per species
    __shared__ int s_timeout;
    R *sF = reinterpret_cast<R *>(dsm);
    R *sJ = sF + 6 * FA;
    R *ring = sJ + 3 * WA;                                                // [kRec3][kThreads3]
    uint32_t *cring = reinterpret_cast<uint32_t *>(ring + kRec3 * kThreads3);  // [kThreads3]
    int32_t *iring = reinterpret_cast<int32_t *>(cring + kThreads3);          // [kThreads3]
    const MeshParams3<R> &m = P.m;

    const int tile = blockIdx.x;
    const int tz = tile / (P.t.ntx * P.t.nty);
    const int rem = tile - tz * P.t.ntx * P.t.nty;
    const int ty = rem / P.t.ntx, tx = rem - ty * P.t.ntx;
    const int wx0 = tx * TX - TC::HX, wy0 = ty * TY - TC::HY, wz0 = tz * TZ - TC::HZ;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, (unsigned)(6 * FA * sizeof(R)));
        tma_load_4d(sF, &tmapEB, &bar, wx0, wy0, wz0, 0);
    }

    R *ring0 = ring + tid;
    auto prefetch = [&](const DevSpecies3<R> &S, int slot, bool live) {
        if (live) {
            R *r = ring0;
            cp_async4(cring + tid, S.cell + slot);
            cp_async_r(r + 0 * kThreads3, S.ox + slot);
            cp_async_r(r + 1 * kThreads3, S.oy + slot);
            cp_async_r(r + 2 * kThreads3, S.oz + slot);
            cp_async_r(r + 3 * kThreads3, S.ux + slot);
            cp_async_r(r + 4 * kThreads3, S.uy + slot);
            cp_async_r(r + 5 * kThreads3, S.uz + slot);
            cp_async_r(r + 6 * kThreads3, S.sx + slot);
            cp_async_r(r + 7 * kThreads3, S.sy + slot);
            cp_async_r(r + 8 * kThreads3, S.sz + slot);
            cp_async_r(r + 9 * kThreads3, S.w + slot);
            if constexpr (BIN) cp_async4(iring + tid, S.id + slot);
        }
        cp_async_commit();
    };
    // binned: the range this tile's particles of species sp live in
    auto own = [&](int sp) { return tile - tx + bin_rot_x(tx, P.t.ntx, P.bin[sp].txo); };
    // the particles of this tile: bin_slot(range, k), k < range.len
    auto range = [&](int sp) {
        const DevSpecies3<R> &S = P.sp[sp];
        if constexpr (BIN) return bin_range(S.tile_start, P.bin[sp].cnt_in, (int)gridDim.x + 1, own(sp));
        BinRange b;
        b.beg = S.tile_start[tile];
        b.len = b.front = b.split = S.tile_start[tile + 1] - b.beg;
        return b;
    };

    constexpr bool diag = DIAG;  // Eq. (4) sums on this step (a separate instantiation)
    int first = -1;
    for (int sp = 0; sp < P.nsp && first < 0; ++sp)
        if (P.sp[sp].mobile) first = sp;
    if (first >= 0) {
        const BinRange rg = range(first);
        prefetch(P.sp[first], tid < rg.len ? bin_slot(rg, tid) : 0, tid < rg.len);
    }
    if constexpr (sizeof(R) == 4) {
        float4 *j4 = reinterpret_cast<float4 *>(sJ);  // 3 WA is a multiple of 4, sJ 16-byte aligned
        for (int i = tid; i < 3 * WA / 4; i += kThreads3) j4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int i = tid; i < 3 * WA; i += kThreads3) sJ[i] = R(0);
    }
    if (tid < PIC_MAXSP) s_front[tid] = 0;
    if (tid == 0) s_timeout = mbar_wait_bounded(&bar, 0) ? 0 : 1;  // one thread waits for the window
    __syncthreads();
    if (s_timeout) {
        if (tid == 0) atomicOr(P.err, PIC_EF_TIMEOUT);
        cp_async_wait0();
        return;
    }
    if constexpr (BIN) {
        // window rows outside the mesh: the wrapped rows' values
        const bool wrap_x = m.bc_x == 1 && (wx0 < 0 || wx0 + FX > m.nx);
        if (wy0 < 0 || wy0 + WY > m.ny || wz0 < 0 || wz0 + WZ > m.nz || wrap_x) {
            for (int e = tid; e < 6 * WZ * WY * FX; e += kThreads3) {
                const int row = e / FX, x = e - row * FX;
                const int c = row / (WZ * WY), zy = row - c * (WZ * WY);
                const int z = zy / WY, y = zy - z * WY;
                const int gz = wz0 + z, gy = wy0 + y;
                const bool row_out = gz < 0 || gz >= m.nz || gy < 0 || gy >= m.ny;
                int gx = wx0 + x;
                if (m.bc_x == 1) gx = wrap3(gx, m.nx);
                if (!row_out && gx == wx0 + x) continue;  // in the mesh: the TMA loaded it
                const size_t g = c * m.plane + ((size_t)wrap3(gz, m.nz) * m.ny + wrap3(gy, m.ny)) * m.ld;
                sF[c * FA + zy * FX + x] = gx >= 0 && gx < m.ld ? m.EB[g + gx] : R(0);
            }
            __syncthreads();
        }
    }

    const SmemMesh3T<R, WX, WY, WA, FX, FA> sm{sF, sJ};
    const int xlo = max(wx0 + 1, 1), xhi = min(wx0 + WX - 3, m.nx - 3);
    const int ylo = max(wy0 + 1, 1), yhi = min(wy0 + WY - 3, m.ny - 3);
    const int zlo = max(wz0 + 1, 1), zhi = min(wz0 + WZ - 3, m.nz - 3);
    const int tx0 = wx0 + TC::HX, ty0 = wy0 + TC::HY, tz0 = wz0 + TC::HZ;
    bool bad = false;

    for (int sp = 0; sp < P.nsp; ++sp) {
        const DevSpecies3<R> &S = P.sp[sp];
        if (!S.mobile) continue;
        const BinRange rg = range(sp);
        const int len = rg.len;
        const R qm = S.qm, a = S.a, q = S.q;
        double *drow = sdiag[tid >> 5];  // this warp's Eq. (4) sums of the species (lanes 4 q add sum q)
        if (diag) {
            if ((tid & 31) < 8) drow[tid & 31] = 0.0;
            __syncwarp();
        }
        if (sp != first) prefetch(S, tid < len ? bin_slot(rg, tid) : 0, tid < len);
        for (int k0 = 0; k0 < len; k0 += kThreads3) {
            const int k = k0 + tid;
            cp_async_wait0();
            if constexpr (BIN) {
                // this lane's particle: a1-a4, then the deposit (form chosen per warp)
                bool valid = false;
                int ix = 0, iy = 0, iz = 0, ix1 = 0, iy1 = 0, iz1 = 0;
                R ox = R(0), oy = R(0), oz = R(0), ox1 = R(0), oy1 = R(0), oz1 = R(0), w = R(0);
                R u[3] = {R(0), R(0), R(0)}, spn[3] = {R(0), R(0), R(0)};
                int32_t id = 0;
                if (k < len) {
                    const R *r = ring0;
                    const uint32_t c = cring[tid];
                    ox = r[0 * kThreads3], oy = r[1 * kThreads3], oz = r[2 * kThreads3];
                    u[0] = r[3 * kThreads3], u[1] = r[4 * kThreads3], u[2] = r[5 * kThreads3];
                    spn[0] = r[6 * kThreads3], spn[1] = r[7 * kThreads3], spn[2] = r[8 * kThreads3];
                    w = r[9 * kThreads3];
                    id = iring[tid];
                    // the slot is free again: request the next record
                    prefetch(S, k + kThreads3 < len ? bin_slot(rg, k + kThreads3) : 0, k + kThreads3 < len);
                    if (c != PIC_DEAD) {
                        unpack_cell3(c, ix, iy, iz);
                        if (ix < tx0 || ix >= tx0 + TX || iy < ty0 || iy >= ty0 + TY || iz < tz0 ||
                            iz >= tz0 + TZ) {
                            atomicOr(P.err, PIC_EF_RANGE);  // not in its tile: only a corrupt layout
                        } else {
                            valid = true;
                            R E[3], B[3];
                            gather_eb3(sm, ix - wx0, iy - wy0, iz - wz0, ox, oy, oz, E, B);
                            push_spin(qm, a, m.dt, E, B, u, spn);
                            const R gi = Real<R>::rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                            ix1 = ix, iy1 = iy, iz1 = iz;
                            ox1 = ox, oy1 = oy, oz1 = oz;
                            advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
                            advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
                            advance_axis(iz1, oz1, u[2] * gi * m.dt_dz);
                        }
                    }
                }
                const bool cross = valid && (ix1 != ix || iy1 != iy || iz1 != iz);
                const bool general = __any_sync(0xFFFFFFFFu, cross);
                int dest = -1;
                uint32_t bcell = PIC_DEAD;
                R bv[10];
#pragma unroll
                for (int q10 = 0; q10 < 10; ++q10) bv[q10] = R(0);
                bool dhas = false;
                if (valid) {
                    const R qw = q * w;
                    if (general) {
                        deposit_esirkepov3(sm, ix - wx0, iy - wy0, iz - wz0, ox, oy, oz, ix1 - wx0, iy1 - wy0,
                                           iz1 - wz0, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt);
                    } else {
                        R v[12];
                        in_cell_weights3(ox, oy, oz, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt, v);
                        deposit_in_cell3(sm, ix - wx0, iy - wy0, iz - wz0, v);
                    }
                    const bool alive = finish_move3(m, ix1, iy1, iz1);
                    const R chk = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + spn[0] * spn[0] + spn[1] * spn[1] +
                                  spn[2] * spn[2];
                    bad |= !isfinite(chk);
                    if (alive) {
                        dhas = DIAG;
                        dest = bin_dest3<TX, TY, TZ>(m, P.t, ix1, iy1, iz1, P.err, P.bin[sp].txo);
                        bcell = pack_cell3(ix1, iy1, iz1);
                        bv[0] = ox1, bv[1] = oy1, bv[2] = oz1, bv[3] = u[0], bv[4] = u[1], bv[5] = u[2];
                        bv[6] = spn[0], bv[7] = spn[1], bv[8] = spn[2], bv[9] = w;
                    }
                }
                if constexpr (DIAG) diag_warp(P.diag, sp, dhas, w, u, spn, drow);
                bin_store3(P.bin[sp], S.tile_start, (int)gridDim.x, own(sp), &s_front[sp], dest, bcell, bv, id, P.err,
                           rg.beg);
            } else {
                // Eq. (4) contribution of this lane's record, summed over the warp below
                bool dhas = false;
                R dw = R(0), du[3] = {R(0), R(0), R(0)}, ds[3] = {R(0), R(0), R(0)};
                if (k < len) {
                    const int slot = rg.beg + k;  // compact layout (in-place rewrite)
                    const R *r = ring0;
                    const uint32_t c = cring[tid];
                    const R ox = r[0 * kThreads3], oy = r[1 * kThreads3], oz = r[2 * kThreads3];
                    R u[3] = {r[3 * kThreads3], r[4 * kThreads3], r[5 * kThreads3]};
                    R spn[3] = {r[6 * kThreads3], r[7 * kThreads3], r[8 * kThreads3]};
                    const R w = r[9 * kThreads3];
                    // the slot is free again: request the next record
                    prefetch(S, k + kThreads3 < len ? bin_slot(rg, k + kThreads3) : 0, k + kThreads3 < len);
                    if (c != PIC_DEAD) {
                        int ix, iy, iz;
                        unpack_cell3(c, ix, iy, iz);
                        const bool fast =
                            ix >= xlo && ix <= xhi && iy >= ylo && iy <= yhi && iz >= zlo && iz <= zhi;
                        R E[3], B[3];
                        if (fast) {
                            gather_eb3(sm, ix - wx0, iy - wy0, iz - wz0, ox, oy, oz, E, B);
                        } else {
                            const NodeBlock3<R> nb(m, ix, iy, iz, P.err);
                            gather_eb3(nb, 1, 1, 1, ox, oy, oz, E, B);
                        }
                        push_spin(qm, a, m.dt, E, B, u, spn);
                        const R gi = Real<R>::rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                        int ix1 = ix, iy1 = iy, iz1 = iz;
                        R ox1 = ox, oy1 = oy, oz1 = oz;
                        advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
                        advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
                        advance_axis(iz1, oz1, u[2] * gi * m.dt_dz);
                        const R qw = q * w;
                        const bool in_cell = ix1 == ix && iy1 == iy && iz1 == iz;
                        if (fast && in_cell) {
                            R v[12];
                            in_cell_weights3(ox, oy, oz, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt, v);
                            deposit_in_cell3(sm, ix - wx0, iy - wy0, iz - wz0, v);
                        } else if (fast) {
                            deposit_esirkepov3(sm, ix - wx0, iy - wy0, iz - wz0, ox, oy, oz, ix1 - wx0, iy1 - wy0,
                                               iz1 - wz0, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt);
                        } else {
                            const NodeBlock3<R> nb(m, ix, iy, iz, P.err);
                            if (in_cell) {
                                R v[12];
                                in_cell_weights3(ox, oy, oz, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt, v);
                                deposit_in_cell3(nb, 1, 1, 1, v);
                            } else {
                                deposit_esirkepov3(nb, 1, 1, 1, ox, oy, oz, ix1 - ix + 1, iy1 - iy + 1,
                                                   iz1 - iz + 1, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt);
                            }
                        }
                        const bool alive = finish_move3(m, ix1, iy1, iz1);
                        const R chk = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + spn[0] * spn[0] +
                                      spn[1] * spn[1] + spn[2] * spn[2];
                        bad |= !isfinite(chk);
                        if (diag && alive) {
                            dhas = true;
                            dw = w;
                            du[0] = u[0], du[1] = u[1], du[2] = u[2];
                            ds[0] = spn[0], ds[1] = spn[1], ds[2] = spn[2];
                        }
                        S.cell[slot] = alive ? pack_cell3(ix1, iy1, iz1) : PIC_DEAD;
                        S.ox[slot] = ox1;
                        S.oy[slot] = oy1;
                        S.oz[slot] = oz1;
                        S.ux[slot] = u[0];
                        S.uy[slot] = u[1];
                        S.uz[slot] = u[2];
                        S.sx[slot] = spn[0];
                        S.sy[slot] = spn[1];
                        S.sz[slot] = spn[2];
                    }
                }
                if constexpr (DIAG) diag_warp(P.diag, sp, dhas, dw, du, ds, drow);
            }
        }
        cp_async_wait0();
        if (diag)  // diagnostic columns: the tiles, then (binned) the overflow CTAs
            store_diag_sums(P.diag, sp, sdiag, kThreads3 / 32, (int)blockIdx.x, (int)gridDim.x + (BIN ? P.nextra : 0));
    }
    if (bad) atomicOr(P.err, PIC_EF_NAN);
    __syncthreads();
    if constexpr (BIN) {
        // the destination range of this tile: its stayers, and where its arrivals start
        if (tid < P.nsp && P.sp[tid].mobile) {
            const int nr = (int)gridDim.x + 1;
            const int r = own(tid);
            P.bin[tid].cnt_out[r] = s_front[tid];
            P.bin[tid].cnt_out[nr + r] = range(tid).len;
        }
    }

    // current window -> J: rows outside the mesh wrapped onto the periodic
    // rows (only the binned layout deposits there), all-zero groups skipped
    if constexpr (sizeof(R) == 4) {
        constexpr int WQ = WX / 4;
        for (int qd = tid; qd < 3 * WZ * WY * WQ; qd += kThreads3) {
            const int row = qd / WQ, xq = qd - row * WQ;
            const int c = row / (WZ * WY), zy = row - c * WZ * WY;
            const int z = zy / WY, y = zy - z * WY;
            const float4 v = *reinterpret_cast<const float4 *>(&sJ[c * WA + zy * WX + 4 * xq]);
            if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
            const int gz = wrap3(wz0 + z, m.nz), gy = wrap3(wy0 + y, m.ny), gx = wx0 + 4 * xq;
            R *row0 = m.J + c * m.plane + ((size_t)gz * m.ny + gy) * m.ld;
            if (gx >= 0 && gx + 3 < m.nx) {
                atomicAdd(reinterpret_cast<float4 *>(row0 + gx), v);
            } else {
                const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    int x = gx + q4;
                    if (m.bc_x == 1) x = wrap3(x, m.nx);
                    if (e[q4] != 0.f && x >= 0 && x < m.nx) atomicAdd(row0 + x, e[q4]);
                }
            }
        }
    } else {
        for (int e = tid; e < 3 * WA; e += kThreads3) {
            const R v = sJ[e];
            if (v == R(0)) continue;
            const int row = e / WX, x = e - row * WX;
            const int c = row / (WZ * WY), zy = row - c * WZ * WY;
            const int z = zy / WY, y = zy - z * WY;
            const int gz = wrap3(wz0 + z, m.nz), gy = wrap3(wy0 + y, m.ny);
            int gx = wx0 + x;
            if (m.bc_x == 1) gx = wrap3(gx, m.nx);
            if (gx < 0 || gx >= m.nx) continue;
            atomicAdd(&m.J[c * m.plane + ((size_t)gz * m.ny + gy) * m.ld + gx], v);
        }
    }
}

// ---------------------------------------------------------------------------
// Split path, a1-a4 (one thread per slot, global-memory gather); keeps x^n for
// the deposit and stores the unwrapped new cell shifted by +1 per axis.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_push_split3(const StepParams3<R> P, int s) {
    const DevSpecies3<R> &S = P.sp[s];
    const MeshParams3<R> &m = P.m;
    unsigned bad = 0;
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[p];
        S.cell_old[p] = c;
        if (c == PIC_DEAD) continue;
        int ix, iy, iz;
        unpack_cell3(c, ix, iy, iz);
        const R ox = S.ox[p], oy = S.oy[p], oz = S.oz[p];
        R u[3] = {S.ux[p], S.uy[p], S.uz[p]};
        R sp[3] = {S.sx[p], S.sy[p], S.sz[p]};
        R E[3], B[3];
        const NodeBlock3<R> nb(m, ix, iy, iz, P.err);
        gather_eb3(nb, 1, 1, 1, ox, oy, oz, E, B);
        push_spin(S.qm, S.a, m.dt, E, B, u, sp);
        const R gi = Real<R>::rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        int ix1 = ix, iy1 = iy, iz1 = iz;
        R ox1 = ox, oy1 = oy, oz1 = oz;
        advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
        advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
        advance_axis(iz1, oz1, u[2] * gi * m.dt_dz);
        if (!finite3(u) || !finite3(sp)) bad |= PIC_EF_NAN;
        S.ox_old[p] = ox;
        S.oy_old[p] = oy;
        S.oz_old[p] = oz;
        S.cell[p] = pack_cell3(ix1 + 1, iy1 + 1, iz1 + 1);
        S.ox[p] = ox1;
        S.oy[p] = oy1;
        S.oz[p] = oz1;
        S.ux[p] = u[0];
        S.uy[p] = u[1];
        S.uz[p] = u[2];
        S.sx[p] = sp[0];
        S.sy[p] = sp[1];
        S.sz[p] = sp[2];
    }
    if (bad) atomicOr(P.err, bad);
}

// Split path, a5: current of the recorded move, then the wrap / removal.
template <typename R>
__global__ void __launch_bounds__(256) k_deposit_split3(const StepParams3<R> P, int s) {
    const DevSpecies3<R> &S = P.sp[s];
    const MeshParams3<R> &m = P.m;
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c0 = S.cell_old[p];
        if (c0 == PIC_DEAD) continue;
        int ix, iy, iz, ix1, iy1, iz1;
        unpack_cell3(c0, ix, iy, iz);
        unpack_cell3(S.cell[p], ix1, iy1, iz1);
        ix1 -= 1;
        iy1 -= 1;
        iz1 -= 1;
        const R ox = S.ox_old[p], oy = S.oy_old[p], oz = S.oz_old[p];
        const R ox1 = S.ox[p], oy1 = S.oy[p], oz1 = S.oz[p];
        const R qw = S.q * S.w[p];
        const NodeBlock3<R> nb(m, ix, iy, iz, P.err);
        if (ix1 == ix && iy1 == iy && iz1 == iz) {
            R v[12];
            in_cell_weights3(ox, oy, oz, ox1, oy1, oz1, qw, m.dx_dt, m.dy_dt, m.dz_dt, v);
            deposit_in_cell3(nb, 1, 1, 1, v);
        } else {
            deposit_esirkepov3(nb, 1, 1, 1, ox, oy, oz, ix1 - ix + 1, iy1 - iy + 1, iz1 - iz + 1, ox1, oy1, oz1, qw,
                               m.dx_dt, m.dy_dt, m.dz_dt);
        }
        const bool alive = finish_move3(m, ix1, iy1, iz1);
        S.cell[p] = alive ? pack_cell3(ix1, iy1, iz1) : PIC_DEAD;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int TX, int TY, int TZ, typename R, bool BIN, bool DIAG>
static cudaError_t launch_fused3_t(const StepParams3<R> &P, const CUtensorMap &tmapEB, cudaStream_t st) {
    using TC = TileConst3<TX, TY, TZ, R>;
    constexpr size_t smem = TC::smem_bytes;
    if (P.t.WX != TC::WX || P.t.WY != TC::WY || P.t.WZ != TC::WZ || P.t.FX != TC::FX || P.t.HX != TC::HX ||
        P.t.HY != TC::HY || P.t.HZ != TC::HZ)
        return cudaErrorInvalidValue;
    if (BIN && P.nextra < 1) return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fused3<TX, TY, TZ, R, BIN, DIAG>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_step_fused3<TX, TY, TZ, R, BIN, DIAG><<<P.t.ntx * P.t.nty * P.t.ntz, kThreads3, smem, st>>>(P, tmapEB);
    if (BIN) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_overflow3<TX, TY, TZ, R><<<P.nextra, kThreads3, 0, st>>>(P);
    }
    return cudaGetLastError();
}

template <int TX, int TY, int TZ, typename R>
static cudaError_t launch_fused3_b(const StepParams3<R> &P, const CUtensorMap &tmapEB, bool binned,
                                   cudaStream_t st) {
    const bool diag = P.diag.on != 0;
    if (binned)
        return diag ? launch_fused3_t<TX, TY, TZ, R, true, true>(P, tmapEB, st)
                    : launch_fused3_t<TX, TY, TZ, R, true, false>(P, tmapEB, st);
    return diag ? launch_fused3_t<TX, TY, TZ, R, false, true>(P, tmapEB, st)
                : launch_fused3_t<TX, TY, TZ, R, false, false>(P, tmapEB, st);
}

bool fused3_tile_supported(int tx, int ty, int tz) {
    return (tx == 8 && ty == 8 && tz == 4) || (tx == 16 && ty == 4 && tz == 4) || (tx == 8 && ty == 4 && tz == 4) ||
           (tx == 16 && ty == 8 && tz == 4) || (tx == 32 && ty == 4 && tz == 4);
}

template <typename R>
cudaError_t launch_step_fused3(const StepParams3<R> &P, const CUtensorMap &tmapEB, bool binned, cudaStream_t st) {
    const int tx = P.t.TX, ty = P.t.TY, tz = P.t.TZ;
    if (tx == 8 && ty == 8 && tz == 4) return launch_fused3_b<8, 8, 4, R>(P, tmapEB, binned, st);
    if (tx == 16 && ty == 4 && tz == 4) return launch_fused3_b<16, 4, 4, R>(P, tmapEB, binned, st);
    if (tx == 8 && ty == 4 && tz == 4) return launch_fused3_b<8, 4, 4, R>(P, tmapEB, binned, st);
    if (tx == 16 && ty == 8 && tz == 4) return launch_fused3_b<16, 8, 4, R>(P, tmapEB, binned, st);
    if (tx == 32 && ty == 4 && tz == 4) return launch_fused3_b<32, 4, 4, R>(P, tmapEB, binned, st);
    return cudaErrorInvalidValue;
}

static int blocks3_for(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b);
}

template <typename R>
cudaError_t launch_push_split3(const StepParams3<R> &P, int s, int n_upper, cudaStream_t st) {
    k_push_split3<R><<<blocks3_for(n_upper), 256, 0, st>>>(P, s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_deposit_split3(const StepParams3<R> &P, int s, int n_upper, cudaStream_t st) {
    k_deposit_split3<R><<<blocks3_for(n_upper), 256, 0, st>>>(P, s);
    return cudaGetLastError();
}

template cudaError_t launch_step_fused3<float>(const StepParams3<float> &, const CUtensorMap &, bool, cudaStream_t);
template cudaError_t launch_step_fused3<double>(const StepParams3<double> &, const CUtensorMap &, bool, cudaStream_t);
template cudaError_t launch_push_split3<float>(const StepParams3<float> &, int, int, cudaStream_t);
template cudaError_t launch_push_split3<double>(const StepParams3<double> &, int, int, cudaStream_t);
template cudaError_t launch_deposit_split3<float>(const StepParams3<float> &, int, int, cudaStream_t);
template cudaError_t launch_deposit_split3<double>(const StepParams3<double> &, int, int, cudaStream_t);
