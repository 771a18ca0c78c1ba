// k_particles.cu -- particle kernels: the fused a1-a5 step kernel (one CTA
// per tile, TMA-staged field window, shared-memory current window) and the
// split a1-a4 / a5 kernels behind pic_gather_push_spin / pic_deposit.
#include <cuda.h>

#include "pic_device.cuh"
#include "pic_kernels.h"
#include "pic_ptx.cuh"

using namespace pic_ptx;

namespace {

// a4 and the boundary rule shared by both paths; returns false if removed
template <typename R>
__device__ __forceinline__ bool finish_move(const MeshParams<R> &m, int &ix1, int &iy1) {
    bool alive = true;
    if (m.bc_x == 0) {
        alive = ix1 >= 2 && ix1 <= m.nx - 3;
    } else {
        if (ix1 < 0) ix1 += m.nx;
        else if (ix1 >= m.nx) ix1 -= m.nx;
    }
    if (iy1 < 0) iy1 += m.ny;
    else if (iy1 >= m.ny) iy1 -= m.ny;
    return alive;
}

}  // namespace

// ---------------------------------------------------------------------------
// Fused step kernel.  CTA = one tile of TX x TY cells (compile-time, so every
// shared-memory offset below is an immediate).  Thread 0 stages the
// 6-component field window (rows padded to 128 bytes with the padding split
// between the two sides of the tile, at least 4 cells each; 6 cells of
// margin along y) with one 3D TMA load (zero fill outside the mesh).  Particle records of the tile (both
// species, one slot range after the other) stream through one shared-memory
// slot per thread: a thread copies the record in hand to registers and at once
// requests its next record into the slot (cp.async), so while it computes one
// record it has the next one in flight.  Each record runs a1-a5, gathering from and
// depositing into shared memory when the particle's 4x4 stencil lies inside
// the window and the mesh (no wrap), otherwise through global memory.  The
// current window is finally added to J with 16-byte vector atomics (float)
// or scalar atomics (double).
// ---------------------------------------------------------------------------
constexpr int kFusedThreads = 256;
#ifndef PIC_FUSED_MINB
#define PIC_FUSED_MINB 3  // resident CTAs per SM the register budget is sized for
#endif
constexpr int kRec = 9;  // staged reals per particle: ox oy ux uy uz sx sy sz w (plus the cell word)

template <int TX, int TY, typename R>
struct TileConst {
    static constexpr int WX = window_wx<R>(TX), WY = window_wy(TY), WA = WX * WY;
    static constexpr int HX = window_hx<R>(TX), HY = window_hy();
    // field window, current window, and one record slot per thread (cell word
    // and reals)
    static constexpr size_t smem_bytes =
        (size_t)9 * WA * sizeof(R) + kFusedThreads * (sizeof(uint32_t) + kRec * sizeof(R));
    // resident CTAs per SM the register budget of the single-run kernel is
    // sized for: without the in-step Eq. (4) sums a fourth CTA where four fit
    // in shared memory (228 KB, 1 KB reserved per CTA), else PIC_FUSED_MINB
    static constexpr int minb_nodiag =
        sizeof(R) == 8 ? 2 : ((int)(228 * 1024 / (smem_bytes + 2048)) >= 4 ? 4 : PIC_FUSED_MINB);
};

template <typename R, int WX, int WA>
struct SmemMeshT {
    const R *F;
    R *Jw;
    __device__ __forceinline__ R f(int c, int x, int y) const { return F[c * WA + y * WX + x]; }
    __device__ __forceinline__ void j(int c, int x, int y, R v) const { atomicAdd(&Jw[c * WA + y * WX + x], v); }
};

// J window -> global J
template <typename R>
__device__ __forceinline__ void flush_add(R *dst, const R *src);
template <>
__device__ __forceinline__ void flush_add<float>(float *dst, const float *src) {
    const float4 v = *reinterpret_cast<const float4 *>(src);
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) return;
    atomicAdd(reinterpret_cast<float4 *>(dst), v);
}
template <>
__device__ __forceinline__ void flush_add<double>(double *dst, const double *src) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (src[k] != 0.0) atomicAdd(dst + k, src[k]);
}
// One tile of the fused step: the body of k_step_fused (one CTA per tile) and
// of k_step_fused_batch (persistent CTAs taking tiles of many runs).  `bar`
// is an initialised mbarrier whose current phase has parity `phase`; `ntiles`
// is the run's tile count (the stride of the diagnostic rows).  Returns false
// if the window wait gave up.
template <int TX, int TY, typename R, bool DIAG = true>
__device__ __forceinline__ bool fused_tile(const StepParams<R> &P, const CUtensorMap *tmap, const int tile,
                                           const int ntiles, uint64_t &bar, const unsigned phase,
                                           unsigned char *dsm, double (*sdiag)[8]) {
    using TC = TileConst<TX, TY, R>;
    constexpr int WX = TC::WX, WY = TC::WY, WA = TC::WA;
    R *sF = reinterpret_cast<R *>(dsm);
    R *sJ = sF + 6 * WA;
    R *ring = sJ + 3 * WA;                                             // [kRec][kFusedThreads]
    uint32_t *cring = reinterpret_cast<uint32_t *>(ring + kRec * kFusedThreads);  // [kFusedThreads]
    const MeshParams<R> &m = P.m;

    const int ty = tile / P.t.ntx, tx = tile - ty * P.t.ntx;
    const int wx0 = tx * TX - TC::HX, wy0 = ty * TY - TC::HY;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_expect_tx(&bar, (unsigned)(6 * WA * sizeof(R)));
        tma_load_3d(sF, tmap, &bar, wx0, wy0, 0);
    }

    R *ring0 = ring + tid;
    // particle record `slot` of species S into this thread's record slot (the
    // thread copies the record in hand to registers first, so one record is
    // in flight while it computes)
    auto prefetch = [&](const DevSpecies<R> &S, int slot, bool live) {
        if (live) {
            R *r = ring0;
            cp_async4(cring + tid, S.cell + slot);
            cp_async_r(r + 0 * kFusedThreads, S.ox + slot);
            cp_async_r(r + 1 * kFusedThreads, S.oy + slot);
            cp_async_r(r + 2 * kFusedThreads, S.ux + slot);
            cp_async_r(r + 3 * kFusedThreads, S.uy + slot);
            cp_async_r(r + 4 * kFusedThreads, S.uz + slot);
            cp_async_r(r + 5 * kFusedThreads, S.sx + slot);
            cp_async_r(r + 6 * kFusedThreads, S.sy + slot);
            cp_async_r(r + 7 * kFusedThreads, S.sz + slot);
            cp_async_r(r + 8 * kFusedThreads, S.w + slot);
        }
        cp_async_commit();
    };

    // Eq. (4) diagnostic sums of one species: float per thread (at most
    // total/256 particles each), then double across the CTA (sdiag)
    const bool diag = DIAG && P.diag.on != 0;  // DIAG = false: the sums are compiled out

    // the first record of the first mobile species is requested before the
    // window wait, so both latencies overlap
    int first = -1;
    for (int sp = 0; sp < P.nsp && first < 0; ++sp)
        if (P.sp[sp].mobile) first = sp;
    if (first >= 0) {
        const int beg = P.sp[first].tile_start[tile];
        prefetch(P.sp[first], beg + tid, tid < P.sp[first].tile_start[tile + 1] - beg);
    }
    for (int i = tid; i < 3 * WA; i += kFusedThreads) sJ[i] = R(0);
    __syncthreads();
    if (!mbar_wait_bounded(&bar, phase)) {
        if (tid == 0) atomicOr(P.err, PIC_EF_TIMEOUT);
        cp_async_wait0();
        return false;
    }

    const SmemMeshT<R, WX, WA> sm{sF, sJ};
    const GlobalMesh<R> gm{m.EB, m.J, m.nx, m.ny, m.ld, m.bc_x == 1, m.plane, P.err};
    // window interior where a whole stencil [i-1, i+2] fits, intersected with the mesh
    const int xlo = max(wx0 + 1, 1), xhi = min(wx0 + WX - 3, m.nx - 3);
    const int ylo = max(wy0 + 1, 1), yhi = min(wy0 + WY - 3, m.ny - 3);
    bool bad = false;
    // In-cell moves (the common case) of consecutive particles of the same
    // cell are summed in registers and added to the shared window once, at
    // the next change of cell: with the layered tile order each thread meets
    // the same cell on every pass through the layers.
    int acc_key = -1;  // window offset of the accumulated cell
    R acc[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    auto acc_flush = [&]() {
        if (acc_key >= 0) {
            atomicAdd(&sJ[acc_key], acc[0]);
            atomicAdd(&sJ[acc_key + WX], acc[1]);
            atomicAdd(&sJ[WA + acc_key], acc[2]);
            atomicAdd(&sJ[WA + acc_key + 1], acc[3]);
            atomicAdd(&sJ[2 * WA + acc_key], acc[4]);
            atomicAdd(&sJ[2 * WA + acc_key + 1], acc[5]);
            atomicAdd(&sJ[2 * WA + acc_key + WX], acc[6]);
            atomicAdd(&sJ[2 * WA + acc_key + WX + 1], acc[7]);
        }
    };

    for (int sp = 0; sp < P.nsp; ++sp) {
        const DevSpecies<R> &S = P.sp[sp];
        if (!S.mobile) continue;
        const int beg = S.tile_start[tile], len = S.tile_start[tile + 1] - beg;
        const R qm = S.qm, a = S.a, q = S.q;
        double *drow = sdiag[tid >> 5];  // this warp's Eq. (4) sums of the species (lanes 4 q add sum q)
        if (diag) {
            if ((tid & 31) < 8) drow[tid & 31] = 0.0;
            __syncwarp();
        }
        if (sp != first) prefetch(S, beg + tid, tid < len);
        for (int k0 = 0; k0 < len; k0 += kFusedThreads) {
            const int k = k0 + tid;
            cp_async_wait0();
            // this lane's contribution to the Eq. (4) sums, summed over the warp below
            bool dhas = false;
            R dw = R(0), du[3] = {R(0), R(0), R(0)}, ds[3] = {R(0), R(0), R(0)};
            if (k < len) {
                const int slot = beg + k;
                const R *r = ring0;
                const uint32_t c = cring[tid];
                const R ox = r[0 * kFusedThreads], oy = r[1 * kFusedThreads];
                R u[3] = {r[2 * kFusedThreads], r[3 * kFusedThreads], r[4 * kFusedThreads]};
                R spn[3] = {r[5 * kFusedThreads], r[6 * kFusedThreads], r[7 * kFusedThreads]};
                const R w = r[8 * kFusedThreads];
                // the slot is free again: request the next record
                prefetch(S, beg + k + kFusedThreads, k + kFusedThreads < len);
                if (c != PIC_DEAD) {
                    const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
                    const bool fast = ix >= xlo && ix <= xhi && iy >= ylo && iy <= yhi;
                    R E[3], B[3];
                    if (fast)
                        gather_eb(sm, ix - wx0, iy - wy0, ox, oy, E, B);
                    else
                        gather_eb(gm, ix, iy, ox, oy, E, B);
                    push_spin(qm, a, m.dt, E, B, u, spn);
                    const R gi = Real<R>::rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                    int ix1 = ix, iy1 = iy;
                    R ox1 = ox, oy1 = oy;
                    advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
                    advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
                    const R qw = q * w, vz = u[2] * gi;
                    if (fast && ix1 == ix && iy1 == iy) {
                        // in-cell Esirkepov weights, summed per cell
                        const int key = (iy - wy0) * WX + (ix - wx0);
                        R v[8];
                        in_cell_weights(ox, oy, ox1, oy1, qw, vz, m.dx_dt, m.dy_dt, v);
                        if (key != acc_key) {
                            acc_flush();
                            acc_key = key;
#pragma unroll
                            for (int q8 = 0; q8 < 8; ++q8) acc[q8] = v[q8];
                        } else {
#pragma unroll
                            for (int q8 = 0; q8 < 8; ++q8) acc[q8] += v[q8];
                        }
                    } else if (fast) {
                        deposit_esirkepov(sm, ix - wx0, iy - wy0, ox, oy, ix1 - wx0, iy1 - wy0, ox1, oy1, qw,
                                          vz, m.dx_dt, m.dy_dt);
                    } else {
                        deposit_esirkepov(gm, ix, iy, ox, oy, ix1, iy1, ox1, oy1, qw, vz, m.dx_dt, m.dy_dt);
                    }
                    const bool alive = finish_move(m, ix1, iy1);
                    const R chk = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + spn[0] * spn[0] +
                                  spn[1] * spn[1] + spn[2] * spn[2];
                    bad |= !isfinite(chk);
                    if (diag && alive) {
                        dhas = true;
                        dw = w;
#pragma unroll
                        for (int d3 = 0; d3 < 3; ++d3) du[d3] = u[d3], ds[d3] = spn[d3];
                    }
                    S.cell[slot] = alive ? pack_cell(ix1, iy1) : PIC_DEAD;
                    S.ox[slot] = ox1;
                    S.oy[slot] = oy1;
                    S.ux[slot] = u[0];
                    S.uy[slot] = u[1];
                    S.uz[slot] = u[2];
                    S.sx[slot] = spn[0];
                    S.sy[slot] = spn[1];
                    S.sz[slot] = spn[2];
                }
            }
            if (diag) diag_warp(P.diag, sp, dhas, dw, du, ds, drow);
        }
        cp_async_wait0();
        if (diag) store_diag_sums(P.diag, sp, sdiag, kFusedThreads / 32, tile, ntiles);
    }
    acc_flush();
    if (bad) atomicOr(P.err, PIC_EF_NAN);
    __syncthreads();

    // flush the current window: groups of 4 values, skipping all-zero ones and
    // rows / columns outside the mesh (nothing is deposited there)
    constexpr int WQ = WX / 4;
    for (int qd = tid; qd < 3 * WY * WQ; qd += kFusedThreads) {
        const int c = qd / (WY * WQ);
        const int rr = qd - c * WY * WQ;
        const int y = rr / WQ, xq = rr - y * WQ;
        const int gy = wy0 + y, gx = wx0 + 4 * xq;
        if (gy < 0 || gy >= m.ny || gx < 0 || gx >= m.ld) continue;
        flush_add<R>(&m.J[c * m.plane + (size_t)gy * m.ld + gx], &sJ[c * WA + y * WX + 4 * xq]);
    }
    return true;
}

template <int TX, int TY, typename R, bool DIAG>
__global__ void __launch_bounds__(kFusedThreads, TileConst<TX, TY, R>::minb_nodiag)
    k_step_fused(const __grid_constant__ StepParams<R> P, const __grid_constant__ CUtensorMap tmapEB) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double sdiag[kFusedThreads / 32][8];
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    // (fused_tile's barrier after clearing the current window orders the
    // initialisation before every other thread's first wait)
    fused_tile<TX, TY, R, DIAG>(P, &tmapEB, blockIdx.x, gridDim.x, bar, 0u, dsm, sdiag);
}

// ---------------------------------------------------------------------------
// Batched step: persistent CTAs (a few per SM) take (run, tile) work items
// from a queue shared by all runs of a batch and run fused_tile on each, with
// the run's parameters and tensor map read from global memory.  Items of runs
// that have finished their steps are skipped.  Batch steps take no in-step
// Eq. (4) sums, so the tile body is the instantiation without them.
// ---------------------------------------------------------------------------
template <int TX, int TY, typename R>
__global__ void __launch_bounds__(kFusedThreads, TileConst<TX, TY, R>::minb_nodiag)
    k_step_fused_batch(const BatchFused<R> W) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double sdiag[kFusedThreads / 32][8];
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    unsigned phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(W.counter, 1);
        __syncthreads();
        const int w = s_item;
        __syncthreads();
        if (w >= W.nwork) break;
        const int2 rt = W.work[w];
        if (W.step[rt.x] >= W.nsteps[rt.x]) continue;
        const CUtensorMap *tm = W.tmaps + rt.x;
        if (threadIdx.x == 0) fence_tensormap_acquire(tm);
        if (!fused_tile<TX, TY, R, false>(W.params[rt.x], tm, rt.y, W.params[rt.x].t.ntx * W.params[rt.x].t.nty,
                                          bar, phase, dsm, sdiag))
            break;
        phase ^= 1u;
    }
}

// ---------------------------------------------------------------------------
// Split path, a1-a4: one thread per slot, global-memory gather; keeps x^n and
// v_z^{n+1/2} for the deposit.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_push_split(const StepParams<R> P, int s) {
    const DevSpecies<R> &S = P.sp[s];
    const MeshParams<R> &m = P.m;
    const GlobalMesh<R> gm{m.EB, m.J, m.nx, m.ny, m.ld, m.bc_x == 1, m.plane, P.err};
    unsigned bad = 0;
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[p];
        S.cell_old[p] = c;
        if (c == PIC_DEAD) continue;
        const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
        const R ox = S.ox[p], oy = S.oy[p];
        R u[3] = {S.ux[p], S.uy[p], S.uz[p]};
        R sp[3] = {S.sx[p], S.sy[p], S.sz[p]};
        R E[3], B[3];
        gather_eb(gm, ix, iy, ox, oy, E, B);
        push_spin(S.qm, S.a, m.dt, E, B, u, sp);
        const R gi = Real<R>::rsqrt(R(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        int ix1 = ix, iy1 = iy;
        R ox1 = ox, oy1 = oy;
        advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
        advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
        if (!finite3(u) || !finite3(sp)) bad |= PIC_EF_NAN;
        // keep the unwrapped new cell for the deposit; removal happens there
        S.ox_old[p] = ox;
        S.oy_old[p] = oy;
        S.vz[p] = u[2] * gi;
        S.cell[p] = pack_cell(ix1 + 1, iy1 + 1);  // +1 so that -1 is representable
        S.ox[p] = ox1;
        S.oy[p] = oy1;
        S.ux[p] = u[0];
        S.uy[p] = u[1];
        S.uz[p] = u[2];
        S.sx[p] = sp[0];
        S.sy[p] = sp[1];
        S.sz[p] = sp[2];
    }
    if (bad) atomicOr(P.err, bad);
}

// Split path, a5: current of the move recorded by k_push_split, then the
// wrap / removal of the new position.
template <typename R>
__global__ void __launch_bounds__(256) k_deposit_split(const StepParams<R> P, int s) {
    const DevSpecies<R> &S = P.sp[s];
    const MeshParams<R> &m = P.m;
    const GlobalMesh<R> gm{m.EB, m.J, m.nx, m.ny, m.ld, m.bc_x == 1, m.plane, P.err};
    const int n = *S.n;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const uint32_t c0 = S.cell_old[p];
        if (c0 == PIC_DEAD) continue;
        const int ix = (int)(c0 & 0xFFFFu), iy = (int)(c0 >> 16);
        const uint32_t c1 = S.cell[p];
        int ix1 = (int)(c1 & 0xFFFFu) - 1, iy1 = (int)(c1 >> 16) - 1;
        const R ox1 = S.ox[p], oy1 = S.oy[p];
        deposit_esirkepov(gm, ix, iy, S.ox_old[p], S.oy_old[p], ix1, iy1, ox1, oy1, S.q * S.w[p], S.vz[p],
                          m.dx_dt, m.dy_dt);
        const bool alive = finish_move(m, ix1, iy1);
        S.cell[p] = alive ? pack_cell(ix1, iy1) : PIC_DEAD;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int TX, int TY, typename R, bool DIAG>
static cudaError_t launch_fused_d(const StepParams<R> &P, const CUtensorMap &tmapEB, cudaStream_t st) {
    using TC = TileConst<TX, TY, R>;
    constexpr size_t smem = TC::smem_bytes;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fused<TX, TY, R, DIAG>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_step_fused<TX, TY, R, DIAG><<<P.t.ntx * P.t.nty, kFusedThreads, smem, st>>>(P, tmapEB);
    return cudaGetLastError();
}

// steps with in-step Eq. (4) sums run their own instantiation
template <int TX, int TY, typename R>
static cudaError_t launch_fused_t(const StepParams<R> &P, const CUtensorMap &tmapEB, cudaStream_t st) {
    using TC = TileConst<TX, TY, R>;
    if (P.t.WX != TC::WX || P.t.WY != TC::WY || P.t.HX != TC::HX || P.t.HY != TC::HY) return cudaErrorInvalidValue;
    return P.diag.on ? launch_fused_d<TX, TY, R, true>(P, tmapEB, st) : launch_fused_d<TX, TY, R, false>(P, tmapEB, st);
}

template <int TX, int TY, typename R>
static cudaError_t launch_fused_batch_t(const BatchFused<R> &W, int ctas, cudaStream_t st) {
    using TC = TileConst<TX, TY, R>;
    constexpr size_t smem = TC::smem_bytes;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fused_batch<TX, TY, R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_step_fused_batch<TX, TY, R><<<ctas, kFusedThreads, smem, st>>>(W);
    return cudaGetLastError();
}

template <int TX, int TY>
static int batch_occupancy_t() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_fused_batch<TX, TY, float>, kFusedThreads,
                                                      TileConst<TX, TY, float>::smem_bytes) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// resident CTAs per SM of the batched kernel for a tile shape
int fused_batch_occupancy(int tx, int ty) {
    if (tx == 8 && ty == 4) return batch_occupancy_t<8, 4>();
    if (tx == 16 && ty == 8) return batch_occupancy_t<16, 8>();
    if (tx == 32 && ty == 8) return batch_occupancy_t<32, 8>();
    if (tx == 32 && ty == 16) return batch_occupancy_t<32, 16>();
    if (tx == 64 && ty == 16) return batch_occupancy_t<64, 16>();
    return 1;
}

template <typename R>
cudaError_t launch_step_fused_batch(const BatchFused<R> &W, int tx, int ty, int ctas, cudaStream_t st) {
    if (tx == 8 && ty == 4) return launch_fused_batch_t<8, 4, R>(W, ctas, st);
    if (tx == 16 && ty == 8) return launch_fused_batch_t<16, 8, R>(W, ctas, st);
    if (tx == 32 && ty == 8) return launch_fused_batch_t<32, 8, R>(W, ctas, st);
    if (tx == 32 && ty == 16) return launch_fused_batch_t<32, 16, R>(W, ctas, st);
    if (tx == 64 && ty == 16) return launch_fused_batch_t<64, 16, R>(W, ctas, st);
    return cudaErrorInvalidValue;
}
template cudaError_t launch_step_fused_batch<float>(const BatchFused<float> &, int, int, int, cudaStream_t);

bool fused_tile_supported(int tx, int ty) {
    return (tx == 8 && ty == 4) || (tx == 16 && ty == 8) || (tx == 32 && ty == 8) ||
           (tx == 32 && ty == 16) || (tx == 64 && ty == 16);
}

template <typename R>
cudaError_t launch_step_fused(const StepParams<R> &P, const CUtensorMap &tmapEB, cudaStream_t st) {
    const int tx = P.t.TX, ty = P.t.TY;
    if (tx == 8 && ty == 4) return launch_fused_t<8, 4, R>(P, tmapEB, st);
    if (tx == 16 && ty == 8) return launch_fused_t<16, 8, R>(P, tmapEB, st);
    if (tx == 32 && ty == 8) return launch_fused_t<32, 8, R>(P, tmapEB, st);
    if (tx == 32 && ty == 16) return launch_fused_t<32, 16, R>(P, tmapEB, st);
    if (tx == 64 && ty == 16) return launch_fused_t<64, 16, R>(P, tmapEB, st);
    return cudaErrorInvalidValue;
}

static int blocks_for(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b);
}

template <typename R>
cudaError_t launch_push_split(const StepParams<R> &P, int s, int n_upper, cudaStream_t st) {
    k_push_split<R><<<blocks_for(n_upper), 256, 0, st>>>(P, s);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_deposit_split(const StepParams<R> &P, int s, int n_upper, cudaStream_t st) {
    k_deposit_split<R><<<blocks_for(n_upper), 256, 0, st>>>(P, s);
    return cudaGetLastError();
}

template cudaError_t launch_step_fused<float>(const StepParams<float> &, const CUtensorMap &, cudaStream_t);
template cudaError_t launch_step_fused<double>(const StepParams<double> &, const CUtensorMap &, cudaStream_t);
template cudaError_t launch_push_split<float>(const StepParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_push_split<double>(const StepParams<double> &, int, int, cudaStream_t);
template cudaError_t launch_deposit_split<float>(const StepParams<float> &, int, int, cudaStream_t);
template cudaError_t launch_deposit_split<double>(const StepParams<double> &, int, int, cudaStream_t);
