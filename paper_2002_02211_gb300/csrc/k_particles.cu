// k_particles.cu -- particle kernels: the fused a1-a5 step kernel (one CTA
// per tile, TMA-staged field window, shared-memory current window) and the
// split a1-a4 / a5 kernels behind pic_gather_push_spin / pic_deposit.
#include <cuda.h>

#include "pic_device.cuh"
#include "pic_kernels.h"

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
    return ok != 0;
}

// bounded wait: about a second at most, then report and give up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase) {
    for (unsigned it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        __nanosleep(64);
    }
    return false;
}

// a4 and the boundary rule shared by both paths; returns false if removed
__device__ __forceinline__ bool finish_move(const MeshParams &m, int &ix1, int &iy1) {
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
// Fused step kernel.  CTA = one tile.  Thread 0 stages the 6-component field
// window [tile - 4, tile + 4) x [tile - 4, tile + 4) with one 3D TMA load
// (zero fill outside the mesh); the CTA then runs a1-a5 for every particle
// of the tile's slot range, gathering from and depositing into shared
// memory when the particle's 4x4 stencil lies inside the window and the mesh
// (no wrap), otherwise through global memory; finally the current window is
// added to J with 16-byte vector atomics.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_step_fused(const StepParams P,
                                                    const __grid_constant__ CUtensorMap tmapEB) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar;
    const MeshParams &m = P.m;
    const TileGeom &T = P.t;
    const int WX = T.WX, WY = T.WY, WA = WX * WY;
    float *sF = reinterpret_cast<float *>(dsm);
    float *sJ = sF + 6 * WA;

    const int tile = blockIdx.x;
    const int ty = tile / T.ntx, tx = tile - ty * T.ntx;
    const int wx0 = tx * T.TX - PIC_HALO, wy0 = ty * T.TY - PIC_HALO;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_expect_tx(&bar, (unsigned)(6 * WA * sizeof(float)));
        tma_load_3d(sF, &tmapEB, &bar, wx0, wy0, 0);
    }
    for (int i = threadIdx.x; i < 3 * WA; i += blockDim.x) sJ[i] = 0.f;
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0)) {
        if (threadIdx.x == 0) atomicOr(P.err, PIC_EF_TIMEOUT);
        return;
    }

    const SmemMesh sm{sF, sJ, WX, WY};
    const GlobalMesh gm{m.EB, m.J, m.nx, m.ny, m.ld, m.bc_x == 1, m.plane, P.err};
    // window interior where a whole stencil [i-1, i+2] fits, intersected with the mesh
    const int xlo = max(wx0 + 1, 1), xhi = min(wx0 + WX - 3, m.nx - 3);
    const int ylo = max(wy0 + 1, 1), yhi = min(wy0 + WY - 3, m.ny - 3);
    unsigned bad = 0;

    for (int s = 0; s < P.nsp; ++s) {
        const DevSpecies &S = P.sp[s];
        if (!S.mobile) continue;
        const int p0 = S.tile_start[tile], p1 = S.tile_start[tile + 1];
        const float qm = S.qm, a = S.a, q = S.q;
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const uint32_t c = S.cell[p];
            if (c == PIC_DEAD) continue;
            const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
            const float ox = S.ox[p], oy = S.oy[p], w = S.w[p];
            float u[3] = {S.ux[p], S.uy[p], S.uz[p]};
            float sp[3] = {S.sx[p], S.sy[p], S.sz[p]};
            const bool fast = ix >= xlo && ix <= xhi && iy >= ylo && iy <= yhi;
            float E[3], B[3];
            if (fast)
                gather_eb(sm, ix - wx0, iy - wy0, ox, oy, E, B);
            else
                gather_eb(gm, ix, iy, ox, oy, E, B);
            push_spin(qm, a, m.dt, E, B, u, sp);
            const float gi = rsqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            int ix1 = ix, iy1 = iy;
            float ox1 = ox, oy1 = oy;
            advance_axis(ix1, ox1, u[0] * gi * m.dt_dx);
            advance_axis(iy1, oy1, u[1] * gi * m.dt_dy);
            const float qw = q * w, vz = u[2] * gi;
            if (fast)
                deposit_esirkepov(sm, ix - wx0, iy - wy0, ox, oy, ix1 - wx0, iy1 - wy0, ox1, oy1,
                                  qw, vz, m.dx_dt, m.dy_dt);
            else
                deposit_esirkepov(gm, ix, iy, ox, oy, ix1, iy1, ox1, oy1, qw, vz, m.dx_dt, m.dy_dt);
            const bool alive = finish_move(m, ix1, iy1);
            if (!finite3(u) || !finite3(sp)) bad |= PIC_EF_NAN;
            S.cell[p] = alive ? pack_cell(ix1, iy1) : PIC_DEAD;
            S.ox[p] = ox1;
            S.oy[p] = oy1;
            S.ux[p] = u[0];
            S.uy[p] = u[1];
            S.uz[p] = u[2];
            S.sx[p] = sp[0];
            S.sy[p] = sp[1];
            S.sz[p] = sp[2];
        }
    }
    if (bad) atomicOr(P.err, bad);
    __syncthreads();

    // flush the current window: 16-byte quads, skipping all-zero ones and
    // rows / columns outside the mesh (nothing is deposited there)
    const int WQ = WX >> 2;
    for (int qd = threadIdx.x; qd < 3 * WY * WQ; qd += blockDim.x) {
        const int c = qd / (WY * WQ);
        const int r = qd - c * WY * WQ;
        const int y = r / WQ, xq = r - y * WQ;
        const int gy = wy0 + y, gx = wx0 + 4 * xq;
        if (gy < 0 || gy >= m.ny || gx < 0 || gx >= m.ld) continue;
        const float4 v = *reinterpret_cast<const float4 *>(&sJ[(c * WY + y) * WX + 4 * xq]);
        if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
        atomicAdd(reinterpret_cast<float4 *>(&m.J[c * m.plane + (size_t)gy * m.ld + gx]), v);
    }
}

// ---------------------------------------------------------------------------
// Split path, a1-a4: one thread per slot, global-memory gather; keeps x^n and
// v_z^{n+1/2} for the deposit.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_push_split(const StepParams P, int s) {
    const DevSpecies &S = P.sp[s];
    const MeshParams &m = P.m;
    const GlobalMesh gm{m.EB, m.J, m.nx, m.ny, m.ld, m.bc_x == 1, m.plane, P.err};
    unsigned bad = 0;
    const int n = *S.n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t c = S.cell[p];
        S.cell_old[p] = c;
        if (c == PIC_DEAD) continue;
        const int ix = (int)(c & 0xFFFFu), iy = (int)(c >> 16);
        const float ox = S.ox[p], oy = S.oy[p];
        float u[3] = {S.ux[p], S.uy[p], S.uz[p]};
        float sp[3] = {S.sx[p], S.sy[p], S.sz[p]};
        float E[3], B[3];
        gather_eb(gm, ix, iy, ox, oy, E, B);
        push_spin(S.qm, S.a, m.dt, E, B, u, sp);
        const float gi = rsqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        int ix1 = ix, iy1 = iy;
        float ox1 = ox, oy1 = oy;
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
__global__ void __launch_bounds__(256) k_deposit_split(const StepParams P, int s) {
    const DevSpecies &S = P.sp[s];
    const MeshParams &m = P.m;
    const GlobalMesh gm{m.EB, m.J, m.nx, m.ny, m.ld, m.bc_x == 1, m.plane, P.err};
    const int n = *S.n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t c0 = S.cell_old[p];
        if (c0 == PIC_DEAD) continue;
        const int ix = (int)(c0 & 0xFFFFu), iy = (int)(c0 >> 16);
        const uint32_t c1 = S.cell[p];
        int ix1 = (int)(c1 & 0xFFFFu) - 1, iy1 = (int)(c1 >> 16) - 1;
        const float ox1 = S.ox[p], oy1 = S.oy[p];
        deposit_esirkepov(gm, ix, iy, S.ox_old[p], S.oy_old[p], ix1, iy1, ox1, oy1,
                          S.q * S.w[p], S.vz[p], m.dx_dt, m.dy_dt);
        const bool alive = finish_move(m, ix1, iy1);
        S.cell[p] = alive ? pack_cell(ix1, iy1) : PIC_DEAD;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t step_fused_smem_bytes(const TileGeom &t) {
    return (size_t)9 * t.WX * t.WY * sizeof(float);
}

cudaError_t launch_step_fused(const StepParams &P, const CUtensorMap &tmapEB, cudaStream_t st) {
    const size_t smem = step_fused_smem_bytes(P.t);
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    const int ntiles = P.t.ntx * P.t.nty;
    k_step_fused<<<ntiles, 256, smem, st>>>(P, tmapEB);
    return cudaGetLastError();
}

static int blocks_for(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b);
}

cudaError_t launch_push_split(const StepParams &P, int s, int n_upper, cudaStream_t st) {
    const int blocks = blocks_for(n_upper);
    k_push_split<<<blocks, 256, 0, st>>>(P, s);
    return cudaGetLastError();
}

cudaError_t launch_deposit_split(const StepParams &P, int s, int n_upper, cudaStream_t st) {
    const int blocks = blocks_for(n_upper);
    k_deposit_split<<<blocks, 256, 0, st>>>(P, s);
    return cudaGetLastError();
}
