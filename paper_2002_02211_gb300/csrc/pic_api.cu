// pic_api.cu -- the C ABI declared in include/pic.h: context, state transfer,
// and the host-side sequencing of the kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "pic.h"
#include "pic_kernels.h"

namespace {

constexpr double kTwoPi = 6.283185307179586;
constexpr double kMec2Mev = 0.51099895;

struct SpeciesBuf {
    uint32_t *cell = nullptr;
    void *f[9] = {};  // ox oy ux uy uz sx sy sz w (float or double)
    void *oz = nullptr;  // 3D3V only
    int32_t *id = nullptr;
};

// One window move's plasma on the device (pic_stage_injection): per species
// the packed cells, the reals of a record (SortArrays order), the ids, and the
// count, on the host and on the device (where the kernels read it).
struct Slab {
    void *mem = nullptr;
    int64_t n[PIC_MAX_SPECIES] = {};
    uint32_t *cell[PIC_MAX_SPECIES] = {};
    void *f[PIC_MAX_SPECIES][10] = {};
    int32_t *id[PIC_MAX_SPECIES] = {};
    int32_t *n_dev[PIC_MAX_SPECIES] = {};
};

struct Ctx {
    pic_config_t cfg{};
    int device = 0;
    int dim = 2;
    double dt = 0, dx = 0, dy = 0, dz = 0;
    int ld = 0;
    size_t plane = 0;  // elements of one mesh component: ny * ld (2D3V), nz * ny * ld (3D3V)
    size_t bnd_n = 0;  // left boundary values per component: ny (2D3V), nz * ny (3D3V)
    TileGeom tg{};
    TileGeom3 tg3{};
    int ntiles = 0;
    int rb = 4;  // bytes per real: 4 for the FP32 path, 8 for the FP64 instantiation
    void *EB = nullptr, *J = nullptr, *bnd = nullptr, *rho = nullptr, *rho_bg = nullptr;
    void *stage = nullptr;  // max(plane, capacity) doubles: precision conversions of transfers
    size_t stage_elems = 0;
    SpeciesBuf buf[PIC_MAX_SPECIES][2];
    int cur[PIC_MAX_SPECIES] = {};
    int n_upper[PIC_MAX_SPECIES] = {};  // host bound on the device slot counts (sizes grids)
    int32_t *tile_start[PIC_MAX_SPECIES] = {};
    uint32_t *cell_old[PIC_MAX_SPECIES] = {};
    void *old_f[PIC_MAX_SPECIES][3] = {};  // ox_old, oy_old, then vz (2D3V) or oz_old (3D3V)
    int32_t *tile_count = nullptr, *tile_cursor = nullptr;
    int32_t *cell_count = nullptr, *cell_off = nullptr, *tile_info = nullptr;
    int32_t *n_dev = nullptr;  // [PIC_MAX_SPECIES + 1] slot counts; the last entry is sort scratch
    int32_t *scratch_i32 = nullptr;  // 3 * max capacity, for ix / iy / iz transfers
    unsigned *err = nullptr;
    double *partials = nullptr, *result = nullptr;
    double *laser_prof = nullptr;  // [2][bnd_n] transverse profile at the Ez and Ey source points
    double *hist = nullptr;        // [PIC_MAX_HIST_BINS][5] energy spectrum
    // in-step Eq. (4) diagnostics
    int diag_every = 0;
    double diag_lo[PIC_MAX_SPECIES] = {}, diag_hi[PIC_MAX_SPECIES] = {};
    double *diag_rows = nullptr, *diag_shift = nullptr;
    pic_moments_dev *diag_out = nullptr;
    long long diag_step = -1;
    CUtensorMap tmapEB;
    bool pending_deposit = false;
    long long step = 0;
    long long window = 0;         // cells the co-moving window has moved
    // co-moving window on the stepping path (pic_set_window): cells a move
    // (0: off), the step index the light front starts from, its speed [c],
    // and the cells moved when the window was set
    int w_ncells = 0;
    long long w_start = 0;
    double w_speed = 1.0;
    long long w_window0 = 0;
    // staged plasma of the next moves, oldest first; memory of consumed
    // slabs is freed at the next synchronous window call (kernels may still
    // read it)
    std::deque<Slab> inj_queue;
    std::vector<void *> inj_spent;
    // binned layout: tile-column relabelling of each species' ranges since
    // its last sort (bin_rot_x)
    int bin_txo[PIC_MAX_SPECIES] = {};
    // live-particle counts the sorts leave in host-mapped memory: once a
    // sort's event has completed, n_live becomes its count plus the particles
    // injected since (a tighter bound than counting every injection)
    volatile long long *live_host = nullptr;
    long long *live_dev = nullptr;
    cudaEvent_t live_ev[PIC_MAX_SPECIES] = {};
    bool live_pending[PIC_MAX_SPECIES] = {};
    int64_t live_added[PIC_MAX_SPECIES] = {};
    // adjoint results: per species the lambdas of the initial state
    // (lx ly lux luy luz lsx lsy lsz lw), the initial cells, and the slot counts
    void *adj_lam[PIC_MAX_SPECIES][9] = {};
    uint32_t *adj_cell0[PIC_MAX_SPECIES] = {};
    long long adj_n[PIC_MAX_SPECIES] = {};
    bool has_background = false;  // pic_capture_background was called
    // binned 3D3V layout (bin_headroom_pct > 0): per mobile species the range
    // counters of both buffers (front, split, back, arrival base per range, Bin3), whether
    // the species is in that layout now, and a host bound on its live
    // particles (sizes the ranges against capacity)
    bool binned = false;
    bool sp_binned[PIC_MAX_SPECIES] = {};
    // the binned step leaves the slots outside the new segments unsealed
    // (stale records); seal_pending writes PIC_DEAD there before any kernel
    // that reads every slot
    bool unsealed[PIC_MAX_SPECIES] = {};
    // host-mapped flag the binned step raises when an overflow range is past
    // half full; the next pic_push_deposit that sees it re-bins first.  It
    // is read without synchronising, so it takes effect at the first step the
    // host issues after the GPU raised it; a range that still fills before
    // that drops particles and reports PIC_ERR_OVERFLOW.
    volatile int *ovf_alert = nullptr;
    int *ovf_alert_dev = nullptr;
    // binned steps in flight are bounded: before a binned step the host waits
    // for the one kAhead steps back, so the alert it reads is at most kAhead
    // steps old however far ahead the caller queues
    static constexpr int kAhead = 4;
    cudaEvent_t ahead_ev[kAhead] = {};
    long long ahead_k = 0;
    int32_t *bin_cnt[PIC_MAX_SPECIES][2] = {};
    int32_t *old_start = nullptr;  // [ntiles + 2]: a sort's source ranges
    // the current buffer is the compact layout of the species' last sort, its
    // slots unchanged since (the next sort can gather tile by tile)
    bool tile_ordered[PIC_MAX_SPECIES] = {};
    int64_t n_live[PIC_MAX_SPECIES] = {};
    // CTAs of the overflow-range kernel: one per 256 slots of the largest
    // overflow range, between kBinCtasMin and kBinCtasMax
    static constexpr int kBinCtasMin = 8, kBinCtasMax = 152 * 4;
    int bin_ctas = kBinCtasMin;
    int since_sort = 0;
    long long launches = 0;  // kernels launched by this context
    // pic_step replays sort-free stretches of steps from CUDA graphs (compact
    // layout): one graph per (length, diagnostic phase, buffer parity,
    // parameter generation), captured on the context's own stream at first use
    struct StepGraph {
        int len;               // steps in the stretch
        int phase;             // step index mod diag_every at its start (-1: diagnostics off)
        unsigned parity;       // bit s: the buffer species s is in
        long long gen;         // graph_gen at capture
        cudaGraphExec_t exec;
        long long launches;    // kernels one replay runs
        int last_diag;         // offset of the stretch's last diagnostic step (-1: none)
    };
    static constexpr int kMaxGraphs = 16;
    std::vector<StepGraph> graphs;
    int graph_max = 32;          // longest stretch replayed as one graph (0: launch every kernel)
    long long graph_gen = 0;     // bumped whenever a captured kernel parameter would change
    long long graph_captures = 0, graph_replays = 0;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {};
    double *laser_tab = nullptr;  // device [2 * graph_max]: (fz, fy) of each step of a replayed stretch
    const double *lf_capture = nullptr;  // while capturing: this step's slot of laser_tab
    // device arrays the caller owns (pic_bind_buffers): never freed here
    std::vector<void *> borrowed;
    std::string last_error;
};

// cudaFree unless the caller owns the array
void free_own(Ctx *c, void *p) {
    if (!p) return;
    for (void *b : c->borrowed)
        if (b == p) return;
    cudaFree(p);
}

void drop_step_graphs(Ctx *c) {
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    c->graph_gen += 1;
}

std::string g_create_error;

pic_status_t fail(Ctx *c, pic_status_t s, const std::string &msg) {
    if (c)
        c->last_error = msg;
    else
        g_create_error = msg;
    return s;
}

#define CK(...)                                                                                 \
    do {                                                                                        \
        cudaError_t e_ = (__VA_ARGS__);                                                         \
        if (e_ != cudaSuccess)                                                                  \
            return fail(c, PIC_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

int round_up(int v, int m) { return (v + m - 1) / m * m; }

template <typename R>
DevSpecies<R> dev_species(Ctx *c, int s, int which) {
    DevSpecies<R> d{};
    const SpeciesBuf &b = c->buf[s][which];
    d.cell = b.cell;
    d.ox = static_cast<R *>(b.f[0]);
    d.oy = static_cast<R *>(b.f[1]);
    d.ux = static_cast<R *>(b.f[2]);
    d.uy = static_cast<R *>(b.f[3]);
    d.uz = static_cast<R *>(b.f[4]);
    d.sx = static_cast<R *>(b.f[5]);
    d.sy = static_cast<R *>(b.f[6]);
    d.sz = static_cast<R *>(b.f[7]);
    d.w = static_cast<R *>(b.f[8]);
    d.id = b.id;
    d.tile_start = c->tile_start[s];
    d.cell_old = c->cell_old[s];
    d.ox_old = static_cast<R *>(c->old_f[s][0]);
    d.oy_old = static_cast<R *>(c->old_f[s][1]);
    d.vz = static_cast<R *>(c->old_f[s][2]);
    const pic_species_t &sp = c->cfg.sp[s];
    d.qm = (R)(sp.q / sp.m);
    d.q = (R)sp.q;
    d.a = (R)sp.a;
    d.mobile = sp.mobile;
    d.n = c->n_dev + s;
    return d;
}

template <typename R>
MeshParams<R> mesh(Ctx *c) {
    MeshParams<R> m{};
    m.nx = c->cfg.nx;
    m.ny = c->cfg.ny;
    m.ld = c->ld;
    m.bc_x = c->cfg.bc_x;
    m.dt = (R)c->dt;
    m.dt_dx = (R)(c->dt / c->dx);
    m.dt_dy = (R)(c->dt / c->dy);
    m.dx_dt = (R)(c->dx / c->dt);
    m.dy_dt = (R)(c->dy / c->dt);
    m.EB = static_cast<R *>(c->EB);
    m.J = static_cast<R *>(c->J);
    m.plane = c->plane;
    return m;
}

template <typename R>
StepParams<R> step_params(Ctx *c) {
    StepParams<R> P{};
    P.m = mesh<R>(c);
    P.t = c->tg;
    P.nsp = c->cfg.nspecies;
    for (int s = 0; s < P.nsp; ++s) P.sp[s] = dev_species<R>(c, s, c->cur[s]);
    P.err = c->err;
    return P;
}

template <typename R>
DevSpecies3<R> dev_species3(Ctx *c, int s, int which) {
    const DevSpecies<R> d = dev_species<R>(c, s, which);
    DevSpecies3<R> e{};
    e.cell = d.cell;
    e.ox = d.ox;
    e.oy = d.oy;
    e.oz = static_cast<R *>(c->buf[s][which].oz);
    e.ux = d.ux;
    e.uy = d.uy;
    e.uz = d.uz;
    e.sx = d.sx;
    e.sy = d.sy;
    e.sz = d.sz;
    e.w = d.w;
    e.id = d.id;
    e.tile_start = d.tile_start;
    e.cell_old = d.cell_old;
    e.ox_old = d.ox_old;
    e.oy_old = d.oy_old;
    e.oz_old = static_cast<R *>(c->old_f[s][2]);
    e.qm = d.qm;
    e.q = d.q;
    e.a = d.a;
    e.mobile = d.mobile;
    e.n = d.n;
    return e;
}

template <typename R>
MeshParams3<R> mesh3(Ctx *c) {
    MeshParams3<R> m{};
    m.nx = c->cfg.nx;
    m.ny = c->cfg.ny;
    m.nz = c->cfg.nz;
    m.ld = c->ld;
    m.bc_x = c->cfg.bc_x;
    m.dt = (R)c->dt;
    m.dt_dx = (R)(c->dt / c->dx);
    m.dt_dy = (R)(c->dt / c->dy);
    m.dt_dz = (R)(c->dt / c->dz);
    m.dx_dt = (R)(c->dx / c->dt);
    m.dy_dt = (R)(c->dy / c->dt);
    m.dz_dt = (R)(c->dz / c->dt);
    m.EB = static_cast<R *>(c->EB);
    m.J = static_cast<R *>(c->J);
    m.plane = c->plane;
    return m;
}

template <typename R>
StepParams3<R> step_params3(Ctx *c) {
    StepParams3<R> P{};
    P.m = mesh3<R>(c);
    P.t = c->tg3;
    P.nsp = c->cfg.nspecies;
    for (int s = 0; s < P.nsp; ++s) P.sp[s] = dev_species3<R>(c, s, c->cur[s]);
    P.err = c->err;
    P.diag_cols0 = c->ntiles;
    return P;
}

// runs f(R{}) with R the context's real type
template <class F>
auto with_real(Ctx *c, F &&f) {
    return c->rb == 8 ? f(double{}) : f(float{});
}

LaserParams laser(Ctx *c) {
    LaserParams L{};
    L.pol = c->cfg.bc_x == PIC_BC_OPEN ? c->cfg.pol : PIC_POL_NONE;
    L.a0 = c->cfg.a0;
    L.w0 = c->cfg.waist_lambda * kTwoPi;
    L.tau = c->cfg.fwhm_periods * kTwoPi / std::sqrt(2.0 * std::log(2.0));
    L.t_peak = c->cfg.t_peak_periods * kTwoPi;
    L.yc = 0.5 * c->cfg.ny * c->dy;
    L.dy = c->dy;
    return L;
}

void choose_tiles3(Ctx *c) {
    int tx = c->cfg.tile_x, ty = c->cfg.tile_y, tz = c->cfg.tile_z;
    if (tx <= 0 || ty <= 0 || tz <= 0) {
        tx = 16;
        ty = 4;
        tz = 4;
    }
    TileGeom3 &t = c->tg3;
    t.TX = tx;
    t.TY = ty;
    t.TZ = tz;
    t.WX = c->rb == 8 ? window3_wx<double>(tx) : window3_wx<float>(tx);
    t.FX = c->rb == 8 ? window3_fx<double>(tx) : window3_fx<float>(tx);
    t.WY = window3_w(ty);
    t.WZ = window3_w(tz);
    t.HX = window3_hx();
    t.HY = window3_h();
    t.HZ = window3_h();
    t.ntx = (c->cfg.nx + tx - 1) / tx;
    t.nty = (c->cfg.ny + ty - 1) / ty;
    t.ntz = (c->cfg.nz + tz - 1) / tz;
    c->ntiles = t.ntx * t.nty * t.ntz;
}

int tile_cells(const Ctx *c) { return c->dim == 3 ? c->tg3.TX * c->tg3.TY * c->tg3.TZ : c->tg.TX * c->tg.TY; }

void choose_tiles(Ctx *c) {
    if (c->dim == 3) {
        choose_tiles3(c);
        return;
    }
    int tx = c->cfg.tile_x, ty = c->cfg.tile_y;
    if (tx <= 0 || ty <= 0) {
        // large meshes: 32 x 8; small ones: 16 x 8, and below 4 CTAs of 16 x 8
        // per SM, 8 x 4 (the L2-resident 256 x 128 run: 42.8 against 56.2 us
        // a step replayed from graphs)
        const long long cells = (long long)c->cfg.nx * c->cfg.ny;
        tx = cells >= (1LL << 19) ? 32 : (cells >= 152LL * 4 * 16 * 8 ? 16 : 8);
        ty = tx == 8 ? 4 : 8;
    }
    // tile shapes the fused kernel is compiled for (pic_validate_config checks)
    c->tg.TX = tx;
    c->tg.TY = ty;
    c->tg.WX = c->rb == 8 ? window_wx<double>(tx) : window_wx<float>(tx);
    c->tg.WY = window_wy(ty);
    c->tg.HX = c->rb == 8 ? window_hx<double>(tx) : window_hx<float>(tx);
    c->tg.HY = window_hy();
    c->tg.ntx = (c->cfg.nx + tx - 1) / tx;
    c->tg.nty = (c->cfg.ny + ty - 1) / ty;
    c->ntiles = c->tg.ntx * c->tg.nty;
}

pic_status_t make_tensor_map(Ctx *c) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess)
        return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const CUtensorMapDataType dtype = c->rb == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r;
    if (c->dim == 3) {
        // [6][nz][ny][ld] as a 4D tensor (x, y, z, component); box = the tile window
        const cuuint64_t dims[4] = {(cuuint64_t)c->cfg.nx, (cuuint64_t)c->cfg.ny, (cuuint64_t)c->cfg.nz, 6};
        const cuuint64_t strides[3] = {(cuuint64_t)c->ld * c->rb, (cuuint64_t)c->ld * c->cfg.ny * c->rb,
                                       (cuuint64_t)c->plane * c->rb};
        const cuuint32_t box[4] = {(cuuint32_t)c->tg3.FX, (cuuint32_t)c->tg3.WY, (cuuint32_t)c->tg3.WZ, 6};
        r = enc(&c->tmapEB, dtype, 4, c->EB, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)c->cfg.nx, (cuuint64_t)c->cfg.ny, 6};
        const cuuint64_t strides[2] = {(cuuint64_t)c->ld * c->rb, (cuuint64_t)c->plane * c->rb};
        const cuuint32_t box[3] = {(cuuint32_t)c->tg.WX, (cuuint32_t)c->tg.WY, 6};
        r = enc(&c->tmapEB, dtype, 3, c->EB, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return PIC_OK;
}

pic_status_t check_flags(Ctx *c, cudaStream_t st) {
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h == 0) return PIC_OK;
    CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st));
    CK(cudaStreamSynchronize(st));
    if (h & PIC_EF_TIMEOUT) return fail(c, PIC_ERR_TIMEOUT, "tile staging wait timed out");
    if (h & PIC_EF_NAN) return fail(c, PIC_ERR_NAN, "non-finite momentum or spin");
    if (h & PIC_EF_CFL) return fail(c, PIC_ERR_CFL, "particle moved a cell or more in one step");
    if (h & PIC_EF_RANGE) return fail(c, PIC_ERR_ARG, "particle cell outside the particle region");
    if (h & PIC_EF_BINS)
        return fail(c, PIC_ERR_OVERFLOW,
                    "binned layout: a tile range and the overflow range were full, particles were lost "
                    "(raise bin_headroom_pct or bin_min_extra, or sort more often)");
    return fail(c, PIC_ERR_CUDA, "unknown device error flag");
}

// Binned layout of species s: the overflow range and the host bound on the
// slot span (every range at its largest, plus the overflow range); false when
// the species is not eligible or its capacity cannot hold that bound.
bool bin_plan(const Ctx *c, int s, int *ovf_cap, int64_t *span) {
    if (!c->binned || !c->cfg.sp[s].mobile) return false;
    const int64_t n = c->n_live[s];
    const int64_t ovf = ((std::max<int64_t>(1024, n / 4) + 7) / 8) * 8;
    const int64_t bound = n + n * c->cfg.bin_headroom_pct / 100 +
                          (int64_t)c->ntiles * (c->cfg.bin_min_extra + 7) + ovf;
    if (bound > c->cfg.sp[s].capacity) return false;
    *ovf_cap = (int)ovf;
    *span = bound;
    return true;
}

// PIC_DEAD into the stale slots the binned steps left in every species'
// current buffer (before a kernel that reads every slot)
pic_status_t seal_pending(Ctx *c, cudaStream_t st) {
    SealArgs a{};
    a.nranges = c->ntiles + 1;
    a.fill = true;
    a.counters = false;
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        if (!c->unsealed[s]) continue;
        a.sp[a.nsp++] = SealSpecies{c->buf[s][c->cur[s]].cell, c->tile_start[s], c->bin_cnt[s][c->cur[s]], nullptr};
        c->unsealed[s] = false;
    }
    if (a.nsp == 0) return PIC_OK;
    CK(launch_seal_bins(a, st));
    c->launches += 1;
    return PIC_OK;
}

// n_live of species s from the last sort's live count once that sort has
// completed (non-blocking), plus the particles injected since
void refresh_live(Ctx *c, int s) {
    if (!c->live_pending[s]) return;
    const cudaError_t q = cudaEventQuery(c->live_ev[s]);
    if (q == cudaErrorNotReady) {
        cudaGetLastError();  // not an error: clear it
        return;
    }
    if (q != cudaSuccess) return;
    c->n_live[s] = std::min<int64_t>(c->n_live[s], c->live_host[s] + c->live_added[s]);
    c->live_pending[s] = false;
}

void add_live(Ctx *c, int s, int64_t m) {
    c->n_live[s] += m;
    c->live_added[s] += m;
}

// the live count of species s into host-mapped memory (after a sort or a
// window move; no-op until the window is used)
pic_status_t live_sample(Ctx *c, int s, cudaStream_t st) {
    if (!c->live_host) return PIC_OK;
    const bool bin = c->sp_binned[s];
    CK(launch_live_sample(c->n_dev + s, bin ? c->tile_start[s] : nullptr, c->bin_cnt[s][c->cur[s]],
                          c->ntiles + 1, c->live_dev + s, st));
    CK(cudaEventRecord(c->live_ev[s], st));
    c->launches += 1;
    c->live_pending[s] = true;
    c->live_added[s] = 0;
    return PIC_OK;
}

// No host synchronisation: the sorted slot count stays on the device.  In the
// compact layout it only shrinks, so n_upper still bounds it; in the binned
// layout n_upper becomes the host bound on the span of the ranges.
// compact_only keeps the compact layout even when the binned one is on.
pic_status_t sort_species(Ctx *c, int s, cudaStream_t st, bool compact_only = false) {
    pic_status_t sr = seal_pending(c, st);
    if (sr != PIC_OK) return sr;
    refresh_live(c, s);
    const int from = c->cur[s], to = 1 - from;
    SortScratch w{c->cell_count, c->cell_off, c->tile_info, c->tile_count, c->tile_cursor, c->scratch_i32};
    BinSort bins{};
    int64_t span = 0;
    const bool bin = c->dim == 3 && !compact_only && bin_plan(c, s, &bins.ovf_cap, &span);
    if (bin) {
        bins.pct = c->cfg.bin_headroom_pct;
        bins.extra = c->cfg.bin_min_extra;
        bins.cnt_to = c->bin_cnt[s][to];
        bins.cnt_from = c->bin_cnt[s][from];
    }
    // a source in the layout of the last sort (binned and sealed above, or
    // compact with its slots unchanged) is gathered tile by tile
    bins.src_binned = c->sp_binned[s];
    bins.src_ordered = c->sp_binned[s] || c->tile_ordered[s];
    bins.txo = c->bin_txo[s];
    bins.old_start = c->old_start;
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        if (c->dim == 3)
            return launch_tile_sort3<T>(dev_species3<T>(c, s, from), dev_species3<T>(c, s, to), c->tg3, w,
                                        c->tile_start[s], c->n_dev + PIC_MAX_SPECIES, c->n_upper[s], bins, st);
        return launch_tile_sort<T>(dev_species<T>(c, s, from), dev_species<T>(c, s, to), c->tg, w, c->tile_start[s],
                                   c->n_dev + PIC_MAX_SPECIES, c->n_upper[s], bins, st);
    }));
    // rank, layout, three scan passes, scatter (a binned source's tiles and
    // then its overflow range), the seal of a binned result
    c->launches += 6 + (bins.src_binned && c->ntiles >= 4 * 152 ? 1 : 0) + (bin ? 1 : 0);
    c->tile_ordered[s] = !bin;
    c->cur[s] = to;
    c->bin_txo[s] = 0;
    if (bin) {
        c->n_upper[s] = (int)span;
        const int want = (bins.ovf_cap + 255) / 256;
        c->bin_ctas = std::min(Ctx::kBinCtasMax, std::max(c->bin_ctas, want));
    }
    else if (c->sp_binned[s])
        c->n_upper[s] = (int)std::min<int64_t>(c->n_upper[s], c->n_live[s]);
    c->sp_binned[s] = bin;
    return live_sample(c, s, st);
}

// every mobile species in the binned layout (the binned step's precondition)
bool all_binned(const Ctx *c) {
    for (int s = 0; s < c->cfg.nspecies; ++s)
        if (c->cfg.sp[s].mobile && !c->sp_binned[s]) return false;
    return true;
}

pic_status_t read_count(Ctx *c, int s, cudaStream_t st, int32_t *n) {
    CK(cudaMemcpyAsync(n, c->n_dev + s, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

// the arrays of species s in buffer `which`, records in SortArrays order
template <typename T>
SortArrays<T> buf_arrays(Ctx *c, int s, int which) {
    const SpeciesBuf &B = c->buf[s][which];
    SortArrays<T> a{};
    a.cell = B.cell;
    a.id = B.id;
    a.n = c->n_dev + s;
    T *const *f = reinterpret_cast<T *const *>(B.f);
    if (c->dim == 3) {
        T *g[10] = {f[0], f[1], static_cast<T *>(B.oz), f[2], f[3], f[4], f[5], f[6], f[7], f[8]};
        for (int k = 0; k < 10; ++k) a.f[k] = g[k];
    } else {
        for (int k = 0; k < 9; ++k) a.f[k] = f[k];
    }
    return a;
}

// device address of a pinned (device-mapped) host array, nullptr for pageable
// memory or when the query fails
const void *mapped_host(const void *p) {
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Host particles p of species s into slots [base, base + p->n) of the current
// buffer (float or double host arrays; converted on the device when the
// context's precision differs), cells packed and range checked; the slot
// count becomes base + p->n.  Synchronous.
template <typename HostT, typename PT>
pic_status_t upload_particles(Ctx *c, int s, const PT *p, int64_t base, cudaStream_t st) {
    const HostT *src[9] = {p->ox, p->oy, p->ux, p->uy, p->uz, p->sx, p->sy, p->sz, p->w};
    const bool d3 = c->dim == 3;
    if (p->n > 0) {
        if (!p->ix || !p->iy || !p->id || (d3 && (!p->iz || !p->oz))) return fail(c, PIC_ERR_ARG, "null particle array");
        for (int k = 0; k < 9; ++k)
            if (!src[k]) return fail(c, PIC_ERR_ARG, "null particle array");
    }
    const size_t n = (size_t)p->n;
    // the uploaded slots are in no tile order: the species is in the compact
    // layout until the sort that follows an upload
    c->sp_binned[s] = false;
    c->tile_ordered[s] = false;
    if (base == 0) {
        c->unsealed[s] = false;  // the upload replaces the layout
        c->live_pending[s] = false;
    } else {
        pic_status_t r = seal_pending(c, st);  // appended after sealed slots
        if (r != PIC_OK) return r;
    }
    const int xlo = c->cfg.bc_x == PIC_BC_OPEN ? 2 : 0;
    const int xhi = c->cfg.bc_x == PIC_BC_OPEN ? c->cfg.nx - 3 : c->cfg.nx - 1;
    // pinned host arrays: one kernel reads them in place over the host link
    // and writes the buffer (cells packed, precision converted on the way)
    UploadSrc<HostT> us{};
    bool direct = n > 0;
    if (direct) {
        us.ix = static_cast<const int32_t *>(mapped_host(p->ix));
        us.iy = static_cast<const int32_t *>(mapped_host(p->iy));
        us.iz = d3 ? static_cast<const int32_t *>(mapped_host(p->iz)) : nullptr;
        us.id = static_cast<const int32_t *>(mapped_host(p->id));
        direct = us.ix && us.iy && us.id && (!d3 || us.iz);
        const HostT *rec3[10] = {p->ox, p->oy, p->oz, p->ux, p->uy, p->uz, p->sx, p->sy, p->sz, p->w};
        for (int k = 0; k < (d3 ? 10 : 9) && direct; ++k) {
            us.f[k] = static_cast<const HostT *>(mapped_host(d3 ? rec3[k] : src[k]));
            direct = us.f[k] != nullptr;
        }
    }
    if (direct) {
        CK(with_real(c, [&](auto z) {
            using T = decltype(z);
            SortArrays<T> d = buf_arrays<T>(c, s, c->cur[s]);
            d.cell += base;
            d.id += base;
            for (int k = 0; k < 10; ++k)
                if (d.f[k]) d.f[k] += base;
            return launch_upload<HostT, T>(us, d, (int)n, xlo, xhi, c->cfg.ny, c->dim == 3 ? c->cfg.nz : 1, d3,
                                           c->err, st);
        }));
        c->launches += 1;
    }
    SpeciesBuf &B = c->buf[s][c->cur[s]];
    const size_t cap = (size_t)c->cfg.sp[s].capacity;
    int32_t *dix = c->scratch_i32, *diy = c->scratch_i32 + cap, *diz = c->scratch_i32 + 2 * cap;
    const size_t rb = c->rb;
    if (n && !direct) {
        CK(cudaMemcpyAsync(dix, p->ix, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(diy, p->iy, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        if (d3) CK(cudaMemcpyAsync(diz, p->iz, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        for (int k = 0; k < (d3 ? 10 : 9); ++k) {
            const HostT *from = k < 9 ? src[k] : p->oz;
            char *to = static_cast<char *>(k < 9 ? B.f[k] : B.oz) + base * rb;
            if (rb == sizeof(HostT)) {
                CK(cudaMemcpyAsync(to, from, n * sizeof(HostT), cudaMemcpyHostToDevice, st));
            } else {  // convert on the device through the staging buffer
                CK(cudaMemcpyAsync(c->stage, from, n * sizeof(HostT), cudaMemcpyHostToDevice, st));
                if (rb == 8)
                    CK(launch_convert<float, double>(static_cast<float *>(c->stage), reinterpret_cast<double *>(to), n, st));
                else
                    CK(launch_convert<double, float>(static_cast<double *>(c->stage), reinterpret_cast<float *>(to), n, st));
                c->launches += 1;
            }
        }
        CK(cudaMemcpyAsync(B.id + base, p->id, n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    if (!direct) {
        if (d3)
            CK(launch_pack_cells3(dix, diy, diz, B.cell + base, (int)n, xlo, xhi, c->cfg.ny, c->cfg.nz, c->err, st));
        else
            CK(launch_pack_cells(dix, diy, B.cell + base, (int)n, xlo, xhi, c->cfg.ny, c->err, st));
        c->launches += n ? 1 : 0;
    }
    const int32_t nn = (int32_t)(base + (int64_t)n);
    CK(cudaMemcpyAsync(c->n_dev + s, &nn, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    c->n_upper[s] = (int)nn;
    pic_status_t r = check_flags(c, st);
    if (r != PIC_OK) {
        const int32_t keep = (int32_t)base;
        cudaMemcpyAsync(c->n_dev + s, &keep, sizeof(int32_t), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
        c->n_upper[s] = (int)base;
        if (base == 0) c->n_live[s] = 0;
        return r;
    }
    if (base == 0)
        c->n_live[s] = (int64_t)n;
    else
        add_live(c, s, (int64_t)n);
    return PIC_OK;
}

// new 2D3V tile shape: the tile-dependent arrays, the window tensor map, and
// every species re-sorted into the new tiles
pic_status_t retile(Ctx *c, int tx, int ty, cudaStream_t st) {
    if (c->dim != 2 || !fused_tile_supported(tx, ty)) return fail(c, PIC_ERR_ARG, "unsupported tile shape");
    CK(cudaStreamSynchronize(st));
    drop_step_graphs(c);  // the tile arrays move
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        cudaFree(c->tile_start[s]);
        c->tile_start[s] = nullptr;
    }
    cudaFree(c->tile_count);
    cudaFree(c->cell_count);
    cudaFree(c->cell_off);
    cudaFree(c->tile_info);
    cudaFree(c->tile_cursor);
    cudaFree(c->diag_rows);
    cudaFree(c->old_start);
    c->old_start = nullptr;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) c->tile_ordered[s] = false;  // the old tiles' order
    c->cfg.tile_x = tx;
    c->cfg.tile_y = ty;
    choose_tiles(c);
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        CK(cudaMalloc(&c->tile_start[s], (c->ntiles + 2) * sizeof(int32_t)));
        CK(cudaMemsetAsync(c->tile_start[s], 0, (c->ntiles + 2) * sizeof(int32_t), st));
    }
    const size_t cells = (size_t)c->ntiles * tile_cells(c);
    CK(cudaMalloc(&c->tile_count, (c->ntiles + 1) * sizeof(int32_t)));
    CK(cudaMalloc(&c->cell_count, cells * sizeof(int32_t)));
    CK(cudaMalloc(&c->cell_off, cells * sizeof(int32_t)));
    CK(cudaMalloc(&c->tile_info, (size_t)c->ntiles * kTileInfo * sizeof(int32_t)));
    CK(cudaMalloc(&c->tile_cursor, c->ntiles * sizeof(int32_t)));
    CK(cudaMalloc(&c->old_start, (c->ntiles + 2) * sizeof(int32_t)));
    CK(cudaMalloc(&c->diag_rows, (size_t)(c->ntiles + Ctx::kBinCtasMax) * PIC_MAX_SPECIES * 8 * sizeof(double)));
    pic_status_t r = make_tensor_map(c);
    if (r != PIC_OK) return r;
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        r = sort_species(c, s, st);
        if (r != PIC_OK) return r;
    }
    c->since_sort = 0;
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status_t alloc_old(Ctx *c, int s) {
    if (c->cell_old[s]) return PIC_OK;
    const size_t cap = (size_t)c->cfg.sp[s].capacity;
    CK(cudaMalloc(&c->cell_old[s], cap * sizeof(uint32_t) + 16));
    for (int k = 0; k < 3; ++k) CK(cudaMalloc(&c->old_f[s][k], cap * c->rb + 16));
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// co-moving window (Sec. 2): staged plasma and the device-side move
// ---------------------------------------------------------------------------

template <typename T>
SortArrays<T> slab_arrays(const Slab &b, int s) {
    SortArrays<T> a{};
    a.cell = b.cell[s];
    a.id = b.id[s];
    a.n = b.n_dev[s];
    for (int k = 0; k < 10; ++k) a.f[k] = static_cast<T *>(b.f[s][k]);
    return a;
}

void ensure_live(Ctx *c) {
    if (c->live_host) return;
    long long *h = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void **>(&h), PIC_MAX_SPECIES * sizeof(long long), cudaHostAllocMapped) !=
        cudaSuccess)
        return;  // without samples n_live only counts up (still a bound)
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) h[s] = 0;
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->live_dev), h, 0) != cudaSuccess) {
        cudaFreeHost(h);
        return;
    }
    for (int s = 0; s < PIC_MAX_SPECIES; ++s)
        if (cudaEventCreateWithFlags(&c->live_ev[s], cudaEventDisableTiming) != cudaSuccess) {
            for (int q = 0; q < s; ++q) cudaEventDestroy(c->live_ev[q]);
            cudaFreeHost(h);
            c->live_dev = nullptr;
            return;
        }
    c->live_host = h;
}

// frees the memory of consumed slabs (kernels that read it are done after
// the stream synchronisation)
pic_status_t free_spent(Ctx *c, cudaStream_t st) {
    if (c->inj_spent.empty()) return PIC_OK;
    CK(cudaStreamSynchronize(st));
    for (void *m : c->inj_spent) cudaFree(m);
    c->inj_spent.clear();
    return PIC_OK;
}

// Host plasma of one move (one set per species, float arrays) into device
// memory: cells packed and checked against the particle region, reals in the
// context's precision.  Synchronous.
pic_status_t stage_slab(Ctx *c, const pic_particles_t *inj, Slab *out, cudaStream_t st) {
    const bool d3 = c->dim == 3;
    const int nf = d3 ? 10 : 9;
    const size_t rb = c->rb;
    auto up16 = [](size_t b) { return (b + 15) / 16 * 16; };
    size_t bytes = 0;
    size_t off_cell[PIC_MAX_SPECIES], off_id[PIC_MAX_SPECIES], off_n[PIC_MAX_SPECIES],
        off_f[PIC_MAX_SPECIES][10];
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        const pic_particles_t &p = inj[s];
        if (p.n < 0) return fail(c, PIC_ERR_ARG, "negative injection count");
        if (p.n > c->cfg.sp[s].capacity) return fail(c, PIC_ERR_OVERFLOW, "injection exceeds the capacity");
        if (p.n > 0) {
            const float *src[9] = {p.ox, p.oy, p.ux, p.uy, p.uz, p.sx, p.sy, p.sz, p.w};
            if (!p.ix || !p.iy || !p.id || (d3 && (!p.iz || !p.oz))) return fail(c, PIC_ERR_ARG, "null particle array");
            for (int k = 0; k < 9; ++k)
                if (!src[k]) return fail(c, PIC_ERR_ARG, "null particle array");
        }
        const size_t n = (size_t)p.n;
        off_cell[s] = bytes, bytes += up16(n * 4);
        off_id[s] = bytes, bytes += up16(n * 4);
        off_n[s] = bytes, bytes += 16;
        for (int k = 0; k < nf; ++k) off_f[s][k] = bytes, bytes += up16(n * rb);
    }
    Slab b;
    CK(cudaMalloc(&b.mem, bytes));
    char *base = static_cast<char *>(b.mem);
    const int xlo = c->cfg.bc_x == PIC_BC_OPEN ? 2 : 0;
    const int xhi = c->cfg.bc_x == PIC_BC_OPEN ? c->cfg.nx - 3 : c->cfg.nx - 1;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < c->cfg.nspecies && e == cudaSuccess; ++s) {
        const pic_particles_t &p = inj[s];
        const size_t n = (size_t)p.n;
        b.n[s] = p.n;
        b.cell[s] = reinterpret_cast<uint32_t *>(base + off_cell[s]);
        b.id[s] = reinterpret_cast<int32_t *>(base + off_id[s]);
        b.n_dev[s] = reinterpret_cast<int32_t *>(base + off_n[s]);
        for (int k = 0; k < nf; ++k) b.f[s][k] = base + off_f[s][k];
        const int32_t n32 = (int32_t)n;
        e = cudaMemcpyAsync(b.n_dev[s], &n32, sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (n == 0 || e != cudaSuccess) continue;
        // cell indices through the scratch (3 x the capacity)
        const size_t room = (size_t)c->cfg.sp[s].capacity;
        int32_t *dix = c->scratch_i32, *diy = dix + room, *diz = diy + room;
        e = cudaMemcpyAsync(dix, p.ix, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(diy, p.iy, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && d3) e = cudaMemcpyAsync(diz, p.iz, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = d3 ? launch_pack_cells3(dix, diy, diz, b.cell[s], (int)n, xlo, xhi, c->cfg.ny, c->cfg.nz, c->err, st)
                   : launch_pack_cells(dix, diy, b.cell[s], (int)n, xlo, xhi, c->cfg.ny, c->err, st);
        const float *src3[10] = {p.ox, p.oy, p.oz, p.ux, p.uy, p.uz, p.sx, p.sy, p.sz, p.w};
        const float *src2[9] = {p.ox, p.oy, p.ux, p.uy, p.uz, p.sx, p.sy, p.sz, p.w};
        for (int k = 0; k < nf && e == cudaSuccess; ++k) {
            const float *from = d3 ? src3[k] : src2[k];
            if (rb == 4) {
                e = cudaMemcpyAsync(b.f[s][k], from, n * sizeof(float), cudaMemcpyHostToDevice, st);
            } else {
                e = cudaMemcpyAsync(c->stage, from, n * sizeof(float), cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess)
                    e = launch_convert<float, double>(static_cast<float *>(c->stage), static_cast<double *>(b.f[s][k]),
                                                      n, st);
            }
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.id[s], p.id, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        // the scratch and the staging buffer are reused by the next species
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(b.mem);
        return fail(c, PIC_ERR_CUDA, std::string("staging the window plasma: ") + cudaGetErrorString(e));
    }
    pic_status_t r = check_flags(c, st);
    if (r != PIC_OK) {
        cudaFree(b.mem);
        return r;
    }
    *out = b;
    return PIC_OK;
}

// One move of the co-moving window by ncells cells (the operation
// pic_shift_window describes) without host synchronisation: the mesh rows
// slide in place; each species either keeps the binned layout, its ranges
// relabelled by whole tile columns (ncells a multiple of the tile width: the
// ranges of the columns that left take the plasma of the uncovered ones, no
// particle moves), or takes the compact path: cells shifted, the plasma
// appended after the slots in use, a sort.  slab: the plasma, or nullptr.
pic_status_t window_move(Ctx *c, int ncells, const Slab *slab, cudaStream_t st) {
    const bool d3 = c->dim == 3;
    CK(with_real(c, [&](auto z) -> cudaError_t {
        using T = decltype(z);
        WindowRows<T> a{};
        T *EB = static_cast<T *>(c->EB), *J = static_cast<T *>(c->J);
        for (int k = 0; k < 6; ++k) a.plane[k] = EB + k * c->plane;
        for (int k = 0; k < 3; ++k) a.plane[6 + k] = J + k * c->plane;
        a.plane[9] = static_cast<T *>(c->rho_bg);
        a.nplanes = 10;
        a.by = 4;
        a.bz = 5;
        a.bnd = static_cast<T *>(c->bnd);
        a.rows = c->bnd_n;
        a.nx = c->cfg.nx;
        a.ld = c->ld;
        a.n = ncells;
        return launch_window_rows<T>(a, st);
    }));
    c->launches += 1;
    bool sort[PIC_MAX_SPECIES] = {};
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        const int64_t m = slab ? slab->n[s] : 0;
        const bool rotate = d3 && c->sp_binned[s] && ncells % c->tg3.TX == 0;
        if (!rotate && c->sp_binned[s]) {
            pic_status_t r = sort_species(c, s, st, true);  // to the compact layout first
            if (r != PIC_OK) return r;
        }
        const int cur = c->cur[s];
        if (rotate) {
            const int nt = c->ntiles, nr = nt + 1, ntx = c->tg3.ntx, kt = ncells / c->tg3.TX;
            int32_t *cnt = c->bin_cnt[s][cur];
            // every slot of the ranges (the span is tile_start[nt + 1])
            CK(launch_shift_cells(c->buf[s][cur].cell, c->tile_start[s] + nt + 1, c->n_upper[s], ncells, true, st));
            c->bin_txo[s] = (c->bin_txo[s] + kt) % ntx;
            CK(launch_window_vacate(cnt, nr, ntx, c->tg3.nty * c->tg3.ntz, kt, c->bin_txo[s], st));
            c->launches += 2;
            if (m > 0) {
                CK(with_real(c, [&](auto z) {
                    using T = decltype(z);
                    return launch_window_inject3<T>(slab_arrays<T>(*slab, s), (int)m, buf_arrays<T>(c, s, cur),
                                                    c->tile_start[s], cnt, c->tg3, c->bin_txo[s], c->err, st);
                }));
                c->launches += 1;
            }
            // arrival bases (and the overflow alert) from the new counters
            SealArgs a{};
            a.nranges = nr;
            a.fill = false;
            a.counters = true;
            a.ovf_alert = c->ovf_alert_dev;
            a.nsp = 1;
            a.sp[0] = SealSpecies{c->buf[s][cur].cell, c->tile_start[s], cnt, nullptr};
            CK(launch_seal_bins(a, st));
            c->launches += 1;
        } else {
            CK(launch_shift_cells(c->buf[s][cur].cell, c->n_dev + s, c->n_upper[s], ncells, d3, st));
            c->launches += 1;
            if (m > 0) {
                CK(with_real(c, [&](auto z) {
                    using T = decltype(z);
                    return launch_window_append<T>(slab_arrays<T>(*slab, s), (int)m, buf_arrays<T>(c, s, cur),
                                                   c->n_dev + s, (int)c->cfg.sp[s].capacity, d3, c->err, st);
                }));
                c->launches += 2;
                c->n_upper[s] = (int)std::min<int64_t>((int64_t)c->n_upper[s] + m, c->cfg.sp[s].capacity);
                c->tile_ordered[s] = false;  // appended after the last tile's range
            }
            sort[s] = true;
        }
        // n_live stays a bound at once; the sample of a binned species (after
        // its plasma) tightens it when it completes
        if (m > 0) add_live(c, s, m);
        if (rotate) {
            pic_status_t lr = live_sample(c, s, st);
            if (lr != PIC_OK) return lr;
        }
        if (m > 0) {
            if (c->has_background) {
                // the plasma brings its immobile ions: rho_bg -= rho(plasma),
                // deposited with the charge negated
                CK(with_real(c, [&](auto z) -> cudaError_t {
                    using T = decltype(z);
                    const SortArrays<T> b = slab_arrays<T>(*slab, s);
                    if (d3) {
                        DevSpecies3<T> v{};
                        v.cell = b.cell;
                        v.ox = b.f[0], v.oy = b.f[1], v.oz = b.f[2], v.w = b.f[9];
                        v.q = (T)(-c->cfg.sp[s].q);
                        v.n = b.n;
                        return launch_rho3<T>(v, (int)m, mesh3<T>(c), static_cast<T *>(c->rho_bg), st);
                    }
                    DevSpecies<T> v{};
                    v.cell = b.cell;
                    v.ox = b.f[0], v.oy = b.f[1], v.w = b.f[8];
                    v.q = (T)(-c->cfg.sp[s].q);
                    v.n = b.n;
                    return launch_rho<T>(v, (int)m, mesh<T>(c), static_cast<T *>(c->rho_bg), st);
                }));
                c->launches += 1;
            }
        }
    }
    bool all = true;
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        if (!sort[s]) {
            all = false;
            continue;
        }
        pic_status_t r = sort_species(c, s, st);
        if (r != PIC_OK) return r;
    }
    if (all) c->since_sort = 0;
    c->window += ncells;
    return PIC_OK;
}

// the window's next move is due before the step from index n: the box lags
// the light front (speed w_speed, leaving at step w_start) by ncells cells
bool window_due(const Ctx *c, long long n) {
    if (c->w_ncells <= 0 || n < c->w_start) return false;
    const double front = std::floor((double)(n - c->w_start) * c->dt * c->w_speed / c->dx);
    return (double)(c->window - c->w_window0 + c->w_ncells) <= front;
}

// steps from the current index to the next due move (>= 1 when none is due
// now; LLONG_MAX with the window off)
long long window_next(const Ctx *c) {
    if (c->w_ncells <= 0) return LLONG_MAX;
    const double need = (double)(c->window - c->w_window0 + c->w_ncells) * c->dx / (c->dt * c->w_speed);
    long long n = c->w_start + (long long)std::ceil(need) - 2;
    n = std::max(n, c->step + 1);
    for (int k = 0; k < 64 && !window_due(c, n); ++k) ++n;
    return n - c->step;
}

// the moves due before the current step, each with the oldest staged plasma
pic_status_t window_catch_up(Ctx *c, cudaStream_t st) {
    while (window_due(c, c->step)) {
        Slab b;
        const bool have = !c->inj_queue.empty();
        if (have) {
            b = c->inj_queue.front();
            c->inj_queue.pop_front();
            c->inj_spent.push_back(b.mem);
        }
        pic_status_t r = window_move(c, c->w_ncells, have ? &b : nullptr, st);
        if (r != PIC_OK) return r;
    }
    return PIC_OK;
}

}  // namespace

void set_global_error(const std::string &msg) { g_create_error = msg; }

extern "C" {

pic_status_t pic_validate_config(const pic_config_t *cfg) {
    Ctx *c = nullptr;
    if (!cfg) return fail(c, PIC_ERR_ARG, "null config");
    if (cfg->dim != 0 && cfg->dim != 2 && cfg->dim != 3) return fail(c, PIC_ERR_ARG, "dim must be 2 or 3 (0: 2)");
    const bool d3 = cfg->dim == 3;
    if (!d3 && (cfg->nx < 8 || cfg->ny < 4 || cfg->nx > 32767 || cfg->ny > 32767))
        return fail(c, PIC_ERR_ARG, "nx must be in [8, 32767] and ny in [4, 32767]");
    if (d3 && (cfg->nx < 8 || cfg->ny < 4 || cfg->nz < 4 || cfg->nx > PIC3_MAX_NX || cfg->ny > PIC3_MAX_NY ||
               cfg->nz > PIC3_MAX_NZ))
        return fail(c, PIC_ERR_ARG, "3D3V needs 8 <= nx <= 2044, 4 <= ny <= 2044, 4 <= nz <= 1020");
    if (d3 && !(cfg->dz_lambda > 0)) return fail(c, PIC_ERR_ARG, "dz_lambda must be > 0");
    if (!(cfg->dx_lambda > 0) || !(cfg->dy_lambda > 0)) return fail(c, PIC_ERR_ARG, "cell sizes must be > 0");
    if (!(cfg->cfl > 0 && cfg->cfl < 1)) return fail(c, PIC_ERR_ARG, "cfl must be in (0, 1)");
    if (cfg->bc_x != PIC_BC_OPEN && cfg->bc_x != PIC_BC_PERIODIC) return fail(c, PIC_ERR_ARG, "bad bc_x");
    if (cfg->pol < PIC_POL_NONE || cfg->pol > PIC_POL_CP) return fail(c, PIC_ERR_ARG, "bad pol");
    if (cfg->pol != PIC_POL_NONE && cfg->bc_x == PIC_BC_OPEN &&
        (!(cfg->waist_lambda > 0) || !(cfg->fwhm_periods > 0)))
        return fail(c, PIC_ERR_ARG, "laser needs waist_lambda > 0 and fwhm_periods > 0");
    if (cfg->nspecies < 1 || cfg->nspecies > PIC_MAX_SPECIES) return fail(c, PIC_ERR_ARG, "nspecies must be 1..4");
    for (int s = 0; s < cfg->nspecies; ++s) {
        const pic_species_t &sp = cfg->sp[s];
        if (!(sp.m > 0)) return fail(c, PIC_ERR_ARG, "species mass must be > 0");
        if (sp.capacity < 0 || sp.capacity > 0x7FFFFFF0LL)
            return fail(c, PIC_ERR_ARG, "species capacity must be in [0, 2^31 - 16]");
    }
    if (!d3 && (cfg->tile_x != 0 || cfg->tile_y != 0) && !fused_tile_supported(cfg->tile_x, cfg->tile_y))
        return fail(c, PIC_ERR_ARG, "tile must be one of 8x4, 16x8, 32x8, 32x16, 64x16 cells");
    if (d3 && (cfg->tile_x != 0 || cfg->tile_y != 0 || cfg->tile_z != 0) &&
        !fused3_tile_supported(cfg->tile_x, cfg->tile_y, cfg->tile_z))
        return fail(c, PIC_ERR_ARG, "3D3V tile must be one of 16x4x4, 8x8x4, 8x4x4, 16x8x4, 32x4x4 cells");
    if (d3) {
        // the tile sort keys every cell of the tile-padded mesh with a 32-bit
        // signed index (tile, cell inside the tile)
        const bool dflt = cfg->tile_x == 0 && cfg->tile_y == 0 && cfg->tile_z == 0;
        const int64_t tx = dflt ? 16 : cfg->tile_x, ty = dflt ? 4 : cfg->tile_y, tz = dflt ? 4 : cfg->tile_z;
        const int64_t padded = (cfg->nx + tx - 1) / tx * tx * ((cfg->ny + ty - 1) / ty * ty) *
                               ((cfg->nz + tz - 1) / tz * tz);
        if (padded > INT_MAX)
            return fail(c, PIC_ERR_ARG, "3D3V mesh padded to whole tiles must hold at most 2^31 - 1 cells");
    }
    if (cfg->sort_every < 0) return fail(c, PIC_ERR_ARG, "sort_every must be >= 0");
    if (cfg->bin_headroom_pct < 0 || cfg->bin_headroom_pct > 400 || cfg->bin_min_extra < 0 ||
        cfg->bin_min_extra > 4096)
        return fail(c, PIC_ERR_ARG, "bin_headroom_pct must be in [0, 400] and bin_min_extra in [0, 4096]");
    if (cfg->bin_headroom_pct > 0 && !d3) return fail(c, PIC_ERR_ARG, "the binned layout is 3D3V only");
    if (cfg->precision != 0 && cfg->precision != 32 && cfg->precision != 64)
        return fail(c, PIC_ERR_ARG, "precision must be 32 or 64 (0: 32)");
    return PIC_OK;
}

pic_status_t pic_create(const pic_config_t *cfg, void *stream, void **ctx_out) {
    Ctx *c = nullptr;
    if (!ctx_out) return fail(c, PIC_ERR_ARG, "null ctx_out");
    *ctx_out = nullptr;
    pic_status_t v = pic_validate_config(cfg);
    if (v != PIC_OK) return v;
    c = new (std::nothrow) Ctx();
    if (!c) return fail(nullptr, PIC_ERR_CUDA, "host allocation failed");
    c->cfg = *cfg;
    if (c->cfg.sort_every == 0) c->cfg.sort_every = 32;
    if (c->cfg.precision == 0) c->cfg.precision = 32;
    c->rb = c->cfg.precision == 64 ? 8 : 4;
    c->dim = c->cfg.dim == 3 ? 3 : 2;
    c->binned = c->dim == 3 && c->cfg.bin_headroom_pct > 0;
    cudaStream_t st = S(stream);
    auto bail = [&](pic_status_t s) {
        g_create_error = c->last_error;
        pic_destroy(c);
        return s;
    };
#define CKC(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            c->last_error = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return bail(PIC_ERR_CUDA);                                                         \
        }                                                                                      \
    } while (0)
    CKC(cudaGetDevice(&c->device));
    c->dx = cfg->dx_lambda * kTwoPi;
    c->dy = cfg->dy_lambda * kTwoPi;
    c->dz = c->dim == 3 ? cfg->dz_lambda * kTwoPi : 0.0;
    {
        double s2 = 1.0 / (c->dx * c->dx) + 1.0 / (c->dy * c->dy);
        if (c->dim == 3) s2 += 1.0 / (c->dz * c->dz);
        c->dt = cfg->cfl / std::sqrt(s2);
    }
    c->ld = round_up(cfg->nx, 32);
    c->bnd_n = (size_t)cfg->ny * (c->dim == 3 ? cfg->nz : 1);
    c->plane = (size_t)c->ld * c->bnd_n;
    choose_tiles(c);
    const size_t rb = c->rb;
    CKC(cudaMalloc(&c->EB, 6 * c->plane * rb));
    CKC(cudaMalloc(&c->J, 3 * c->plane * rb));
    CKC(cudaMalloc(&c->bnd, 2 * c->bnd_n * rb));
    CKC(cudaMalloc(&c->rho, c->plane * rb));
    CKC(cudaMalloc(&c->rho_bg, c->plane * rb));
    CKC(cudaMemsetAsync(c->EB, 0, 6 * c->plane * rb, st));
    CKC(cudaMemsetAsync(c->J, 0, 3 * c->plane * rb, st));
    CKC(cudaMemsetAsync(c->bnd, 0, 2 * c->bnd_n * rb, st));
    CKC(cudaMemsetAsync(c->rho_bg, 0, c->plane * rb, st));
    int64_t capmax = 0;
    for (int s = 0; s < cfg->nspecies; ++s) {
        const size_t cap = (size_t)cfg->sp[s].capacity;
        capmax = capmax > (int64_t)cap ? capmax : (int64_t)cap;
        for (int b = 0; b < 2; ++b) {
            CKC(cudaMalloc(&c->buf[s][b].cell, cap * sizeof(uint32_t) + 16));
            for (int k = 0; k < 9; ++k) CKC(cudaMalloc(&c->buf[s][b].f[k], cap * rb + 16));
            if (c->dim == 3) CKC(cudaMalloc(&c->buf[s][b].oz, cap * rb + 16));
            CKC(cudaMalloc(&c->buf[s][b].id, cap * sizeof(int32_t) + 16));
        }
        CKC(cudaMalloc(&c->tile_start[s], (c->ntiles + 2) * sizeof(int32_t)));
        CKC(cudaMemsetAsync(c->tile_start[s], 0, (c->ntiles + 2) * sizeof(int32_t), st));
        if (c->binned && cfg->sp[s].mobile && !c->ovf_alert) {
            int *h = nullptr;
            CKC(cudaHostAlloc(reinterpret_cast<void **>(&h), sizeof(int), cudaHostAllocMapped));
            *h = 0;
            c->ovf_alert = h;
            CKC(cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->ovf_alert_dev), h, 0));
        }
        if (!c->old_start) CKC(cudaMalloc(&c->old_start, (c->ntiles + 2) * sizeof(int32_t)));
        if (c->binned && cfg->sp[s].mobile)
            for (int b = 0; b < 2; ++b) {
                CKC(cudaMalloc(&c->bin_cnt[s][b], 4 * (c->ntiles + 1) * sizeof(int32_t)));
                CKC(cudaMemsetAsync(c->bin_cnt[s][b], 0, 4 * (c->ntiles + 1) * sizeof(int32_t), st));
            }
    }
    CKC(cudaMalloc(&c->tile_count, (c->ntiles + 1) * sizeof(int32_t)));
    CKC(cudaMalloc(&c->cell_count, (size_t)c->ntiles * tile_cells(c) * sizeof(int32_t)));
    CKC(cudaMalloc(&c->cell_off, (size_t)c->ntiles * tile_cells(c) * sizeof(int32_t)));
    CKC(cudaMalloc(&c->tile_info, (size_t)c->ntiles * kTileInfo * sizeof(int32_t)));
    CKC(cudaMalloc(&c->tile_cursor, c->ntiles * sizeof(int32_t)));
    CKC(cudaMalloc(&c->n_dev, (PIC_MAX_SPECIES + 1) * sizeof(int32_t)));
    CKC(cudaMemsetAsync(c->n_dev, 0, (PIC_MAX_SPECIES + 1) * sizeof(int32_t), st));
    CKC(cudaMalloc(&c->scratch_i32, 3 * (size_t)capmax * sizeof(int32_t) + 16));
    c->stage_elems = std::max((size_t)capmax, c->plane);
    CKC(cudaMalloc(&c->stage, c->stage_elems * sizeof(double) + 16));
    CKC(cudaMalloc(&c->err, sizeof(unsigned)));
    CKC(cudaMemsetAsync(c->err, 0, sizeof(unsigned), st));
    CKC(cudaMalloc(&c->partials, (size_t)reduce_blocks() * 8 * sizeof(double)));
    CKC(cudaMalloc(&c->result, 64 * sizeof(double)));  // moments results and diagnostic column sums
    CKC(cudaMalloc(&c->hist, (size_t)PIC_MAX_HIST_BINS * 5 * sizeof(double)));
    CKC(cudaMalloc(&c->diag_rows, (size_t)(c->ntiles + Ctx::kBinCtasMax) * PIC_MAX_SPECIES * 8 * sizeof(double)));
    CKC(cudaMalloc(&c->diag_shift, PIC_MAX_SPECIES * sizeof(double)));
    CKC(cudaMemsetAsync(c->diag_shift, 0, PIC_MAX_SPECIES * sizeof(double), st));
    CKC(cudaMalloc(&c->diag_out, PIC_MAX_SPECIES * sizeof(pic_moments_dev)));
    CKC(cudaMemsetAsync(c->diag_out, 0, PIC_MAX_SPECIES * sizeof(pic_moments_dev), st));
    {
        std::vector<double> prof(2 * c->bnd_n);
        if (c->dim == 3)
            laser_profile3(laser(c), cfg->ny, cfg->nz, c->dz, prof.data());
        else
            laser_profile(laser(c), cfg->ny, prof.data());
        CKC(cudaMalloc(&c->laser_prof, prof.size() * sizeof(double)));
        CKC(cudaMemcpyAsync(c->laser_prof, prof.data(), prof.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        CKC(cudaStreamSynchronize(st));
    }
    if (make_tensor_map(c) != PIC_OK) return bail(PIC_ERR_CUDA);
    CKC(cudaStreamSynchronize(st));
#undef CKC
    *ctx_out = c;
    return PIC_OK;
}

void pic_destroy(void *ctx) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return;
    free_own(c, c->EB);
    free_own(c, c->J);
    cudaFree(c->bnd);
    cudaFree(c->rho);
    cudaFree(c->rho_bg);
    cudaFree(c->stage);
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
        for (int b = 0; b < 2; ++b) {
            free_own(c, c->buf[s][b].cell);
            for (int k = 0; k < 9; ++k) free_own(c, c->buf[s][b].f[k]);
            free_own(c, c->buf[s][b].oz);
            free_own(c, c->buf[s][b].id);
        }
        cudaFree(c->tile_start[s]);
        if (s == 0) cudaFree(c->old_start);
        cudaFree(c->bin_cnt[s][0]);
        cudaFree(c->bin_cnt[s][1]);
        cudaFree(c->cell_old[s]);
        for (int k = 0; k < 3; ++k) cudaFree(c->old_f[s][k]);
        for (int k = 0; k < 9; ++k) cudaFree(c->adj_lam[s][k]);
        cudaFree(c->adj_cell0[s]);
    }
    cudaFree(c->tile_count);
    cudaFree(c->cell_count);
    cudaFree(c->cell_off);
    cudaFree(c->tile_info);
    cudaFree(c->tile_cursor);
    cudaFree(c->n_dev);
    cudaFree(c->scratch_i32);
    cudaFree(c->err);
    cudaFree(c->partials);
    cudaFree(c->result);
    cudaFree(c->diag_rows);
    cudaFree(c->diag_shift);
    cudaFree(c->diag_out);
    cudaFree(c->laser_prof);
    cudaFree(c->hist);
    if (c->ovf_alert) cudaFreeHost(const_cast<int *>(c->ovf_alert));
    for (auto &b : c->inj_queue) cudaFree(b.mem);
    for (void *m : c->inj_spent) cudaFree(m);
    if (c->live_host) {
        cudaFreeHost(const_cast<long long *>(c->live_host));
        for (int s = 0; s < PIC_MAX_SPECIES; ++s)
            if (c->live_ev[s]) cudaEventDestroy(c->live_ev[s]);
    }
    drop_step_graphs(c);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (int k = 0; k < 2; ++k)
        if (c->gev[k]) cudaEventDestroy(c->gev[k]);
    cudaFree(c->laser_tab);
    for (int k = 0; k < Ctx::kAhead; ++k)
        if (c->ahead_ev[k]) cudaEventDestroy(c->ahead_ev[k]);
    delete c;
}

pic_status_t pic_get_grid(void *ctx, double *dt, double *dx, double *dy, double *dz) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (dt) *dt = c->dt;
    if (dx) *dx = c->dx;
    if (dy) *dy = c->dy;
    if (dz) *dz = c->dz;
    return PIC_OK;
}

pic_status_t pic_set_particles(void *ctx, int s, const pic_particles_t *p, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (s < 0 || s >= c->cfg.nspecies || !p) return fail(c, PIC_ERR_ARG, "bad species or particles");
    if (p->n < 0) return fail(c, PIC_ERR_ARG, "negative particle count");
    if (p->n > c->cfg.sp[s].capacity) return fail(c, PIC_ERR_OVERFLOW, "more particles than capacity");
    cudaStream_t st = S(stream);
    pic_status_t r = upload_particles<float>(c, s, p, 0, st);
    if (r != PIC_OK) return r;
    c->pending_deposit = false;
    r = sort_species(c, s, st);
    if (r != PIC_OK) return r;
    c->since_sort = 0;
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status_t pic_set_particles_f64(void *ctx, int s, const pic_particles_f64_t *p, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (s < 0 || s >= c->cfg.nspecies || !p) return fail(c, PIC_ERR_ARG, "bad species or particles");
    if (p->n < 0) return fail(c, PIC_ERR_ARG, "negative particle count");
    if (p->n > c->cfg.sp[s].capacity) return fail(c, PIC_ERR_OVERFLOW, "more particles than capacity");
    if (p->n > 0 && (int64_t)c->stage_elems < p->n) return fail(c, PIC_ERR_ARG, "too many particles");
    cudaStream_t st = S(stream);
    pic_status_t r = upload_particles<double>(c, s, p, 0, st);
    if (r != PIC_OK) return r;
    c->pending_deposit = false;
    r = sort_species(c, s, st);
    if (r != PIC_OK) return r;
    c->since_sort = 0;
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

pic_status_t pic_get_count(void *ctx, int s, int64_t *n) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (s < 0 || s >= c->cfg.nspecies || !n) return fail(c, PIC_ERR_ARG, "bad species");
    int32_t v = 0;
    pic_status_t r = read_count(c, s, nullptr, &v);
    *n = v;
    return r;
}

}  // extern "C"

// particle slots of one species -> host arrays of float (OutT = float) or
// double (OutT = double), whatever the context's precision
template <typename OutT, typename PT>
static pic_status_t get_particles_t(Ctx *c, int s, PT *out, cudaStream_t st) {
    if (s < 0 || s >= c->cfg.nspecies || !out) return fail(c, PIC_ERR_ARG, "bad species or output");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    if (c->sp_binned[s]) {
        // the spare slots of the binned ranges hold stale records: read back
        // the compact layout (the next step re-bins)
        pic_status_t r = sort_species(c, s, st, true);
        if (r != PIC_OK) return r;
    }
    int32_t nv = 0;
    pic_status_t rc = read_count(c, s, st, &nv);
    if (rc != PIC_OK) return rc;
    const size_t n = (size_t)nv;
    if ((int64_t)n > out->n) return fail(c, PIC_ERR_ARG, "output arrays too small");
    out->n = (int64_t)n;
    if (!n) return PIC_OK;
    const bool d3 = c->dim == 3;
    OutT *dst[10] = {out->ox, out->oy, out->ux, out->uy, out->uz, out->sx, out->sy, out->sz, out->w, out->oz};
    if (!out->ix || !out->iy || !out->id || (d3 && (!out->iz || !out->oz)))
        return fail(c, PIC_ERR_ARG, "null output array");
    for (int k = 0; k < 9; ++k)
        if (!dst[k]) return fail(c, PIC_ERR_ARG, "null output array");
    const SpeciesBuf &B = c->buf[s][c->cur[s]];
    const size_t cap = (size_t)c->cfg.sp[s].capacity;
    int32_t *dix = c->scratch_i32, *diy = c->scratch_i32 + cap, *diz = c->scratch_i32 + 2 * cap;
    if (d3)
        CK(launch_unpack_cells3(B.cell, dix, diy, diz, (int)n, st));
    else
        CK(launch_unpack_cells(B.cell, dix, diy, (int)n, st));
    c->launches += 1;
    CK(cudaMemcpyAsync(out->ix, dix, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out->iy, diy, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (d3) CK(cudaMemcpyAsync(out->iz, diz, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    for (int k = 0; k < (d3 ? 10 : 9); ++k) {
        const void *from = k < 9 ? B.f[k] : B.oz;
        if ((size_t)c->rb == sizeof(OutT)) {
            CK(cudaMemcpyAsync(dst[k], from, n * sizeof(OutT), cudaMemcpyDeviceToHost, st));
        } else {
            if (c->rb == 8)
                CK(launch_convert<double, float>(static_cast<const double *>(from), static_cast<float *>(c->stage), n, st));
            else
                CK(launch_convert<float, double>(static_cast<const float *>(from), static_cast<double *>(c->stage), n, st));
            c->launches += 1;
            CK(cudaMemcpyAsync(dst[k], c->stage, n * sizeof(OutT), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));  // stage is reused by the next array
        }
    }
    CK(cudaMemcpyAsync(out->id, B.id, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    // device error flags of the steps before (a binned step that dropped
    // particles, a non-finite value) are reported with the state they concern
    return check_flags(c, st);
}

extern "C" {

pic_status_t pic_get_particles(void *ctx, int s, pic_particles_t *out, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    return get_particles_t<float>(c, s, out, S(stream));
}

pic_status_t pic_get_particles_f64(void *ctx, int s, pic_particles_f64_t *out, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    return get_particles_t<double>(c, s, out, S(stream));
}

}  // extern "C"

// one pitched device array of `rows` x `cols` reals <-> a dense host array of
// HostT, converting through the staging buffer when the types differ
template <typename HostT>
static pic_status_t xfer_plane(Ctx *c, HostT *host, void *dev, size_t rows, size_t cols, size_t pitch_elems,
                               bool to_dev, cudaStream_t st) {
    const size_t hp = cols * sizeof(HostT);
    if ((size_t)c->rb == sizeof(HostT)) {
        if (to_dev)
            CK(cudaMemcpy2DAsync(dev, pitch_elems * c->rb, host, hp, hp, rows, cudaMemcpyHostToDevice, st));
        else
            CK(cudaMemcpy2DAsync(host, hp, dev, pitch_elems * c->rb, hp, rows, cudaMemcpyDeviceToHost, st));
        return PIC_OK;
    }
    const size_t total = rows * pitch_elems;
    if (total > c->stage_elems) return fail(c, PIC_ERR_CUDA, "staging buffer too small");
    if (to_dev) {
        CK(cudaMemcpy2DAsync(c->stage, pitch_elems * sizeof(HostT), host, hp, hp, rows, cudaMemcpyHostToDevice, st));
        if (c->rb == 8)
            CK(launch_convert<float, double>(static_cast<const float *>(c->stage), static_cast<double *>(dev), total, st));
        else
            CK(launch_convert<double, float>(static_cast<const double *>(c->stage), static_cast<float *>(dev), total, st));
    } else {
        if (c->rb == 8)
            CK(launch_convert<double, float>(static_cast<const double *>(dev), static_cast<float *>(c->stage), total, st));
        else
            CK(launch_convert<float, double>(static_cast<const float *>(dev), static_cast<double *>(c->stage), total, st));
        CK(cudaMemcpy2DAsync(host, hp, c->stage, pitch_elems * sizeof(HostT), hp, rows, cudaMemcpyDeviceToHost, st));
    }
    c->launches += 1;
    CK(cudaStreamSynchronize(st));  // the stage is reused by the next plane
    return PIC_OK;
}

template <typename HostT, typename FT>
static pic_status_t copy_fields(Ctx *c, FT *f, bool to_dev, cudaStream_t st) {
    HostT *host[9] = {f->ex, f->ey, f->ez, f->bx, f->by, f->bz, f->jx, f->jy, f->jz};
    const size_t nx = c->cfg.nx, ny = c->bnd_n;  // rows: ny (2D3V) or nz * ny (3D3V)
    for (int k = 0; k < 9; ++k) {
        if (!host[k]) continue;
        char *base = static_cast<char *>(k < 6 ? c->EB : c->J);
        void *d = base + (size_t)(k < 6 ? k : k - 6) * c->plane * c->rb;
        pic_status_t r = xfer_plane<HostT>(c, host[k], d, ny, nx, c->ld, to_dev, st);
        if (r != PIC_OK) return r;
    }
    HostT *lb[2] = {f->by_left, f->bz_left};
    for (int k = 0; k < 2; ++k) {
        if (!lb[k]) continue;
        void *d = static_cast<char *>(c->bnd) + (size_t)k * ny * c->rb;
        pic_status_t r = xfer_plane<HostT>(c, lb[k], d, 1, ny, ny, to_dev, st);
        if (r != PIC_OK) return r;
    }
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

extern "C" {

pic_status_t pic_set_fields(void *ctx, const pic_fields_t *f, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!f) return fail(c, PIC_ERR_ARG, "null fields");
    pic_fields_t tmp = *f;
    return copy_fields<float>(c, &tmp, true, S(stream));
}

pic_status_t pic_get_fields(void *ctx, pic_fields_t *f, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!f) return fail(c, PIC_ERR_ARG, "null fields");
    return copy_fields<float>(c, f, false, S(stream));
}

pic_status_t pic_get_fields_f64(void *ctx, pic_fields_f64_t *f, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!f) return fail(c, PIC_ERR_ARG, "null fields");
    return copy_fields<double>(c, f, false, S(stream));
}

pic_status_t pic_set_step(void *ctx, int64_t step) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    c->step = step;
    return PIC_OK;
}

pic_status_t pic_get_step(void *ctx, int64_t *step) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !step) return fail(c, PIC_ERR_ARG, "null argument");
    *step = c->step;
    return PIC_OK;
}

pic_status_t pic_gather_push_spin(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    pic_status_t sr = seal_pending(c, st);  // the split kernels read every slot
    if (sr != PIC_OK) return sr;
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        if (!c->cfg.sp[s].mobile) continue;
        pic_status_t r = alloc_old(c, s);
        if (r != PIC_OK) return r;
    }
    for (int s = 0; s < c->cfg.nspecies; ++s)
        if (c->cfg.sp[s].mobile) {
            CK(with_real(c, [&](auto z) {
                using T = decltype(z);
                if (c->dim == 3) return launch_push_split3<T>(step_params3<T>(c), s, c->n_upper[s], st);
                return launch_push_split<T>(step_params<T>(c), s, c->n_upper[s], st);
            }));
            c->launches += 1;
        }
    c->pending_deposit = true;
    return PIC_OK;
}

pic_status_t pic_deposit(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!c->pending_deposit) return fail(c, PIC_ERR_STATE, "no pending move: call pic_gather_push_spin first");
    cudaStream_t st = S(stream);
    for (int s = 0; s < c->cfg.nspecies; ++s)
        if (c->cfg.sp[s].mobile) {
            CK(with_real(c, [&](auto z) {
                using T = decltype(z);
                if (c->dim == 3) return launch_deposit_split3<T>(step_params3<T>(c), s, c->n_upper[s], st);
                return launch_deposit_split<T>(step_params<T>(c), s, c->n_upper[s], st);
            }));
            c->launches += 1;
            // the split kernels move particles in their slots: a binned range
            // may now hold particles of other tiles, so the next binned step
            // re-bins first
            c->sp_binned[s] = false;
        }
    c->pending_deposit = false;
    return PIC_OK;
}

pic_status_t pic_field_update(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        if (c->dim == 3)
            return launch_field_update3<T>(mesh3<T>(c), static_cast<T *>(c->bnd), c->laser_prof, laser(c), c->dt,
                                           c->dx, c->dy, c->dz, c->step, S(stream), c->lf_capture);
        return launch_field_update<T>(mesh<T>(c), static_cast<T *>(c->bnd), c->laser_prof, laser(c), c->dt, c->dx,
                                      c->dy, c->step, S(stream), c->lf_capture);
    }));
    c->launches += c->cfg.bc_x == PIC_BC_OPEN ? 4 : 3;
    c->step += 1;
    return PIC_OK;
}

pic_status_t pic_push_deposit(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    const bool diag = c->diag_every > 0 && (c->step + 1) % c->diag_every == 0;
    DiagParams D{};
    if (diag) {
        D.on = 1;
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            D.lo[s] = c->diag_lo[s];
            D.hi[s] = c->diag_hi[s];
            D.m_mev[s] = c->cfg.sp[s].m * kMec2Mev;
        }
        D.shift = c->diag_shift;
        D.rows = c->diag_rows;
    }
    // binned layout: every mobile species must be in it (after a set of
    // particles, a compacting read-back or a window shift, re-bin first); an
    // overflow range past half full also asks for a re-bin
    bool rebin = false;
    cudaEvent_t ahead = nullptr;
    if (c->binned) {
        cudaEvent_t &ev = c->ahead_ev[c->ahead_k % Ctx::kAhead];
        if (!ev) CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        else if (c->ahead_k >= Ctx::kAhead) CK(cudaEventSynchronize(ev));
        ahead = ev;
    }
    if (c->binned && c->ovf_alert && *c->ovf_alert) {
        *c->ovf_alert = 0;
        rebin = true;
    }
    if (c->binned && (rebin || !all_binned(c))) {
        // re-bin every species when the capacities allow it, else bring the
        // binned ones back to the compact layout the compact kernel reads
        bool fits = true;
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            int ovf;
            int64_t span;
            refresh_live(c, s);
            if (c->cfg.sp[s].mobile && !bin_plan(c, s, &ovf, &span)) fits = false;
        }
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            if (!fits && !c->sp_binned[s]) continue;
            pic_status_t r = sort_species(c, s, S(stream), !fits);
            if (r != PIC_OK) return r;
        }
        c->since_sort = 0;
    }
    const bool bin = c->binned && all_binned(c);
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        if (c->dim == 3) {
            StepParams3<T> P = step_params3<T>(c);
            P.diag = D;
            if (bin) {
                P.nextra = c->bin_ctas;
                for (int s = 0; s < c->cfg.nspecies; ++s) {
                    if (!c->cfg.sp[s].mobile) continue;
                    const int to = 1 - c->cur[s];
                    const DevSpecies3<T> o = dev_species3<T>(c, s, to);
                    Bin3<T> &b = P.bin[s];
                    b.cell = o.cell;
                    T *f[10] = {o.ox, o.oy, o.oz, o.ux, o.uy, o.uz, o.sx, o.sy, o.sz, o.w};
                    for (int k = 0; k < 10; ++k) b.f[k] = f[k];
                    b.id = o.id;
                    b.cnt_in = c->bin_cnt[s][c->cur[s]];
                    b.cnt_out = c->bin_cnt[s][to];
                    b.txo = c->bin_txo[s];
                }
            }
            return launch_step_fused3<T>(P, c->tmapEB, bin, S(stream));
        }
        StepParams<T> P = step_params<T>(c);
        P.diag = D;
        return launch_step_fused<T>(P, c->tmapEB, S(stream));
    }));
    c->launches += bin ? 2 : 1;  // binned: the fused kernel and the overflow-range kernel
    if (bin) {
        // the particles now live in the other buffer: its arrival bases for
        // the next step, the consumed buffer's counters cleared; the slots
        // outside the new segments are sealed only when a slot-wise kernel
        // needs them (seal_pending)
        SealArgs a{};
        a.nranges = c->ntiles + 1;
        a.fill = false;
        a.counters = true;
        a.ovf_alert = c->ovf_alert_dev;
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            if (!c->cfg.sp[s].mobile) continue;
            const int to = 1 - c->cur[s];
            a.sp[a.nsp++] = SealSpecies{c->buf[s][to].cell, c->tile_start[s], c->bin_cnt[s][to],
                                        c->bin_cnt[s][c->cur[s]]};
            c->cur[s] = to;
            c->unsealed[s] = true;
        }
        CK(launch_seal_bins(a, S(stream)));
        c->launches += 1;
    }
    if (ahead) {
        CK(cudaEventRecord(ahead, S(stream)));
        c->ahead_k += 1;
    }
    if (diag) {
        const int ncols = c->ntiles + (bin ? c->bin_ctas : 0);
        CK(launch_diag_final(c->diag_rows, ncols, c->cfg.nspecies, c->diag_shift, c->diag_out, c->result,
                             S(stream)));
        c->launches += 2;
        c->diag_step = c->step + 1;
    }
    return PIC_OK;
}

pic_status_t pic_set_diagnostics(void *ctx, int every, const double *emin_mev, const double *emax_mev) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (every < 0) return fail(c, PIC_ERR_ARG, "every must be >= 0");
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        const double lo = emin_mev ? emin_mev[s] : -INFINITY, hi = emax_mev ? emax_mev[s] : INFINITY;
        if (!(lo < hi)) return fail(c, PIC_ERR_ARG, "energy window must have emin < emax");
        c->diag_lo[s] = lo;
        c->diag_hi[s] = hi;
    }
    c->diag_every = every;
    drop_step_graphs(c);  // the windows are kernel parameters of the captured steps
    return PIC_OK;
}

pic_status_t pic_get_diagnostics(void *ctx, pic_moments_t *out, int64_t *step, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!out) return fail(c, PIC_ERR_ARG, "null output");
    cudaStream_t st = S(stream);
    pic_moments_dev h[PIC_MAX_SPECIES];
    CK(cudaMemcpyAsync(h, c->diag_out, sizeof(h), cudaMemcpyDeviceToHost, st));
    pic_status_t fl = check_flags(c, st);
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        for (int k = 0; k < 3; ++k) out[s].P[k] = h[s].P[k];
        out[s].sum_w = h[s].sum_w;
        out[s].count = h[s].count;
        out[s].ekin_mean = h[s].ekin_mean;
        out[s].ekin_var = h[s].ekin_var;
    }
    if (step) *step = c->diag_step;
    return fl;
}

pic_status_t pic_sort(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        pic_status_t r = sort_species(c, s, S(stream));
        if (r != PIC_OK) return r;
    }
    c->since_sort = 0;
    return PIC_OK;
}

}  // extern "C"

// len whole steps (no sort among them) replayed from a CUDA graph on the
// context's stream, ordered after and before the caller's stream by events.
// The graph is captured at the first stretch with its key; the capture is
// itself the first execution (its host-side bookkeeping stands), later
// replays apply the recorded bookkeeping.  The laser time factors of the
// stretch are computed on the host as for launched steps and copied into the
// device table the captured boundary kernels read, so a replayed step runs
// the same kernels with the same arguments as a launched one.
static pic_status_t graph_steps(Ctx *c, int len, void *stream) {
    cudaStream_t user = S(stream);
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&c->gev[k], cudaEventDisableTiming));
        CK(cudaMalloc(&c->laser_tab, 2 * sizeof(double) * (size_t)std::max(c->graph_max, 1)));
    }
    unsigned parity = 0;
    for (int s = 0; s < c->cfg.nspecies; ++s) parity |= (unsigned)c->cur[s] << s;
    const int phase = c->diag_every > 0 ? (int)(c->step % c->diag_every) : -1;
    Ctx::StepGraph *g = nullptr;
    for (auto &e : c->graphs)
        if (e.len == len && e.phase == phase && e.parity == parity && e.gen == c->graph_gen) g = &e;
    std::vector<double> tab(2 * (size_t)len, 0.0);
    if (c->cfg.bc_x == PIC_BC_OPEN)
        for (int q = 0; q < len; ++q)
            laser_time_factors(laser(c), ((double)(c->step + q) + 0.5) * c->dt, &tab[2 * q], &tab[2 * q + 1]);
    CK(cudaEventRecord(c->gev[0], user));
    CK(cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    // pageable source: staged before the call returns, ordered before the replay
    CK(cudaMemcpyAsync(c->laser_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, c->gstream));
    if (g) {
        CK(cudaGraphLaunch(g->exec, c->gstream));
        const long long step0 = c->step;
        c->step += len;
        c->launches += g->launches;
        if (g->last_diag >= 0) c->diag_step = step0 + g->last_diag + 1;
        c->graph_replays += 1;
    } else {
        const long long step0 = c->step, launches0 = c->launches, diag0 = c->diag_step;
        CK(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeRelaxed));
        pic_status_t r = PIC_OK;
        for (int q = 0; q < len && r == PIC_OK; ++q) {
            c->lf_capture = c->laser_tab + 2 * q;
            r = pic_push_deposit(c, c->gstream);
            if (r == PIC_OK) r = pic_field_update(c, c->gstream);
        }
        c->lf_capture = nullptr;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->gstream, &graph);
        cudaGraphExec_t exec = nullptr;
        cudaError_t ei = cudaSuccess;
        if (r == PIC_OK && ec == cudaSuccess) ei = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (r != PIC_OK || ec != cudaSuccess || ei != cudaSuccess) {
            // nothing ran: the host-side bookkeeping of the capture is undone
            c->step = step0;
            c->launches = launches0;
            c->diag_step = diag0;
            if (exec) cudaGraphExecDestroy(exec);
            if (r != PIC_OK) return r;
            return fail(c, PIC_ERR_CUDA, std::string("pic_step graph capture: ") +
                                             cudaGetErrorString(ec != cudaSuccess ? ec : ei));
        }
        if ((int)c->graphs.size() >= Ctx::kMaxGraphs) {
            cudaGraphExecDestroy(c->graphs.front().exec);
            c->graphs.erase(c->graphs.begin());
        }
        Ctx::StepGraph e{len, phase, parity, c->graph_gen, exec, c->launches - launches0,
                         c->diag_step > step0 ? (int)(c->diag_step - 1 - step0) : -1};
        c->graphs.push_back(e);
        c->graph_captures += 1;
        CK(cudaGraphLaunch(exec, c->gstream));
    }
    CK(cudaEventRecord(c->gev[1], c->gstream));
    CK(cudaStreamWaitEvent(user, c->gev[1], 0));
    return PIC_OK;
}

extern "C" {

pic_status_t pic_step(void *ctx, int nsteps, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (nsteps < 0) return fail(c, PIC_ERR_ARG, "negative step count");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    // the binned layout decides on the host, between steps, whether to re-bin:
    // its steps are launched one by one
    const bool graphs = c->graph_max > 0 && !c->binned;
    int k = 0;
    while (k < nsteps) {
        // co-moving window: the moves due before this step, then stretches
        // that end where the next one is due
        pic_status_t r = window_catch_up(c, S(stream));
        if (r != PIC_OK) return r;
        if (c->since_sort >= c->cfg.sort_every) r = pic_sort(c, stream);
        if (r != PIC_OK) return r;
        int len = std::min(nsteps - k, c->cfg.sort_every - c->since_sort);
        len = (int)std::min<long long>(len, window_next(c));
        if (graphs && len >= 2) {
            len = std::min(len, c->graph_max);
            r = graph_steps(c, len, stream);
        } else {
            len = 1;
            r = pic_push_deposit(c, stream);
            if (r == PIC_OK) r = pic_field_update(c, stream);
        }
        if (r != PIC_OK) return r;
        c->since_sort += len;
        k += len;
    }
    return PIC_OK;
}

pic_status_t pic_set_graphs(void *ctx, int max_steps) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (max_steps < 0 || max_steps > 4096) return fail(c, PIC_ERR_ARG, "max_steps must be in [0, 4096]");
    drop_step_graphs(c);
    if (c->laser_tab && max_steps > c->graph_max) {
        cudaFree(c->laser_tab);
        c->laser_tab = nullptr;
        CK(cudaMalloc(&c->laser_tab, 2 * sizeof(double) * (size_t)max_steps));
    }
    c->graph_max = max_steps;
    return PIC_OK;
}

pic_status_t pic_graph_stats(void *ctx, int64_t *captures, int64_t *replays) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (captures) *captures = c->graph_captures;
    if (replays) *replays = c->graph_replays;
    return PIC_OK;
}

pic_status_t pic_polarization(void *ctx, int s, double emin, double emax, pic_moments_t *out, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (s < 0 || s >= c->cfg.nspecies || !out) return fail(c, PIC_ERR_ARG, "bad species or output");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    pic_status_t sr = seal_pending(c, st);
    if (sr != PIC_OK) return sr;
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        const T lo = std::isinf(emin) && emin < 0 ? -(T)INFINITY : (T)emin;
        const T hi = std::isinf(emax) && emax > 0 ? (T)INFINITY : (T)emax;
        return launch_moments<T>(dev_species<T>(c, s, c->cur[s]), (T)(c->cfg.sp[s].m * kMec2Mev), lo, hi,
                                 c->partials, c->result, st);
    }));
    c->launches += 4;
    double r[7];
    CK(cudaMemcpyAsync(r, c->result, 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
    pic_status_t fl = check_flags(c, st);
    const double sw = r[0];
    for (int k = 0; k < 3; ++k) out->P[k] = sw > 0 ? r[1 + k] / sw : 0.0;
    out->sum_w = sw;
    out->count = r[5];
    out->ekin_mean = sw > 0 ? r[4] / sw : 0.0;
    out->ekin_var = sw > 0 ? r[6] / sw : 0.0;
    return fl;
}

pic_status_t pic_energy_histogram(void *ctx, int s, double emin, double emax, int nbins, int log_bins,
                                  double *out, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (s < 0 || s >= c->cfg.nspecies || !out) return fail(c, PIC_ERR_ARG, "bad species or output");
    if (nbins < 1 || nbins > PIC_MAX_HIST_BINS) return fail(c, PIC_ERR_ARG, "nbins must be in [1, 1024]");
    if (!(emin < emax) || !std::isfinite(emin) || !std::isfinite(emax) || (log_bins && !(emin > 0)))
        return fail(c, PIC_ERR_ARG, "need finite emin < emax (and emin > 0 for log bins)");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    pic_status_t sr = seal_pending(c, st);
    if (sr != PIC_OK) return sr;
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        return launch_histogram<T>(dev_species<T>(c, s, c->cur[s]), (T)(c->cfg.sp[s].m * kMec2Mev), (T)emin,
                                   (T)emax, nbins, log_bins ? 1 : 0, c->hist, st);
    }));
    c->launches += 1;
    CK(cudaMemcpyAsync(out, c->hist, sizeof(double) * 5 * nbins, cudaMemcpyDeviceToHost, st));
    return check_flags(c, st);
}

pic_status_t pic_capture_background(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    c->has_background = true;
    cudaStream_t st = S(stream);
    pic_status_t sr = seal_pending(c, st);
    if (sr != PIC_OK) return sr;
    CK(cudaMemsetAsync(c->rho, 0, c->plane * c->rb, st));
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            cudaError_t e = c->dim == 3 ? launch_rho3<T>(dev_species3<T>(c, s, c->cur[s]), c->n_upper[s], mesh3<T>(c),
                                                          static_cast<T *>(c->rho), st)
                                        : launch_rho<T>(dev_species<T>(c, s, c->cur[s]), c->n_upper[s], mesh<T>(c),
                                                        static_cast<T *>(c->rho), st);
            if (e != cudaSuccess) return e;
        }
        return launch_negate_copy<T>(static_cast<const T *>(c->rho), static_cast<T *>(c->rho_bg), c->plane, st);
    }));
    c->launches += c->cfg.nspecies + 1;
    return PIC_OK;
}

pic_status_t pic_gauss_residual(void *ctx, double out[2], void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!out) return fail(c, PIC_ERR_ARG, "null output");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    pic_status_t sr = seal_pending(c, st);
    if (sr != PIC_OK) return sr;
    CK(cudaMemsetAsync(c->rho, 0, c->plane * c->rb, st));
    c->launches += c->cfg.nspecies + 2;
    const bool open = c->cfg.bc_x == PIC_BC_OPEN;
    const int i0 = open ? 3 : 0, i1 = open ? c->cfg.nx - 4 : c->cfg.nx - 1;
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            cudaError_t e = c->dim == 3 ? launch_rho3<T>(dev_species3<T>(c, s, c->cur[s]), c->n_upper[s], mesh3<T>(c),
                                                          static_cast<T *>(c->rho), st)
                                        : launch_rho<T>(dev_species<T>(c, s, c->cur[s]), c->n_upper[s], mesh<T>(c),
                                                        static_cast<T *>(c->rho), st);
            if (e != cudaSuccess) return e;
        }
        if (c->dim == 3)
            return launch_gauss3<T>(mesh3<T>(c), static_cast<const T *>(c->rho), static_cast<const T *>(c->rho_bg),
                                    c->dx, c->dy, c->dz, i0, i1, c->partials, c->result, st);
        return launch_gauss<T>(mesh<T>(c), static_cast<const T *>(c->rho), static_cast<const T *>(c->rho_bg),
                               c->dx, c->dy, i0, i1, c->partials, c->result, st);
    }));
    double r[2];
    CK(cudaMemcpyAsync(r, c->result, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double cnt = (double)(i1 - i0 + 1) * c->bnd_n;
    out[0] = r[0];
    out[1] = std::sqrt(r[1] / cnt);
    return PIC_OK;
}

pic_status_t pic_shift_window(void *ctx, int ncells, const pic_particles_t *inject, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (c->cfg.bc_x != PIC_BC_OPEN) return fail(c, PIC_ERR_ARG, "the moving window needs open x boundaries");
    if (ncells < 1 || ncells > c->cfg.nx - 8) return fail(c, PIC_ERR_ARG, "ncells must be in [1, nx - 8]");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    ensure_live(c);
    pic_status_t r = free_spent(c, st);
    if (r != PIC_OK) return r;
    if (inject) {
        // species that take the compact path append after their slots: the
        // plasma must fit the capacity (checked before anything changes)
        for (int s = 0; s < c->cfg.nspecies; ++s) {
            if (inject[s].n < 0) return fail(c, PIC_ERR_ARG, "negative injection count");
            const bool rotate = c->dim == 3 && c->sp_binned[s] && ncells % c->tg3.TX == 0;
            if (rotate || inject[s].n == 0) continue;
            if (c->sp_binned[s]) {
                r = sort_species(c, s, st, true);
                if (r != PIC_OK) return r;
            }
            int32_t cur = 0;
            r = read_count(c, s, st, &cur);
            if (r != PIC_OK) return r;
            if (cur + inject[s].n > c->cfg.sp[s].capacity)
                return fail(c, PIC_ERR_OVERFLOW, "injection exceeds the capacity");
        }
    }
    Slab b;
    if (inject) {
        r = stage_slab(c, inject, &b, st);
        if (r != PIC_OK) return r;
    }
    r = window_move(c, ncells, inject ? &b : nullptr, st);
    if (b.mem) {
        cudaStreamSynchronize(st);
        cudaFree(b.mem);
    }
    if (r != PIC_OK) return r;
    return check_flags(c, st);
}

pic_status_t pic_set_window(void *ctx, int ncells, int64_t start_step, double speed) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (ncells == 0) {
        c->w_ncells = 0;
        return PIC_OK;
    }
    if (c->cfg.bc_x != PIC_BC_OPEN) return fail(c, PIC_ERR_ARG, "the moving window needs open x boundaries");
    if (ncells < 1 || ncells > c->cfg.nx - 8) return fail(c, PIC_ERR_ARG, "ncells must be 0 or in [1, nx - 8]");
    if (!(speed > 0.0) || !std::isfinite(speed)) return fail(c, PIC_ERR_ARG, "speed must be positive and finite");
    ensure_live(c);
    c->w_ncells = ncells;
    c->w_start = start_step;
    c->w_speed = speed;
    c->w_window0 = c->window;
    return PIC_OK;
}

pic_status_t pic_stage_injection(void *ctx, const pic_particles_t *inject, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!inject) return fail(c, PIC_ERR_ARG, "null injection");
    if (c->cfg.bc_x != PIC_BC_OPEN) return fail(c, PIC_ERR_ARG, "the moving window needs open x boundaries");
    cudaStream_t st = S(stream);
    pic_status_t r = free_spent(c, st);
    if (r != PIC_OK) return r;
    Slab b;
    r = stage_slab(c, inject, &b, st);
    if (r != PIC_OK) return r;
    c->inj_queue.push_back(b);
    return PIC_OK;
}

pic_status_t pic_get_layout(void *ctx, int s, int *binned) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !binned) return fail(c, PIC_ERR_ARG, "null argument");
    if (s < 0 || s >= c->cfg.nspecies) return fail(c, PIC_ERR_ARG, "species out of range");
    *binned = c->sp_binned[s] ? 1 : 0;
    return PIC_OK;
}

pic_status_t pic_staged_injections(void *ctx, int64_t *count) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !count) return fail(c, PIC_ERR_ARG, "null argument");
    *count = (int64_t)c->inj_queue.size();
    return PIC_OK;
}

pic_status_t pic_buffer_sizes(void *ctx, int64_t *ld, int64_t *plane, int *real_bytes,
                              int64_t capacity[PIC_MAX_SPECIES]) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !ld || !plane || !real_bytes || !capacity) return fail(c, PIC_ERR_ARG, "null argument");
    *ld = c->ld;
    *plane = (int64_t)c->plane;
    *real_bytes = c->rb;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) capacity[s] = s < c->cfg.nspecies ? c->cfg.sp[s].capacity : 0;
    return PIC_OK;
}

pic_status_t pic_bind_buffers(void *ctx, const pic_buffers_t *b, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !b) return fail(c, PIC_ERR_ARG, "null argument");
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    // (slot in the context, caller's array, bytes)
    struct Swap {
        void **own;
        void *mine;
        size_t bytes;
    };
    std::vector<Swap> sw, all;  // the arrays replaced; every array slot of the context
    const size_t rb = c->rb;
    auto add = [&](void **own, void *mine, size_t bytes) {
        all.push_back(Swap{own, mine, bytes});
        if (mine) sw.push_back(Swap{own, mine, bytes});
    };
    add(&c->EB, b->eb, 6 * c->plane * rb);
    add(&c->J, b->j, 3 * c->plane * rb);
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        const size_t cap = (size_t)c->cfg.sp[s].capacity;
        for (int q = 0; q < 2; ++q) {
            const pic_particle_buffer_t &u = b->sp[s][q];
            SpeciesBuf &B = c->buf[s][q];
            add(reinterpret_cast<void **>(&B.cell), u.cell, cap * sizeof(uint32_t));
            void *rec[9] = {u.ox, u.oy, u.ux, u.uy, u.uz, u.sx, u.sy, u.sz, u.w};
            for (int k = 0; k < 9; ++k) add(&B.f[k], rec[k], cap * rb);
            if (c->dim == 3) add(&B.oz, u.oz, cap * rb);
            add(reinterpret_cast<void **>(&B.id), u.id, cap * sizeof(int32_t));
        }
    }
    {
        // after the bind no two arrays of the context may share a byte
        std::vector<std::pair<uintptr_t, uintptr_t>> iv;
        for (const Swap &w : all) {
            const uintptr_t p = reinterpret_cast<uintptr_t>(w.mine ? w.mine : *w.own);
            if (p && w.bytes) iv.emplace_back(p, p + w.bytes);
        }
        std::sort(iv.begin(), iv.end());
        for (size_t k = 1; k < iv.size(); ++k)
            if (iv[k].first < iv[k - 1].second) return fail(c, PIC_ERR_ARG, "bound arrays overlap");
    }
    for (const Swap &w : sw) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, w.mine) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PIC_ERR_ARG, "bound array: not a CUDA pointer");
        }
        const bool dev = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        if (!dev || a.device != c->device)
            return fail(c, PIC_ERR_ARG, "bound array: not memory of the context's device");
        if (reinterpret_cast<uintptr_t>(w.mine) % 16 != 0)
            return fail(c, PIC_ERR_ARG, "bound array: not 16-byte aligned");
    }
    if (sw.empty()) return PIC_OK;
    for (const Swap &w : sw) CK(cudaMemcpyAsync(w.mine, *w.own, w.bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    for (const Swap &w : sw) {
        free_own(c, *w.own);
        *w.own = w.mine;
        c->borrowed.push_back(w.mine);
    }
    drop_step_graphs(c);
    return make_tensor_map(c);
}

pic_status_t pic_current_buffer(void *ctx, int s, int *which) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !which) return fail(c, PIC_ERR_ARG, "null argument");
    if (s < 0 || s >= c->cfg.nspecies) return fail(c, PIC_ERR_ARG, "species out of range");
    *which = c->cur[s];
    return PIC_OK;
}

pic_status_t pic_get_window(void *ctx, int64_t *offset) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !offset) return fail(c, PIC_ERR_ARG, "null argument");
    *offset = c->window;
    return PIC_OK;
}

pic_status_t pic_sync(void *ctx, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    return check_flags(c, S(stream));
}

pic_status_t pic_launch_count(void *ctx, int64_t *count) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c || !count) return fail(c, PIC_ERR_ARG, "null argument");
    *count = c->launches;
    return PIC_OK;
}

const char *pic_last_error(void *ctx) {
    Ctx *c = static_cast<Ctx *>(ctx);
    return c ? c->last_error.c_str() : g_create_error.c_str();
}

}  // extern "C"


// ===========================================================================
// Batches of independent 2D3V runs (parameter scans: density, a0, mesh size,
// particles per cell, run length).  Each run keeps its own context (state,
// buffers, tile arrays); a batch step is one launch of the persistent fused
// kernel over the (run, tile) items of every active run, the batched field
// update over every (run, row), and a step-counter advance.  Sort-free
// stretches of steps are captured once in a CUDA graph (one per buffer
// parity) and replayed; the tile sorts run per run between replays.
// ===========================================================================
namespace {

struct Batch {
    std::vector<Ctx *> runs;
    std::vector<long long> todo;   // steps each run still has to take
    std::vector<long long> done;   // steps taken in this batch
    int tx = 16, ty = 8, sort_every = 32, since_sort = 0, parity = -1;
    bool prepared = false;
    StepParams<float> *params[2] = {};
    CUtensorMap *tmaps = nullptr;
    BatchField<float> *fields = nullptr;
    double *laser = nullptr;
    int2 *work = nullptr, *rows = nullptr;
    int nwork = 0, nrows = 0, ctas = 0;
    long long *step = nullptr, *nsteps = nullptr;
    int *counter = nullptr;
    long long launches = 0;  // kernels the batch launched (graph nodes included, run contexts' own not)
    std::vector<std::pair<int, cudaGraphExec_t>> graphs[2];  // (steps, graph) per parity
    std::string last_error;
};

pic_status_t bfail(Batch *b, pic_status_t s, const std::string &msg) {
    if (b) b->last_error = msg;
    else g_create_error = msg;
    return s;
}

#define BCK(...)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (__VA_ARGS__);                                                         \
        if (e_ != cudaSuccess)                                                                  \
            return bfail(b, PIC_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void drop_graphs(Batch *b) {
    for (auto &v : b->graphs)
        for (auto &g : v) cudaGraphExecDestroy(g.second);
    b->graphs[0].clear();
    b->graphs[1].clear();
}

void free_tables(Batch *b) {
    drop_graphs(b);
    cudaFree(b->params[0]);
    cudaFree(b->params[1]);
    cudaFree(b->tmaps);
    cudaFree(b->fields);
    cudaFree(b->laser);
    cudaFree(b->work);
    cudaFree(b->rows);
    cudaFree(b->step);
    cudaFree(b->nsteps);
    cudaFree(b->counter);
    b->params[0] = b->params[1] = nullptr;
    b->tmaps = nullptr;
    b->fields = nullptr;
    b->laser = nullptr;
    b->work = b->rows = nullptr;
    b->step = b->nsteps = nullptr;
    b->counter = nullptr;
    b->prepared = false;
}

// every species of every run in buffer `parity`
pic_status_t align_parity(Batch *b, cudaStream_t st) {
    if (b->parity < 0) b->parity = b->runs[0]->cur[0];
    for (Ctx *c : b->runs)
        for (int s = 0; s < c->cfg.nspecies; ++s)
            if (c->cur[s] != b->parity) {
                pic_status_t r = sort_species(c, s, st);
                if (r != PIC_OK) return bfail(b, r, c->last_error);
            }
    return PIC_OK;
}

// device tables of the batch: per-run parameters for both parities, tensor
// maps, field data with laser tables, work items (largest runs first), rows
pic_status_t prepare(Batch *b, cudaStream_t st) {
    free_tables(b);
    const int n = (int)b->runs.size();
    std::vector<StepParams<float>> P[2];
    std::vector<CUtensorMap> tm(n);
    std::vector<BatchField<float>> F(n);
    std::vector<long long> step0(n), end(n);
    std::vector<size_t> laser_off(n);
    size_t laser_total = 0;
    std::vector<long long> left(n);
    for (int r = 0; r < n; ++r) {
        left[r] = b->todo[r] - b->done[r];
        laser_off[r] = laser_total;
        laser_total += 2 * (size_t)std::max<long long>(left[r], 1);
    }
    std::vector<double> lt(laser_total, 0.0);
    std::vector<std::pair<long long, int>> order;
    for (int r = 0; r < n; ++r) {
        Ctx *c = b->runs[r];
        for (int p = 0; p < 2; ++p) {
            StepParams<float> q = step_params<float>(c);
            for (int s = 0; s < q.nsp; ++s) q.sp[s] = dev_species<float>(c, s, p);
            q.diag = DiagParams{};
            P[p].push_back(q);
        }
        tm[r] = c->tmapEB;
        F[r].m = mesh<float>(c);
        F[r].bnd = static_cast<float *>(c->bnd);
        F[r].prof = c->laser_prof;
        F[r].step0 = c->step;
        F[r].r = c->dt / c->dx;
        F[r].q = c->dt / c->dy;
        step0[r] = c->step;
        end[r] = c->step + left[r];
        const LaserParams L = laser(c);
        for (long long k = 0; k < left[r]; ++k)
            laser_time_factors(L, ((double)(c->step + k) + 0.5) * c->dt, &lt[laser_off[r] + 2 * k],
                               &lt[laser_off[r] + 2 * k + 1]);
        order.push_back({-(long long)c->ntiles * left[r], r});
    }
    std::sort(order.begin(), order.end());
    std::vector<int2> work, rows;
    for (auto &o : order) {
        Ctx *c = b->runs[o.second];
        for (int t = 0; t < c->ntiles; ++t) work.push_back(make_int2(o.second, t));
        for (int j = 0; j < c->cfg.ny; ++j) rows.push_back(make_int2(o.second, j));
    }
    b->nwork = (int)work.size();
    b->nrows = (int)rows.size();
    BCK(cudaMalloc(&b->laser, lt.size() * sizeof(double)));
    BCK(cudaMemcpyAsync(b->laser, lt.data(), lt.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    for (int r = 0; r < n; ++r) F[r].laser = b->laser + laser_off[r];
    for (int p = 0; p < 2; ++p) {
        BCK(cudaMalloc(&b->params[p], n * sizeof(StepParams<float>)));
        BCK(cudaMemcpyAsync(b->params[p], P[p].data(), n * sizeof(StepParams<float>), cudaMemcpyHostToDevice, st));
    }
    BCK(cudaMalloc(&b->tmaps, n * sizeof(CUtensorMap)));
    BCK(cudaMemcpyAsync(b->tmaps, tm.data(), n * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
    BCK(cudaMalloc(&b->fields, n * sizeof(BatchField<float>)));
    BCK(cudaMemcpyAsync(b->fields, F.data(), n * sizeof(BatchField<float>), cudaMemcpyHostToDevice, st));
    BCK(cudaMalloc(&b->work, work.size() * sizeof(int2)));
    BCK(cudaMemcpyAsync(b->work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    BCK(cudaMalloc(&b->rows, rows.size() * sizeof(int2)));
    BCK(cudaMemcpyAsync(b->rows, rows.data(), rows.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    BCK(cudaMalloc(&b->step, n * sizeof(long long)));
    BCK(cudaMemcpyAsync(b->step, step0.data(), n * sizeof(long long), cudaMemcpyHostToDevice, st));
    BCK(cudaMalloc(&b->nsteps, n * sizeof(long long)));
    BCK(cudaMemcpyAsync(b->nsteps, end.data(), n * sizeof(long long), cudaMemcpyHostToDevice, st));
    BCK(cudaMalloc(&b->counter, sizeof(int)));
    BCK(cudaMemsetAsync(b->counter, 0, sizeof(int), st));
    BCK(cudaStreamSynchronize(st));
    int dev = 0, sms = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    b->ctas = sms * fused_batch_occupancy(b->tx, b->ty);
    b->prepared = true;
    return PIC_OK;
}

// one batch step on the stream (launches only; capturable)
cudaError_t enqueue_step(Batch *b, int parity, cudaStream_t st) {
    BatchFused<float> W{b->params[parity], b->tmaps, b->work, b->nwork, b->counter, b->step, b->nsteps};
    cudaError_t e = launch_step_fused_batch<float>(W, b->tx, b->ty, b->ctas, st);
    if (e != cudaSuccess) return e;
    return launch_field_update_batch<float>(b->fields, b->rows, b->nrows, b->step, b->nsteps, (int)b->runs.size(),
                                            b->counter, st);
}

pic_status_t run_graph(Batch *b, int steps, cudaStream_t st) {
    auto &cache = b->graphs[b->parity];
    cudaGraphExec_t exec = nullptr;
    for (auto &g : cache)
        if (g.first == steps) exec = g.second;
    if (!exec) {
        cudaStream_t cs;
        BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) e = enqueue_step(b, b->parity, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        BCK(e);
        BCK(e2);
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        BCK(e);
        cache.push_back({steps, exec});
    }
    BCK(cudaGraphLaunch(exec, st));
    b->launches += 6LL * steps;  // fused, 2 x B half step, boundary, E step, advance
    return PIC_OK;
}

// up to nsteps batch steps: sort-free stretches as graph replays, tile sorts
// between them (runs still active only)
pic_status_t batch_advance(Batch *b, long long nsteps, cudaStream_t st) {
    const int n = (int)b->runs.size();
    pic_status_t r = align_parity(b, st);
    if (r != PIC_OK) return r;
    if (!b->prepared) {
        r = prepare(b, st);
        if (r != PIC_OK) return r;
    }
    while (nsteps > 0) {
        long long active = 0;
        for (int k = 0; k < n; ++k) active += b->done[k] < b->todo[k];
        if (!active) break;
        const int chunk = (int)std::min<long long>(nsteps, b->sort_every - b->since_sort);
        r = run_graph(b, chunk, st);
        if (r != PIC_OK) return r;
        for (int k = 0; k < n; ++k) {
            const long long take = std::min<long long>(chunk, b->todo[k] - b->done[k]);
            if (take > 0) {
                b->done[k] += take;
                b->runs[k]->step += take;
            }
        }
        nsteps -= chunk;
        b->since_sort += chunk;
        if (b->since_sort >= b->sort_every) {
            const int next = 1 - b->parity;
            for (int k = 0; k < n; ++k) {
                Ctx *c = b->runs[k];
                for (int s = 0; s < c->cfg.nspecies; ++s) {
                    r = sort_species(c, s, st);
                    if (r != PIC_OK) return bfail(b, r, c->last_error);
                }
            }
            b->parity = next;
            b->since_sort = 0;
        }
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status_t pic_batch_create(const pic_config_t *cfgs, int nruns, const int64_t *nsteps, void *stream,
                              void **batch_out) {
    Batch *b = nullptr;
    if (!batch_out || !cfgs || !nsteps || nruns < 1) return bfail(b, PIC_ERR_ARG, "need configs, steps and nruns >= 1");
    *batch_out = nullptr;
    b = new (std::nothrow) Batch();
    if (!b) return bfail(nullptr, PIC_ERR_CUDA, "host allocation failed");
    b->tx = cfgs[0].tile_x > 0 ? cfgs[0].tile_x : 16;
    b->ty = cfgs[0].tile_y > 0 ? cfgs[0].tile_y : 8;
    b->sort_every = cfgs[0].sort_every > 0 ? cfgs[0].sort_every : 32;
    for (int r = 0; r < nruns; ++r) {
        pic_config_t cfg = cfgs[r];
        if ((cfg.dim != 0 && cfg.dim != 2) || (cfg.precision != 0 && cfg.precision != 32) || nsteps[r] < 0) {
            pic_batch_destroy(b);
            return bfail(nullptr, PIC_ERR_ARG, "batch runs must be 2D3V, precision 32, steps >= 0");
        }
        cfg.tile_x = b->tx;
        cfg.tile_y = b->ty;
        void *h = nullptr;
        pic_status_t st = pic_create(&cfg, stream, &h);
        if (st != PIC_OK) {
            const std::string why = "run " + std::to_string(r) + ": " + g_create_error;
            pic_batch_destroy(b);
            return bfail(nullptr, st, why);
        }
        b->runs.push_back(static_cast<Ctx *>(h));
        b->todo.push_back(nsteps[r]);
        b->done.push_back(0);
    }
    *batch_out = b;
    return PIC_OK;
}

void pic_batch_destroy(void *batch) {
    Batch *b = static_cast<Batch *>(batch);
    if (!b) return;
    free_tables(b);
    for (Ctx *c : b->runs) pic_destroy(c);
    delete b;
}

pic_status_t pic_batch_run(void *batch, int r, void **ctx) {
    Batch *b = static_cast<Batch *>(batch);
    if (!b || !ctx || r < 0 || r >= (int)b->runs.size()) return bfail(b, PIC_ERR_ARG, "bad batch or run index");
    b->prepared = false;  // the caller may change the run's state (particles, fields, step)
    *ctx = b->runs[r];
    return PIC_OK;
}

pic_status_t pic_batch_step(void *batch, int64_t nsteps, void *stream) {
    Batch *b = static_cast<Batch *>(batch);
    if (!b) return bfail(nullptr, PIC_ERR_ARG, "null batch");
    if (nsteps < 0) return bfail(b, PIC_ERR_ARG, "negative step count");
    cudaStream_t st = S(stream);
    for (Ctx *c : b->runs)
        if (c->pending_deposit) return bfail(b, PIC_ERR_STATE, "a run has a move waiting for pic_deposit");
    pic_status_t r = batch_advance(b, nsteps, st);
    if (r != PIC_OK) return r;
    for (size_t k = 0; k < b->runs.size(); ++k) {
        r = check_flags(b->runs[k], st);
        if (r != PIC_OK) return bfail(b, r, "run " + std::to_string(k) + ": " + b->runs[k]->last_error);
    }
    return PIC_OK;
}

pic_status_t pic_batch_steps_done(void *batch, int64_t *done) {
    Batch *b = static_cast<Batch *>(batch);
    if (!b || !done) return bfail(b, PIC_ERR_ARG, "null argument");
    for (size_t k = 0; k < b->runs.size(); ++k) done[k] = b->done[k];
    return PIC_OK;
}

pic_status_t pic_batch_tune(void *batch, int probe_steps, const int *tiles, int ntiles, const int *sorts, int nsorts,
                            int *chosen, void *stream) {
    Batch *b = static_cast<Batch *>(batch);
    if (!b) return bfail(nullptr, PIC_ERR_ARG, "null batch");
    if (probe_steps < 1 || !tiles || ntiles < 1 || !sorts || nsorts < 1 || !chosen)
        return bfail(b, PIC_ERR_ARG, "need probe_steps >= 1 and candidate tiles and sort cadences");
    for (int k = 0; k < ntiles; ++k)
        if (!fused_tile_supported(tiles[2 * k], tiles[2 * k + 1])) return bfail(b, PIC_ERR_ARG, "unsupported tile");
    for (int k = 0; k < nsorts; ++k)
        if (sorts[k] < 1) return bfail(b, PIC_ERR_ARG, "sort cadence must be >= 1");
    cudaStream_t st = S(stream);
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    double best = -1.0;
    int bt = 0, bs = 0;
    pic_status_t r = PIC_OK;
    for (int t = 0; t < ntiles && r == PIC_OK; ++t) {
        if (tiles[2 * t] != b->tx || tiles[2 * t + 1] != b->ty) {
            for (Ctx *c : b->runs)
                if ((r = retile(c, tiles[2 * t], tiles[2 * t + 1], st)) != PIC_OK) break;
            if (r != PIC_OK) break;
            b->tx = tiles[2 * t];
            b->ty = tiles[2 * t + 1];
            b->parity = -1;
            b->since_sort = 0;
            free_tables(b);
        }
        for (int q = 0; q < nsorts && r == PIC_OK; ++q) {
            b->sort_every = sorts[q];
            b->since_sort = 0;
            // one sort cycle as warm-up (graph capture), then the probe
            if ((r = batch_advance(b, sorts[q], st)) != PIC_OK) break;
            std::vector<long long> before = b->done;
            long long parts = 0;
            for (Ctx *c : b->runs)
                for (int s = 0; s < c->cfg.nspecies; ++s) parts += c->cfg.sp[s].mobile ? c->n_upper[s] : 0;
            cudaEventRecord(e0, st);
            if ((r = batch_advance(b, probe_steps, st)) != PIC_OK) break;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            long long taken = 0;
            for (size_t k = 0; k < b->runs.size(); ++k) taken += b->done[k] - before[k];
            const double rate = taken > 0 && ms > 0 ? (double)parts * probe_steps / ms : 0.0;
            if (rate > best) {
                best = rate;
                bt = t;
                bs = q;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != PIC_OK) return r;
    if (tiles[2 * bt] != b->tx || tiles[2 * bt + 1] != b->ty) {
        for (Ctx *c : b->runs)
            if ((r = retile(c, tiles[2 * bt], tiles[2 * bt + 1], st)) != PIC_OK) return bfail(b, r, c->last_error);
        b->tx = tiles[2 * bt];
        b->ty = tiles[2 * bt + 1];
        b->parity = -1;
        free_tables(b);
    }
    b->sort_every = sorts[bs];
    b->since_sort = 0;
    chosen[0] = b->tx;
    chosen[1] = b->ty;
    chosen[2] = b->sort_every;
    return PIC_OK;
}

pic_status_t pic_batch_launch_count(void *batch, int64_t *count) {
    Batch *b = static_cast<Batch *>(batch);
    if (!b || !count) return bfail(b, PIC_ERR_ARG, "null argument");
    long long n = b->launches;
    for (Ctx *c : b->runs) n += c->launches;  // the runs' own: uploads, sorts, reductions
    *count = n;
    return PIC_OK;
}

const char *pic_batch_last_error(void *batch) {
    Batch *b = static_cast<Batch *>(batch);
    return b ? b->last_error.c_str() : g_create_error.c_str();
}

}  // extern "C"


// ===========================================================================
// Adjoint of the 2D3V step: the gradient of a loss on the final particle
// state (the energy-weighted polarization above a cut, the beam quality the
// paper's runs look at) with respect to the initial particle state, the
// particle weights and the laser amplitude.  The forward pass runs the fused
// kernel (FP32; the split kernels in FP64) without tile sorts (slots keep
// their particles) and keeps a
// checkpoint every K steps; the backward pass recomputes each stretch of K
// steps from its checkpoint, storing every step's state, and runs the adjoint
// kernels back through it.
// ===========================================================================
namespace {

// one stored state: every species' cell words and 8 reals per slot
// (ox oy ux uy uz sx sy sz), then E, B
struct Snap {
    size_t bytes = 0;
    size_t off_cell[PIC_MAX_SPECIES] = {}, off_real[PIC_MAX_SPECIES] = {}, off_eb = 0;
};

Snap snap_layout(Ctx *c, const long long *n) {
    Snap L;
    size_t o = 0;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        L.off_cell[s] = o;
        o = al(o + (size_t)n[s] * sizeof(uint32_t));
        L.off_real[s] = o;
        o = al(o + (size_t)n[s] * 8 * c->rb);
    }
    L.off_eb = o;
    o = al(o + 6 * c->plane * c->rb);
    L.bytes = o;
    return L;
}

static const int kSnapField[8] = {0, 1, 2, 3, 4, 5, 6, 7};  // SpeciesBuf::f index of each stored real

pic_status_t snap_copy(Ctx *c, const Snap &L, const long long *n, char *snap, bool save, cudaStream_t st) {
    for (int s = 0; s < c->cfg.nspecies; ++s) {
        SpeciesBuf &B = c->buf[s][c->cur[s]];
        char *cs = snap + L.off_cell[s];
        if (n[s] == 0) continue;
        if (save) CK(cudaMemcpyAsync(cs, B.cell, n[s] * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        else CK(cudaMemcpyAsync(B.cell, cs, n[s] * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < 8; ++k) {
            char *r = snap + L.off_real[s] + (size_t)k * n[s] * c->rb;
            if (save) CK(cudaMemcpyAsync(r, B.f[kSnapField[k]], n[s] * c->rb, cudaMemcpyDeviceToDevice, st));
            else CK(cudaMemcpyAsync(B.f[kSnapField[k]], r, n[s] * c->rb, cudaMemcpyDeviceToDevice, st));
        }
    }
    char *eb = snap + L.off_eb;
    if (save) CK(cudaMemcpyAsync(eb, c->EB, 6 * c->plane * c->rb, cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemcpyAsync(c->EB, eb, 6 * c->plane * c->rb, cudaMemcpyDeviceToDevice, st));
    return PIC_OK;
}

template <typename R>
AdjParticles<R> adj_particles(Ctx *c, int s, const Snap &L, const long long *n, const char *snap) {
    AdjParticles<R> P{};
    P.n = n[s];
    P.cell = reinterpret_cast<const uint32_t *>(snap + L.off_cell[s]);
    const R *r = reinterpret_cast<const R *>(snap + L.off_real[s]);
    P.ox = r;
    P.oy = r + n[s];
    P.ux = r + 2 * n[s];
    P.uy = r + 3 * n[s];
    P.uz = r + 4 * n[s];
    P.sx = r + 5 * n[s];
    P.sy = r + 6 * n[s];
    P.sz = r + 7 * n[s];
    P.w = static_cast<const R *>(c->buf[s][c->cur[s]].f[8]);
    P.EB = reinterpret_cast<const R *>(snap + L.off_eb);
    const pic_species_t &sp = c->cfg.sp[s];
    P.qm = (R)(sp.q / sp.m);
    P.q = (R)sp.q;
    P.a = (R)sp.a;
    R **lam[9] = {&P.lx, &P.ly, &P.lux, &P.luy, &P.luz, &P.lsx, &P.lsy, &P.lsz, &P.lw};
    for (int k = 0; k < 9; ++k) *lam[k] = static_cast<R *>(c->adj_lam[s][k]);
    return P;
}

template <typename R>
AdjMesh<R> adj_mesh(Ctx *c, void *LEB, void *LJ, void *Lbnd) {
    const MeshParams<R> m = mesh<R>(c);
    AdjMesh<R> A{};
    A.nx = m.nx;
    A.ny = m.ny;
    A.ld = m.ld;
    A.bc_x = m.bc_x;
    A.plane = m.plane;
    A.dt = m.dt;
    A.dt_dx = m.dt_dx;
    A.dt_dy = m.dt_dy;
    A.dx_dt = m.dx_dt;
    A.dy_dt = m.dy_dt;
    A.r = c->dt / c->dx;
    A.q = c->dt / c->dy;
    A.LEB = static_cast<R *>(LEB);
    A.LJ = static_cast<R *>(LJ);
    A.Lbnd = static_cast<R *>(Lbnd);
    return A;
}

// The adjoint's forward step, without tile sorts (every particle keeps its
// slot) and without in-step diagnostics: the fused kernel in FP32; in FP64 the
// split kernels, which run faster than the FP64 fused kernel once the
// particles have drifted out of their tiles.
pic_status_t forward_adjoint_step(Ctx *c, cudaStream_t st) {
    pic_status_t r = PIC_OK;
    if (c->rb == 8) {
        r = pic_gather_push_spin(c, st);
        if (r == PIC_OK) r = pic_deposit(c, st);
    } else {
        const int diag_every = c->diag_every;
        c->diag_every = 0;
        r = pic_push_deposit(c, st);
        c->diag_every = diag_every;
    }
    if (r == PIC_OK) r = pic_field_update(c, st);
    return r;
}

pic_status_t check_loss(Ctx *c, const pic_loss_t *loss) {
    if (!loss) return fail(c, PIC_ERR_ARG, "null loss");
    if (loss->species < 0 || loss->species >= c->cfg.nspecies) return fail(c, PIC_ERR_ARG, "bad loss species");
    if (loss->axis < 0 || loss->axis > 2) return fail(c, PIC_ERR_ARG, "loss axis must be 0, 1 or 2");
    if (!(loss->e_width_mev > 0)) return fail(c, PIC_ERR_ARG, "loss width must be > 0");
    return PIC_OK;
}

LossParams loss_params(Ctx *c, const pic_loss_t *loss) {
    return LossParams{c->cfg.sp[loss->species].m * kMec2Mev, loss->e_cut_mev, loss->e_width_mev, loss->axis};
}

}  // namespace

extern "C" {

pic_status_t pic_loss(void *ctx, const pic_loss_t *loss, double *value, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (!value) return fail(c, PIC_ERR_ARG, "null output");
    pic_status_t r = check_loss(c, loss);
    if (r != PIC_OK) return r;
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    const int s = loss->species;
    int32_t n = 0;
    if ((r = read_count(c, s, st, &n)) != PIC_OK) return r;
    CK(with_real(c, [&](auto z) {
        using T = decltype(z);
        AdjParticles<T> P{};
        const DevSpecies<T> d = dev_species<T>(c, s, c->cur[s]);
        P.n = n;
        P.cell = d.cell;
        P.ox = d.ox; P.oy = d.oy; P.ux = d.ux; P.uy = d.uy; P.uz = d.uz; P.sx = d.sx; P.sy = d.sy; P.sz = d.sz;
        P.w = d.w;
        return launch_loss<T>(P, loss_params(c, loss), c->result, false, st);
    }));
    double h[2];
    CK(cudaMemcpyAsync(h, c->result, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *value = h[0] > 0 ? h[1] / h[0] : 0.0;
    return check_flags(c, st);
}

pic_status_t pic_adjoint(void *ctx, int nsteps, int checkpoint_every, const pic_loss_t *loss, double *loss_value,
                         double *dloss_da0, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (c->dim != 2) return fail(c, PIC_ERR_ARG, "the adjoint is built for 2D3V");
    if (nsteps < 1 || checkpoint_every < 1) return fail(c, PIC_ERR_ARG, "need nsteps >= 1 and checkpoint_every >= 1");
    pic_status_t r = check_loss(c, loss);
    if (r != PIC_OK) return r;
    if (c->pending_deposit) return fail(c, PIC_ERR_STATE, "a move is waiting for pic_deposit");
    cudaStream_t st = S(stream);
    const int nsp = c->cfg.nspecies, K = checkpoint_every;
    long long n[PIC_MAX_SPECIES] = {};
    for (int s = 0; s < nsp; ++s) {
        int32_t v = 0;
        if ((r = read_count(c, s, st, &v)) != PIC_OK) return r;
        n[s] = v;
    }
    const Snap L = snap_layout(c, n);
    const int nck = (nsteps + K - 1) / K;
    // checkpoints, two stretches (the backward of one stretch reads one while
    // the recompute of the stretch before it fills the other), the final state
    const size_t nsnap = (size_t)nck + 2 * (size_t)K + 1;
    char *store = nullptr;
    void *LEB = nullptr, *LJ = nullptr, *Lbnd = nullptr;
    double *sums = nullptr, *dla0 = nullptr;
    cudaStream_t s2 = nullptr;  // the recompute stream
    cudaEvent_t ready[2] = {}, freed[2] = {};
    auto cleanup = [&]() {
        if (s2) {
            cudaStreamSynchronize(s2);
            cudaStreamDestroy(s2);
        }
        for (int b = 0; b < 2; ++b) {
            if (ready[b]) cudaEventDestroy(ready[b]);
            if (freed[b]) cudaEventDestroy(freed[b]);
        }
        cudaFree(store);
        cudaFree(LEB);
        cudaFree(LJ);
        cudaFree(Lbnd);
        cudaFree(sums);
        cudaFree(dla0);
    };
#define ACK(...)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (__VA_ARGS__);                                                                \
        if (e_ != cudaSuccess) {                                                                       \
            cleanup();                                                                                 \
            return fail(c, PIC_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));   \
        }                                                                                              \
    } while (0)
#define ARET(expr)                                                                                     \
    do {                                                                                               \
        pic_status_t r_ = (expr);                                                                      \
        if (r_ != PIC_OK) {                                                                            \
            cleanup();                                                                                 \
            return r_;                                                                                 \
        }                                                                                              \
    } while (0)
    ACK(cudaMalloc(&store, nsnap * L.bytes));
    ACK(cudaMalloc(&LEB, 6 * c->plane * c->rb));
    ACK(cudaMalloc(&LJ, 3 * c->plane * c->rb));
    ACK(cudaMalloc(&Lbnd, 2 * (size_t)c->cfg.ny * c->rb));
    ACK(cudaMalloc(&sums, 2 * sizeof(double)));
    ACK(cudaMalloc(&dla0, sizeof(double)));
    for (int s = 0; s < nsp; ++s) {
        for (int k = 0; k < 9; ++k) {
            cudaFree(c->adj_lam[s][k]);
            c->adj_lam[s][k] = nullptr;
            ACK(cudaMalloc(&c->adj_lam[s][k], (size_t)n[s] * c->rb + 16));
            ACK(cudaMemsetAsync(c->adj_lam[s][k], 0, (size_t)n[s] * c->rb + 16, st));
        }
        cudaFree(c->adj_cell0[s]);
        c->adj_cell0[s] = nullptr;
        ACK(cudaMalloc(&c->adj_cell0[s], (size_t)n[s] * sizeof(uint32_t) + 16));
        if (n[s]) ACK(cudaMemcpyAsync(c->adj_cell0[s], c->buf[s][c->cur[s]].cell, n[s] * sizeof(uint32_t),
                                      cudaMemcpyDeviceToDevice, st));
        c->adj_n[s] = n[s];
    }
    auto snap = [&](size_t k) { return store + k * L.bytes; };
    auto stretch = [&](int b, int j) { return snap((size_t)nck + (size_t)b * K + j); };
    char *final_state = snap((size_t)nck + 2 * (size_t)K);
    ACK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        ACK(cudaEventCreateWithFlags(&ready[b], cudaEventDisableTiming));
        ACK(cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming));
    }
    const long long step0 = c->step;
    // forward with checkpoints; the states of the last stretch are kept as
    // they pass (its backward comes first and needs no recompute)
    const int klast = (nck - 1) * K;
    for (int k = 0; k < nsteps; ++k) {
        if (k % K == 0) ARET(snap_copy(c, L, n, snap(k / K), true, st));
        if (k >= klast) ARET(snap_copy(c, L, n, stretch((nck - 1) & 1, k - klast), true, st));
        ARET(forward_adjoint_step(c, st));
    }
    ARET(snap_copy(c, L, n, final_state, true, st));
    // loss and the lambdas of the final state
    const int ls = loss->species;
    ACK(with_real(c, [&](auto z) {
        using T = decltype(z);
        return launch_loss<T>(adj_particles<T>(c, ls, L, n, final_state), loss_params(c, loss), sums, true, st);
    }));
    double h[2];
    ACK(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
    ACK(cudaMemsetAsync(LEB, 0, 6 * c->plane * c->rb, st));
    ACK(cudaMemsetAsync(LJ, 0, 3 * c->plane * c->rb, st));
    ACK(cudaMemsetAsync(Lbnd, 0, 2 * (size_t)c->cfg.ny * c->rb, st));
    ACK(cudaMemsetAsync(dla0, 0, sizeof(double), st));
    LaserParams unit = laser(c);
    unit.a0 = 1.0;  // time factors per unit a0: the source is linear in a0
    // backward, one stretch at a time.  The recompute of stretch i - 1 (from
    // its checkpoint, in the context's buffers, on stream s2) and the backward
    // of stretch i (from stored states and the lambda buffers, on st) touch
    // disjoint memory, so they run at the same time; events order each
    // stretch buffer's fill before its backward and its backward before the
    // next fill.
    ACK(cudaEventRecord(freed[0], st));  // the forward pass above, done on st
    ACK(cudaStreamWaitEvent(s2, freed[0], 0));
    auto recompute = [&](int i) -> pic_status_t {
        const int b = i & 1, k0 = i * K, k1 = std::min(nsteps, k0 + K);
        pic_status_t q = snap_copy(c, L, n, snap(i), false, s2);
        c->step = step0 + k0;
        for (int k = k0; k < k1 && q == PIC_OK; ++k) {
            q = snap_copy(c, L, n, stretch(b, k - k0), true, s2);
            if (q == PIC_OK && k + 1 < k1) q = forward_adjoint_step(c, s2);
        }
        if (q == PIC_OK && cudaEventRecord(ready[b], s2) != cudaSuccess)
            q = fail(c, PIC_ERR_CUDA, "adjoint: event record failed");
        return q;
    };
    ACK(cudaEventRecord(ready[(nck - 1) & 1], st));
    for (int i = nck - 1; i >= 0; --i) {
        const int b = i & 1, k0 = i * K, k1 = std::min(nsteps, k0 + K);
        ACK(cudaStreamWaitEvent(st, ready[b], 0));
        if (i > 0) {
            // stretch i - 1 goes into the other buffer once its last reader
            // (the backward of stretch i + 1) is done
            if (i + 1 < nck) ACK(cudaStreamWaitEvent(s2, freed[(i + 1) & 1], 0));
            ARET(recompute(i - 1));
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const char *state = stretch(b, k - k0);
            double phz = 0.0, phy = 0.0;
            laser_time_factors(unit, ((double)(step0 + k) + 0.5) * c->dt, &phz, &phy);
            ACK(with_real(c, [&](auto z) -> cudaError_t {
                using T = decltype(z);
                const AdjMesh<T> A = adj_mesh<T>(c, LEB, LJ, Lbnd);
                cudaError_t e = launch_adjoint_fields<T>(A, c->laser_prof, phz, phy, dla0, st);
                for (int s = 0; s < nsp && e == cudaSuccess; ++s)
                    if (c->cfg.sp[s].mobile) e = launch_adjoint_particles<T>(A, adj_particles<T>(c, s, L, n, state), st);
                return e;
            }));
            c->launches += 4 + nsp;
        }
        ACK(cudaEventRecord(freed[b], st));
    }
    // the context ends in the final forward state (after the last recompute)
    ACK(cudaEventRecord(ready[0], s2));
    ACK(cudaStreamWaitEvent(st, ready[0], 0));
    ARET(snap_copy(c, L, n, final_state, false, st));
    c->step = step0 + nsteps;
    double g = 0.0;
    ACK(cudaMemcpyAsync(&g, dla0, sizeof(double), cudaMemcpyDeviceToHost, st));
    ACK(cudaStreamSynchronize(st));
    cleanup();
#undef ACK
#undef ARET
    if (loss_value) *loss_value = h[0] > 0 ? h[1] / h[0] : 0.0;
    if (dloss_da0) *dloss_da0 = g;
    return check_flags(c, st);
}

pic_status_t pic_adjoint_particle_grads(void *ctx, int s, pic_particles_f64_t *out, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (!c) return fail(nullptr, PIC_ERR_ARG, "null context");
    if (s < 0 || s >= c->cfg.nspecies || !out) return fail(c, PIC_ERR_ARG, "bad species or output");
    if (!c->adj_lam[s][0]) return fail(c, PIC_ERR_STATE, "no adjoint has run");
    const long long n = c->adj_n[s];
    if (out->n < n) return fail(c, PIC_ERR_ARG, "output arrays too small");
    out->n = n;
    if (!n) return PIC_OK;
    double *dst[9] = {out->ox, out->oy, out->ux, out->uy, out->uz, out->sx, out->sy, out->sz, out->w};
    for (int k = 0; k < 9; ++k)
        if (!dst[k]) return fail(c, PIC_ERR_ARG, "null output array");
    if (!out->ix || !out->iy || !out->id) return fail(c, PIC_ERR_ARG, "null output array");
    cudaStream_t st = S(stream);
    for (int k = 0; k < 9; ++k) {
        if (c->rb == 8) {
            CK(cudaMemcpyAsync(dst[k], c->adj_lam[s][k], n * sizeof(double), cudaMemcpyDeviceToHost, st));
        } else {
            CK(launch_convert<float, double>(static_cast<const float *>(c->adj_lam[s][k]),
                                             static_cast<double *>(c->stage), n, st));
            CK(cudaMemcpyAsync(dst[k], c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
    }
    int32_t *dix = c->scratch_i32, *diy = c->scratch_i32 + c->cfg.sp[s].capacity;
    CK(launch_unpack_cells(c->adj_cell0[s], dix, diy, (int)n, st));
    CK(cudaMemcpyAsync(out->ix, dix, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out->iy, diy, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out->id, c->buf[s][c->cur[s]].id, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return PIC_OK;
}

}  // extern "C"
