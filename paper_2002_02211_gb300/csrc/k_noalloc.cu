// k_noalloc.cu -- pic_moments_noalloc: the Eq. (4) moments reduction over
// particle arrays the caller already holds on the device, run without any
// device allocation.
//
// Some callers cannot let a library allocate: code recording a CUDA graph or
// running inside a stream capture, where cudaMalloc is not allowed; callers
// whose device memory all comes from their own pool and who must not have a
// library reserve memory behind it; and latency-critical loops, where
// cudaMalloc's implicit device synchronisation would stall other streams.
// For them the per-block partial sums live in the fixed file-scope array
// below, loaded with the library and kept by every GPU that loads it until
// the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "pic.h"
#include "pic_kernels.h"

namespace {

constexpr int kMaxDevices = 128;
// scratch layout (doubles): [0, 6 * RB) per-block partials, then 8 result
// slots, then one slot whose first 4 bytes hold the particle count
constexpr int kPartials = 6 * 608;
constexpr int kResult = kPartials;
constexpr int kCount = kPartials + 8;
constexpr int kScratchDoubles = kPartials + 16;

static __device__ __align__(256) double g_moments_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is only a stand-in and must
// never reach a kernel).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_moments_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void k_store_count(int32_t *dst, int32_t n) { *dst = n; }

__global__ void k_moments_out(const double *r, pic_moments_t *out) {
    const double sw = r[0];
    pic_moments_t m;
    for (int k = 0; k < 3; ++k) m.P[k] = sw > 0 ? r[1 + k] / sw : 0.0;
    m.sum_w = sw;
    m.count = r[5];
    m.ekin_mean = sw > 0 ? r[4] / sw : 0.0;
    m.ekin_var = sw > 0 ? r[6] / sw : 0.0;
    *out = m;
}

}  // namespace

extern "C" pic_status_t pic_moments_noalloc(int64_t n, const uint32_t *cell, const float *ux,
                                            const float *uy, const float *uz, const float *sx,
                                            const float *sy, const float *sz, const float *w,
                                            double mass_me, double emin_mev, double emax_mev,
                                            pic_moments_t *out_dev, void *stream) {
    if (n < 0 || n > PIC_NOALLOC_MAX_PARTICLES) {
        set_global_error("pic_moments_noalloc: n must be in [0, 2^31 - 1]");
        return PIC_ERR_ARG;
    }
    if (!out_dev || (n > 0 && (!cell || !ux || !uy || !uz || !sx || !sy || !sz || !w))) {
        set_global_error("pic_moments_noalloc: null device pointer");
        return PIC_ERR_ARG;
    }
    if (!(mass_me > 0)) {
        set_global_error("pic_moments_noalloc: mass must be > 0");
        return PIC_ERR_ARG;
    }
    if (reduce_blocks() * 6 > kPartials) {
        set_global_error("pic_moments_noalloc: scratch smaller than the reduction grid");
        return PIC_ERR_CUDA;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_global_error(std::string("pic_moments_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t *count = reinterpret_cast<int32_t *>(scratch + kCount);
    k_store_count<<<1, 1, 0, st>>>(count, (int32_t)n);
    DevSpecies<float> d{};
    d.cell = const_cast<uint32_t *>(cell);
    d.ux = const_cast<float *>(ux);
    d.uy = const_cast<float *>(uy);
    d.uz = const_cast<float *>(uz);
    d.sx = const_cast<float *>(sx);
    d.sy = const_cast<float *>(sy);
    d.sz = const_cast<float *>(sz);
    d.w = const_cast<float *>(w);
    d.n = count;
    const float lo = std::isinf(emin_mev) && emin_mev < 0 ? -INFINITY : (float)emin_mev;
    const float hi = std::isinf(emax_mev) && emax_mev > 0 ? INFINITY : (float)emax_mev;
    e = launch_moments<float>(d, (float)(mass_me * 0.51099895), lo, hi, scratch, scratch + kResult, st);
    if (e == cudaSuccess) {
        k_moments_out<<<1, 1, 0, st>>>(scratch + kResult, out_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("pic_moments_noalloc: launch: ") + cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}
