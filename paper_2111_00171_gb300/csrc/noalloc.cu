// acom_bounds_static: the shell contraction (spectral bounds) with its scratch
// in a fixed, file-scope device array instead of the plan's workspace, for
// callers that must not allocate device memory while they run.
//
// The array holds, for one chunk of patterns, the pattern spectra the
// contraction reads (FP32 frequency-major for FP32 plans, BF16 tensor-core
// tiles for BF16 plans) and ||X||^2.  Host code never touches it by name: the
// first call on a device looks up its device address with
// cudaGetSymbolAddress (that device current) and caches it per device.
#include <cuda.h>

#include <mutex>

#include "acom_internal.cuh"

namespace acom {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;    // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once).
static acom_status static_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "bounds_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(ACOM_ERR_UNSUPPORTED, "bounds_static: device index >= 64");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_error(e, "bounds_static: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ACOM_OK;
}

// Patterns per chunk that fit the array for this plan: a multiple of 64 (the
// tensor-core pattern tile), 0 when not even 64 fit.
static int static_chunk(const acom_plan_s* p) {
    const size_t per = p->precision == ACOM_PREC_BF16
                           ? (size_t)p->F * 2 * p->Spad * 2          // BF16 re, im rows
                           : (size_t)2 * p->F * p->Spad * 4;          // FP32 re, im
    const size_t fits = (kStaticScratchBytes - 4096) / (per + sizeof(float));
    return (int)(fits / 64 * 64);
}

}  // namespace acom

using namespace acom;

extern "C" acom_status acom_bounds_static(acom_plan p, const acom_peaks_csr* peaks, float* dst,
                                          void* cuda_stream) {
    clear_error();
    if (!p || !dst) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    if (!peaks) return set_error(ACOM_ERR_INVALID_ARG, "null peaks");
    if (peaks->n_patterns < 0) return set_error(ACOM_ERR_INVALID_ARG, "n_patterns < 0");
    if (peaks->n_patterns > 0 && (!peaks->row_ptr || !peaks->qx || !peaks->qy || !peaks->I))
        return set_error(ACOM_ERR_INVALID_ARG, "null peak array");
    const int chunk = static_chunk(p);
    if (chunk < 64)
        return set_error(ACOM_ERR_UNSUPPORTED,
                         "bounds_static: the plan's spectra need more than the 32 MiB static "
                         "scratch for 64 patterns (n_phi x shells too large)");
    const int64_t B = peaks->n_patterns;
    if (B == 0) return ACOM_OK;
    void* base = nullptr;
    acom_status s = static_scratch_address(&base);
    if (s != ACOM_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool tc = p->precision == ACOM_PREC_BF16;
    const size_t spec = (size_t)chunk * p->F * p->Spad;
    unsigned char* cur = reinterpret_cast<unsigned char*>(base);
    float* Xr = nullptr;
    float* Xi = nullptr;
    void* XB = nullptr;
    const int PTs = chunk / 64;
    if (tc) {
        XB = cur;
        cur += spec * 2 * 2;
    } else {
        Xr = reinterpret_cast<float*>(cur);
        Xi = Xr + spec;
        cur += spec * 2 * sizeof(float);
    }
    float* xnorm2 = reinterpret_cast<float*>(cur);
    alignas(64) unsigned char map_x[128];
    if (tc) {
        s = make_bf16_map(map_x, XB, (uint64_t)p->F * PTs * 128, (uint64_t)p->Spad);
        if (s != ACOM_OK) return s;
    }
    prof_suppress(true);
    cudaError_t e = cudaMemsetAsync(p->err, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        prof_suppress(false);
        return cuda_error(e, "bounds_static: clearing the error word");
    }
    // row_ptr[0] == 0 (the raster checks the rest of the row pointers)
    launch_check_row0(peaks->row_ptr, p->err, st);
    RasterGeom geo{p->S, p->Spad, p->N, p->F, (float)p->dq, (float)p->delta, (float)p->gamma_pow, 0};
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, B - c0);
        PatternSource src{XB, PTs, peaks->row_ptr + c0, peaks->qx, peaks->qy, peaks->I, nb,
                          (float)p->gamma_pow, (float)p->omega};
        RasterOut ro;
        ro.re = Xr;
        ro.im = Xi;
        ro.sumsq = xnorm2;
        launch_raster_patterns(geo, src, ro, p->err, st);
        float* U = dst + c0 * (int64_t)p->Z;
        if (tc)
            launch_contract_bound_tc(p, map_x, PTs, nb, U, st);
        else
            launch_contract_bound_fp32(p, Xr, Xi, nb, U, st);
    }
    prof_suppress(false);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "bounds_static launch");
    int herr = 0;
    e = cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "bounds_static");
    if (herr & kErrTimeout) return set_error(ACOM_ERR_TIMEOUT, "device wait timed out");
    if (herr) return set_error(ACOM_ERR_BAD_INPUT, "bad peak data (row_ptr, values or count)");
    return ACOM_OK;
}
