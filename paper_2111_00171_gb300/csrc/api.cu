// C ABI of libacom: argument validation, the zone-axis grid and its frames
// (host FP64), plan ownership, and the chunked match loop.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "acom_internal.cuh"

namespace acom {

static thread_local std::string g_last_error;

acom_status set_error(acom_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

acom_status cuda_error(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? ACOM_ERR_OOM : ACOM_ERR_CUDA;
}

void clear_error() { g_last_error.clear(); }

// device and pinned allocations the library has requested (acom_device_allocations)
static std::atomic<long long> g_allocs{0};
void count_allocation() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

static void normalize3(double* v) {
    double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n;
    v[1] /= n;
    v[2] /= n;
}

// Spherical linear interpolation between unit vectors (Shoemake).
static void slerp3(const double* p0, const double* p1, double t, double* out) {
    double d = p0[0] * p1[0] + p0[1] * p1[1] + p0[2] * p1[2];
    d = d > 1.0 ? 1.0 : (d < -1.0 ? -1.0 : d);
    double om = std::acos(d);
    if (om < 1e-15) {
        out[0] = p0[0];
        out[1] = p0[1];
        out[2] = p0[2];
        return;
    }
    double a = std::sin((1.0 - t) * om) / std::sin(om), b = std::sin(t * om) / std::sin(om);
    for (int i = 0; i < 3; ++i) out[i] = a * p0[i] + b * p1[i];
}

// Grid of zone axes spanning v0, v1, v2: n = floor(sqrt(2 Omega)/step)
// subdivisions; row i interpolates between slerp(v0,v1,i/n) and
// slerp(v0,v2,i/n) at j/i, j = 0..i.
static std::vector<double> zone_axes(const acom_za_grid* g) {
    double v[3][3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) v[r][c] = g->v[r][c];
        normalize3(v[r]);
    }
    int n = (int)std::floor(std::sqrt(2.0 * g->solid_angle) / (g->step_deg * M_PI / 180.0));
    if (n < 1) n = 1;
    std::vector<double> out;
    out.reserve(3 * (size_t)(n + 1) * (n + 2) / 2);
    for (int i = 0; i <= n; ++i) {
        if (i == 0) {
            out.insert(out.end(), v[0], v[0] + 3);
            continue;
        }
        double a[3], b[3], w[3];
        slerp3(v[0], v[1], (double)i / n, a);
        slerp3(v[0], v[2], (double)i / n, b);
        for (int j = 0; j <= i; ++j) {
            slerp3(a, b, (double)j / i, w);
            normalize3(w);
            out.insert(out.end(), w, w + 3);
        }
    }
    return out;
}

// R = Rz(phi1) Rx(theta2) with R z_hat = w (Eq. 10 sign convention):
// columns ... third column (-S1 S2, C1 S2, C2).
static void za_frame(const double* w, double* R) {
    double th = std::acos(w[2] > 1.0 ? 1.0 : (w[2] < -1.0 ? -1.0 : w[2]));
    double ph = std::atan2(-w[0], w[1]);
    double c1 = std::cos(ph), s1 = std::sin(ph), c2 = std::cos(th), s2 = std::sin(th);
    R[0] = c1; R[1] = -s1 * c2; R[2] = -s1 * s2;
    R[3] = s1; R[4] = c1 * c2;  R[5] = c1 * s2;
    R[6] = 0;  R[7] = -s2;      R[8] = c2;
}

// One pool per device; freed blocks stay in it (up to kPoolKeepBytes) so that
// a plan built per scan, and its workspace, reuse memory instead of paying for
// cudaMalloc and cudaFree every time.
constexpr uint64_t kPoolKeepBytes = 32ull << 30;
constexpr int kMaxDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kMaxDevices];

static cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    count_allocation();
    cudaMemPool_t pool = device_pool();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, st);
}

void pool_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

template <class T>
static cudaError_t dalloc(T** p, size_t n, size_t* acc, cudaStream_t st) {
    const size_t b = sizeof(T) * (n ? n : 1);
    cudaError_t e = pool_alloc(reinterpret_cast<void**>(p), b, st);
    if (e == cudaSuccess) *acc += b;
    return e;
}

static void free_workspace(Workspace& ws, cudaStream_t st) {
    pool_free(ws.Xr, st);
    pool_free(ws.Xi, st);
    pool_free(ws.Xsr, st);
    pool_free(ws.Xsi, st);
    pool_free(ws.xnorm2, st);
    pool_free(ws.Chat, st);
    pool_free(ws.U, st);
    pool_free(ws.xfn, st);
    pool_free(ws.n_eval, st);
    pool_free(ws.srange, st);
    pool_free(ws.rmask, st);
    pool_free(ws.best, st);
    pool_free(ws.za_scores, st);
    pool_free(ws.XB, st);
    pool_free(ws.xscale, st);
    pool_free(ws.XB8, st);
    pool_free(ws.oin, st);
    ws = Workspace{};
}

// need_fmajor: the frequency-major pattern spectra (FP32 contraction, export)
static acom_status ensure_ws(acom_plan_s* p, Workspace& ws, int chunk, bool need_chat,
                             bool need_fmajor, cudaStream_t st) {
    if (ws.chunk >= chunk && (!need_chat || ws.Chat) && (!need_fmajor || ws.Xr))
        return ACOM_OK;
    need_chat = need_chat || ws.Chat;
    need_fmajor = need_fmajor || need_chat || ws.Xr;
    if (ws.chunk > chunk) chunk = ws.chunk;
    free_workspace(ws, st);
    size_t acc = 0;
    const size_t spec = (size_t)chunk * p->F * p->Spad;
    const size_t sspec = (size_t)chunk * shell_row_stride(p->F) * p->Spad;
    cudaError_t e = cudaSuccess;
    // Every raster writes whole rows of its layouts (the pad frequencies of the
    // shell-major rows as zeros; every shell of the BF16 tiles), so nothing here
    // needs clearing.  Rows of the BF16 tiles past the last pattern of a chunk
    // keep stale values: each MMA row depends on its own pattern row only, and
    // those patterns' bounds are never written.
    if (need_fmajor && (e = dalloc(&ws.Xr, spec, &acc, st)) != cudaSuccess) goto fail;
    if (need_fmajor && (e = dalloc(&ws.Xi, spec, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.Xsr, sspec, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.Xsi, sspec, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.xnorm2, (size_t)chunk, &acc, st)) != cudaSuccess) goto fail;
    if (need_chat &&
        (e = dalloc(&ws.Chat, (size_t)4 * p->F * chunk * p->Zp, &acc, st)) != cudaSuccess)
        goto fail;
    if ((e = dalloc(&ws.U, (size_t)chunk * p->Z, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.xfn, (size_t)chunk * p->F, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.n_eval, (size_t)1, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.srange, (size_t)chunk, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.rmask, (size_t)chunk * (p->Spad / 32), &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.best, (size_t)chunk, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.za_scores, (size_t)chunk * p->Z, &acc, st)) != cudaSuccess) goto fail;
    if ((e = dalloc(&ws.oin, (size_t)chunk, &acc, st)) != cudaSuccess) goto fail;
    if (tc_precision(p->precision)) {
        // the raster writes BF16, or FP16 with a per-pattern scale; E4M3
        // operands are converted from the FP16 rows
        const bool scaled = p->precision != ACOM_PREC_BF16;
        const bool fp8 = p->precision == ACOM_PREC_FP8;
        ws.PTs = (chunk + 63) / 64;
        const size_t rows = (size_t)p->F * ws.PTs * 128;
        if ((e = pool_alloc(&ws.XB, rows * p->Spad * 2, st)) != cudaSuccess) goto fail;
        acc += rows * p->Spad * 2;
        if (fp8) {
            if ((e = pool_alloc(&ws.XB8, rows * p->Spad, st)) != cudaSuccess) goto fail;
            acc += rows * p->Spad;
        }
        if (scaled && (e = dalloc(&ws.xscale, (size_t)chunk, &acc, st)) != cudaSuccess) goto fail;
        acom_status ms = make_bf16_map(ws.map_x, fp8 ? ws.XB8 : ws.XB, rows, (uint64_t)p->Spad,
                                       tc_kind(p->precision));
        if (ms != ACOM_OK) {
            free_workspace(ws, st);
            return ms;
        }
    }
    ws.chunk = chunk;
    ws.bytes = acc;
    return ACOM_OK;
fail:
    free_workspace(ws, st);
    return cuda_error(e, "match workspace allocation");
}

static acom_status ensure_workspace(acom_plan_s* p, int chunk, bool need_chat, bool need_fmajor,
                                    cudaStream_t st) {
    return ensure_ws(p, p->ws, chunk, need_chat, need_fmajor, st);
}

// Every library call has synchronised its stream before returning, so the
// plan's memory goes back to the pool in the order of the default stream.
static void destroy_plan(acom_plan_s* p) {
    if (!p) return;
    const cudaStream_t st = 0;
    free_workspace(p->ws, st);
    pool_free(p->Pr, st);
    pool_free(p->Pi, st);
    pool_free(p->Psr, st);
    pool_free(p->Psi, st);
    pool_free(p->za, st);
    pool_free(p->frames, st);
    pool_free(p->nbr_ptr, st);
    pool_free(p->nbr_idx, st);
    pool_free(p->refl_g, st);
    pool_free(p->refl_amp, st);
    pool_free(p->err, st);
    pool_free(p->pfmax, st);
    pool_free(p->Pb, st);
    pool_free(p->phase_off, st);
    pool_free(p->refl_tab, st);
    pool_free(p->refine_pairs, st);
    pool_free(p->smask, st);
    if (p->host_words) cudaFreeHost(p->host_words);
    delete p;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// p->k0 from the plan's shell masks (synchronous copy): the lowest shell with a
// non-zero plan row on any axis, rounded down to a multiple of 16 (one MMA's K);
// 0 when the plan has no non-zero row at all.
static cudaError_t plan_k0(acom_plan_s* p, cudaStream_t st) {
    const int MW = p->Spad / 32;
    std::vector<uint32_t> m((size_t)p->Zp * MW);
    cudaError_t e = cudaMemcpyAsync(m.data(), p->smask, sizeof(uint32_t) * m.size(),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    int lo = p->Spad;
    for (int z = 0; z < p->Z; ++z)
        for (int w = 0; w < MW; ++w) {
            const uint32_t v = m[(size_t)z * MW + w];
            if (v) {
                int b = 0;
                while (!((v >> b) & 1u)) ++b;
                lo = std::min(lo, 32 * w + b);
                break;
            }
        }
    p->k0 = lo < p->Spad ? lo / 16 * 16 : 0;
    return cudaSuccess;
}

// The first row pointer of a CSR batch must be 0 (the other row checks run in
// the raster, per pattern); one thread, no allocation.
__global__ void k_check_row0(const int64_t* row_ptr, int* err) {
    if (row_ptr[0] != 0) atomicOr(err, kErrRowPtr);
}

void launch_check_row0(const int64_t* row_ptr, int* err, cudaStream_t st) {
    prof_begin(kKMisc, st);
    k_check_row0<<<1, 1, 0, st>>>(row_ptr, err);
    prof_end(kKMisc, st);
}

}  // namespace acom

using namespace acom;

extern "C" {

int32_t acom_version(void) { return 1; }

int64_t acom_device_allocations(void) { return (int64_t)g_allocs.load(); }

void acom_set_device_wait_limit(int64_t cycles) { set_wait_cycles((long long)cycles); }

const char* acom_status_str(acom_status s) {
    switch (s) {
        case ACOM_OK: return "ACOM_OK";
        case ACOM_ERR_INVALID_ARG: return "ACOM_ERR_INVALID_ARG";
        case ACOM_ERR_OOM: return "ACOM_ERR_OOM";
        case ACOM_ERR_CUDA: return "ACOM_ERR_CUDA";
        case ACOM_ERR_TIMEOUT: return "ACOM_ERR_TIMEOUT";
        case ACOM_ERR_UNSUPPORTED: return "ACOM_ERR_UNSUPPORTED";
        case ACOM_ERR_BAD_INPUT: return "ACOM_ERR_BAD_INPUT";
    }
    return "ACOM_ERR_UNKNOWN";
}

const char* acom_last_error(void) { return g_last_error.c_str(); }

acom_status acom_plan_create(const acom_crystal* crystal, const acom_za_grid* grid,
                             const acom_shells* shells, int32_t n_phi, double sigma_exc,
                             const acom_plan_opts* opts, void* cuda_stream, acom_plan* out) {
    g_last_error.clear();
    if (!crystal || !grid || !shells || !opts || !out)
        return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (crystal->n_atoms < 1 || crystal->n_atoms > 64 || !crystal->frac_pos || !crystal->ff_A ||
        !crystal->ff_B)
        return set_error(ACOM_ERR_INVALID_ARG, "crystal: n_atoms in 1..64 and basis arrays required");
    for (int i = 0; i < 3 * crystal->n_atoms; ++i)
        if (!std::isfinite(crystal->frac_pos[i]))
            return set_error(ACOM_ERR_INVALID_ARG, "crystal: non-finite fractional position");
    for (int i = 0; i < crystal->n_atoms; ++i)
        if (!std::isfinite(crystal->ff_A[i]) || !std::isfinite(crystal->ff_B[i]))
            return set_error(ACOM_ERR_INVALID_ARG, "crystal: non-finite form factor");
    if (!finite_pos(grid->step_deg) || !finite_pos(grid->solid_angle) || grid->solid_angle > 4 * M_PI)
        return set_error(ACOM_ERR_INVALID_ARG, "grid: step_deg and solid_angle must be positive");
    for (int r = 0; r < 3; ++r) {
        double n2 = 0;
        for (int c = 0; c < 3; ++c) n2 += grid->v[r][c] * grid->v[r][c];
        if (!(n2 > 0) || !std::isfinite(n2))
            return set_error(ACOM_ERR_INVALID_ARG, "grid: zero or non-finite boundary vector");
    }
    if (shells->n_shells < 1 || shells->n_shells > kMaxShells || !finite_pos(shells->dq))
        return set_error(ACOM_ERR_INVALID_ARG, "shells: n_shells in 1..512, dq > 0");
    if (n_phi < 8 || n_phi > kMaxPhi || (n_phi & 1))
        return set_error(ACOM_ERR_INVALID_ARG, "n_phi must be even, 8..720");
    if (!finite_pos(opts->delta) || !finite_pos(opts->lambda) || !finite_pos(opts->q_max) ||
        !std::isfinite(opts->gamma_pow) || !std::isfinite(opts->omega) || opts->omega < 0)
        return set_error(ACOM_ERR_INVALID_ARG, "opts: delta, lambda, q_max > 0; finite powers");
    if (opts->precision != ACOM_PREC_FP32 && !tc_precision(opts->precision))
        return set_error(ACOM_ERR_INVALID_ARG, "opts: unknown precision");

    std::vector<double> za = zone_axes(grid);
    const int Z = (int)(za.size() / 3);
    if (Z > 65535) return set_error(ACOM_ERR_UNSUPPORTED, "more than 65535 zone axes");

    acom_plan_s* p = new acom_plan_s();
    cudaGetDevice(&p->device);
    p->Z = Z;
    p->S = shells->n_shells;
    p->N = n_phi;
    p->F = n_phi / 2 + 1;
    p->Spad = (p->S + 31) / 32 * 32;     // K tiles of 32 for the tensor-core operands
    p->Zp = (Z + 127) / 128 * 128;       // M tiles of 128
    p->delta = opts->delta;
    p->gamma_pow = opts->gamma_pow;
    p->omega = opts->omega;
    p->lambda = opts->lambda;
    p->q_max = opts->q_max;
    p->sigma_exc = sigma_exc;
    p->step_deg = grid->step_deg;
    p->dq = shells->dq;
    p->precision = opts->precision;
    p->za_host = za;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    std::vector<double> frames(9 * (size_t)Z);
    for (int z = 0; z < Z; ++z) za_frame(&za[3 * z], &frames[9 * z]);
    // grid neighbours: axes within 1.5 steps
    std::vector<int> nptr(Z + 1, 0), nidx;
    const double lim = std::cos(1.5 * grid->step_deg * M_PI / 180.0);
    for (int z = 0; z < Z; ++z) {
        for (int z2 = 0; z2 < Z; ++z2) {
            double c = za[3 * z] * za[3 * z2] + za[3 * z + 1] * za[3 * z2 + 1] +
                       za[3 * z + 2] * za[3 * z2 + 2];
            if (c >= lim) nidx.push_back(z2);
        }
        nptr[z + 1] = (int)nidx.size();
    }

    cudaError_t e = cudaSuccess;
    acom_status s;
    const size_t pelems = (size_t)p->Zp * p->F * p->Spad;
    const size_t selems = (size_t)p->Zp * shell_row_stride(p->F) * p->Spad;
#define ACOM_CK(x)                                     \
    do {                                               \
        e = (x);                                       \
        if (e != cudaSuccess) goto cuda_fail;          \
    } while (0)
    ACOM_CK(dalloc(&p->Pr, pelems, &p->bytes, st));
    ACOM_CK(dalloc(&p->Pi, pelems, &p->bytes, st));
    ACOM_CK(dalloc(&p->Psr, selems, &p->bytes, st));
    ACOM_CK(dalloc(&p->Psi, selems, &p->bytes, st));
    ACOM_CK(dalloc(&p->za, za.size(), &p->bytes, st));
    ACOM_CK(dalloc(&p->frames, frames.size(), &p->bytes, st));
    ACOM_CK(dalloc(&p->nbr_ptr, nptr.size(), &p->bytes, st));
    ACOM_CK(dalloc(&p->nbr_idx, nidx.size(), &p->bytes, st));
    ACOM_CK(dalloc(&p->err, 1, &p->bytes, st));
    ACOM_CK(dalloc(&p->pfmax, (size_t)p->F, &p->bytes, st));
    p->phase_off_host = {0, Z};
    ACOM_CK(dalloc(&p->phase_off, 2, &p->bytes, st));
    count_allocation();
    ACOM_CK(cudaMallocHost(reinterpret_cast<void**>(&p->host_words), 2 * sizeof(int)));
    p->host_words[0] = p->host_words[1] = 0;
    ACOM_CK(cudaMemcpyAsync(p->phase_off, p->phase_off_host.data(), sizeof(int) * 2,
                            cudaMemcpyHostToDevice, st));
    ACOM_CK(cudaMemsetAsync(p->Pr, 0, sizeof(float) * pelems, st));
    ACOM_CK(cudaMemsetAsync(p->Pi, 0, sizeof(float) * pelems, st));
    ACOM_CK(cudaMemsetAsync(p->Psr, 0, sizeof(float) * selems, st));
    ACOM_CK(cudaMemsetAsync(p->Psi, 0, sizeof(float) * selems, st));
    ACOM_CK(cudaMemsetAsync(p->err, 0, sizeof(int), st));
    ACOM_CK(cudaMemcpyAsync(p->za, za.data(), sizeof(double) * za.size(), cudaMemcpyHostToDevice, st));
    ACOM_CK(cudaMemcpyAsync(p->frames, frames.data(), sizeof(double) * frames.size(),
                            cudaMemcpyHostToDevice, st));
    ACOM_CK(cudaMemcpyAsync(p->nbr_ptr, nptr.data(), sizeof(int) * nptr.size(),
                            cudaMemcpyHostToDevice, st));
    ACOM_CK(cudaMemcpyAsync(p->nbr_idx, nidx.data(), sizeof(int) * nidx.size(),
                            cudaMemcpyHostToDevice, st));
    s = build_plan_device(p, crystal, st);
    if (s != ACOM_OK) {
        destroy_plan(p);
        return s;
    }
    launch_plan_fnorm_max(p, p->pfmax, st);
    ACOM_CK(dalloc(&p->smask, (size_t)p->Zp * (p->Spad / 32), &p->bytes, st));
    launch_plan_shell_mask(p, st);
    ACOM_CK(cudaGetLastError());
    if (tc_precision(p->precision)) {
        const int kind = tc_kind(p->precision);
        p->pscale = kind == 0 ? 1.0f
                              : fp16_plan_scale(p->N) * (kind == 2 ? kFp8Shift : 1.0f);
        const size_t n = (size_t)p->F * p->Zp * p->Spad * tc_elem_bytes(p->precision);
        ACOM_CK(pool_alloc(&p->Pb, 2 * n, st));
        p->bytes += 2 * n;
        launch_plan_to_operand(p->Pr, p->Pi, p->Zp, p->F, p->Spad, p->Pb, st, kind, p->pscale);
        ACOM_CK(cudaGetLastError());
        s = make_bf16_map(p->map_p, p->Pb, (uint64_t)p->F * p->Zp * 2, (uint64_t)p->Spad, kind,
                          256);
        if (s == ACOM_OK)
            s = make_bf16_map(p->map_p128, p->Pb, (uint64_t)p->F * p->Zp * 2, (uint64_t)p->Spad,
                              kind, 128);
        if (s != ACOM_OK) {
            destroy_plan(p);
            return s;
        }
    }
    ACOM_CK(cudaStreamSynchronize(st));
    ACOM_CK(plan_k0(p, st));
    prof_resolve();
    *out = p;
    return ACOM_OK;
cuda_fail:
    destroy_plan(p);
    return cuda_error(e, "plan_create");
#undef ACOM_CK
}

acom_status acom_plan_concat(const acom_plan* plans, int32_t n_plans, void* cuda_stream,
                             acom_plan* out) {
    g_last_error.clear();
    if (!plans || !out || n_plans < 1)
        return set_error(ACOM_ERR_INVALID_ARG, "concat: plans, n_plans >= 1 and out required");
    const acom_plan_s* a = plans[0];
    if (!a) return set_error(ACOM_ERR_INVALID_ARG, "concat: null plan");
    int dev = 0;
    cudaGetDevice(&dev);
    int Z = 0, nph = 0, G = 0;
    for (int i = 0; i < n_plans; ++i) {
        const acom_plan_s* q = plans[i];
        if (!q) return set_error(ACOM_ERR_INVALID_ARG, "concat: null plan");
        if (q->device != dev)
            return set_error(ACOM_ERR_INVALID_ARG, "concat: a plan lives on another device");
        if (q->S != a->S || q->N != a->N || q->dq != a->dq || q->delta != a->delta ||
            q->gamma_pow != a->gamma_pow || q->omega != a->omega || q->precision != a->precision)
            return set_error(ACOM_ERR_INVALID_ARG,
                             "concat: plans differ in shells, bins, tent, exponents or precision");
        Z += q->Z;
        nph += q->n_phases;
        G += q->G;
    }
    if (nph > kMaxPhases) return set_error(ACOM_ERR_INVALID_ARG, "concat: more than 8 phases");
    if (Z > 65535) return set_error(ACOM_ERR_UNSUPPORTED, "concat: more than 65535 zone axes");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    acom_plan_s* p = new acom_plan_s();
    p->device = dev;
    p->Z = Z;
    p->S = a->S;
    p->N = a->N;
    p->F = a->F;
    p->Spad = a->Spad;
    p->Zp = (Z + 127) / 128 * 128;
    p->G = G;
    p->delta = a->delta;
    p->gamma_pow = a->gamma_pow;
    p->omega = a->omega;
    p->lambda = a->lambda;
    p->q_max = a->q_max;
    p->sigma_exc = a->sigma_exc;
    p->step_deg = a->step_deg;
    p->dq = a->dq;
    p->precision = a->precision;
    p->pscale = a->pscale;
    p->n_phases = nph;
    const int F = p->F, Spad = p->Spad, Fs = shell_row_stride(F);
    const size_t pelems = (size_t)p->Zp * F * Spad, selems = (size_t)p->Zp * Fs * Spad;
    std::vector<int> nptr(1, 0), nidx, qptr, qidx;
    std::vector<float> fmax((size_t)F, 0.f), qf((size_t)F);
    p->phase_off_host.assign(1, 0);
    cudaError_t e = cudaSuccess;
#define ACOM_CK(x)                                     \
    do {                                               \
        e = (x);                                       \
        if (e != cudaSuccess) goto cuda_fail;          \
    } while (0)
    // host side: axes, phase offsets, neighbour lists (offset into the
    // concatenation, so neighbours stay within their phase) and max_z ||P^_zf||
    for (int i = 0, base = 0; i < n_plans; base += plans[i]->Z, ++i) {
        const acom_plan_s* q = plans[i];
        p->za_host.insert(p->za_host.end(), q->za_host.begin(), q->za_host.end());
        for (int k = 1; k <= q->n_phases; ++k) p->phase_off_host.push_back(base + q->phase_off_host[k]);
        qptr.resize((size_t)q->Z + 1);
        ACOM_CK(cudaMemcpyAsync(qptr.data(), q->nbr_ptr, sizeof(int) * qptr.size(),
                                cudaMemcpyDeviceToHost, st));
        ACOM_CK(cudaStreamSynchronize(st));
        qidx.resize((size_t)qptr.back());
        if (!qidx.empty())
            ACOM_CK(cudaMemcpyAsync(qidx.data(), q->nbr_idx, sizeof(int) * qidx.size(),
                                    cudaMemcpyDeviceToHost, st));
        ACOM_CK(cudaMemcpyAsync(qf.data(), q->pfmax, sizeof(float) * F, cudaMemcpyDeviceToHost, st));
        ACOM_CK(cudaStreamSynchronize(st));
        const int ibase = (int)nidx.size();
        for (int z = 0; z < q->Z; ++z) nptr.push_back(ibase + qptr[(size_t)z + 1]);
        for (int v : qidx) nidx.push_back(base + v);
        for (int f = 0; f < F; ++f) fmax[f] = std::max(fmax[f], qf[f]);
    }
    ACOM_CK(dalloc(&p->Pr, pelems, &p->bytes, st));
    ACOM_CK(dalloc(&p->Pi, pelems, &p->bytes, st));
    ACOM_CK(dalloc(&p->Psr, selems, &p->bytes, st));
    ACOM_CK(dalloc(&p->Psi, selems, &p->bytes, st));
    ACOM_CK(dalloc(&p->za, (size_t)3 * Z, &p->bytes, st));
    ACOM_CK(dalloc(&p->frames, (size_t)9 * Z, &p->bytes, st));
    ACOM_CK(dalloc(&p->nbr_ptr, nptr.size(), &p->bytes, st));
    ACOM_CK(dalloc(&p->nbr_idx, nidx.size(), &p->bytes, st));
    ACOM_CK(dalloc(&p->err, 1, &p->bytes, st));
    ACOM_CK(dalloc(&p->pfmax, (size_t)F, &p->bytes, st));
    ACOM_CK(dalloc(&p->phase_off, p->phase_off_host.size(), &p->bytes, st));
    count_allocation();
    ACOM_CK(cudaMallocHost(reinterpret_cast<void**>(&p->host_words), 2 * sizeof(int)));
    p->host_words[0] = p->host_words[1] = 0;
    ACOM_CK(cudaMemsetAsync(p->Pr, 0, sizeof(float) * pelems, st));
    ACOM_CK(cudaMemsetAsync(p->Pi, 0, sizeof(float) * pelems, st));
    ACOM_CK(cudaMemsetAsync(p->Psr, 0, sizeof(float) * selems, st));
    ACOM_CK(cudaMemsetAsync(p->Psi, 0, sizeof(float) * selems, st));
    ACOM_CK(cudaMemsetAsync(p->err, 0, sizeof(int), st));
    ACOM_CK(cudaMemcpyAsync(p->nbr_ptr, nptr.data(), sizeof(int) * nptr.size(),
                            cudaMemcpyHostToDevice, st));
    if (!nidx.empty())
        ACOM_CK(cudaMemcpyAsync(p->nbr_idx, nidx.data(), sizeof(int) * nidx.size(),
                                cudaMemcpyHostToDevice, st));
    ACOM_CK(cudaMemcpyAsync(p->pfmax, fmax.data(), sizeof(float) * F, cudaMemcpyHostToDevice, st));
    ACOM_CK(cudaMemcpyAsync(p->phase_off, p->phase_off_host.data(),
                            sizeof(int) * p->phase_off_host.size(), cudaMemcpyHostToDevice, st));
    // device side: each input's rows at its offset (zone-axis-major layouts
    // are one contiguous block per input)
    for (int i = 0, base = 0; i < n_plans; base += plans[i]->Z, ++i) {
        const acom_plan_s* q = plans[i];
        const size_t zr = (size_t)q->Z;
        ACOM_CK(cudaMemcpyAsync(p->Pr + (size_t)base * F * Spad, q->Pr, sizeof(float) * zr * F * Spad,
                                cudaMemcpyDeviceToDevice, st));
        ACOM_CK(cudaMemcpyAsync(p->Pi + (size_t)base * F * Spad, q->Pi, sizeof(float) * zr * F * Spad,
                                cudaMemcpyDeviceToDevice, st));
        ACOM_CK(cudaMemcpyAsync(p->Psr + (size_t)base * Fs * Spad, q->Psr,
                                sizeof(float) * zr * Fs * Spad, cudaMemcpyDeviceToDevice, st));
        ACOM_CK(cudaMemcpyAsync(p->Psi + (size_t)base * Fs * Spad, q->Psi,
                                sizeof(float) * zr * Fs * Spad, cudaMemcpyDeviceToDevice, st));
        ACOM_CK(cudaMemcpyAsync(p->za + (size_t)3 * base, q->za, sizeof(double) * 3 * zr,
                                cudaMemcpyDeviceToDevice, st));
        ACOM_CK(cudaMemcpyAsync(p->frames + (size_t)9 * base, q->frames, sizeof(double) * 9 * zr,
                                cudaMemcpyDeviceToDevice, st));
    }
    ACOM_CK(dalloc(&p->smask, (size_t)p->Zp * (Spad / 32), &p->bytes, st));
    launch_plan_shell_mask(p, st);
    if (tc_precision(p->precision)) {
        // the merged [F][Zp / 128][256][Spad] operand of the concatenation
        const int kind = tc_kind(p->precision);
        const size_t eb = (size_t)tc_elem_bytes(p->precision);
        const size_t n = (size_t)F * p->Zp * Spad;
        ACOM_CK(pool_alloc(&p->Pb, 2 * n * eb, st));
        p->bytes += 2 * n * eb;
        // the merged operand from the concatenated FP32 spectra (the phases'
        // axes no longer start on 128-axis tiles)
        launch_plan_to_operand(p->Pr, p->Pi, p->Zp, F, Spad, p->Pb, st, kind, p->pscale);
        ACOM_CK(cudaGetLastError());
        acom_status s = make_bf16_map(p->map_p, p->Pb, (uint64_t)F * p->Zp * 2, (uint64_t)Spad,
                                      kind, 256);
        if (s == ACOM_OK)
            s = make_bf16_map(p->map_p128, p->Pb, (uint64_t)F * p->Zp * 2, (uint64_t)Spad, kind,
                              128);
        if (s != ACOM_OK) {
            cudaStreamSynchronize(st);
            destroy_plan(p);
            return s;
        }
    }
    ACOM_CK(cudaStreamSynchronize(st));
    ACOM_CK(plan_k0(p, st));
    *out = p;
    return ACOM_OK;
cuda_fail:
    cudaStreamSynchronize(st);
    destroy_plan(p);
    return cuda_error(e, "plan_concat");
#undef ACOM_CK
}

acom_status acom_plan_get_phases(acom_plan p, int32_t* dst) {
    if (!p || !dst) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    for (size_t i = 0; i < p->phase_off_host.size(); ++i) dst[i] = p->phase_off_host[i];
    return ACOM_OK;
}

acom_status acom_plan_destroy(acom_plan plan) {
    if (!plan) return set_error(ACOM_ERR_INVALID_ARG, "null plan");
    destroy_plan(plan);
    return ACOM_OK;
}

acom_status acom_plan_get_info(acom_plan p, acom_plan_info* info) {
    if (!p || !info) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    info->n_za = p->Z;
    info->n_shells = p->S;
    info->n_phi = p->N;
    info->n_freq = p->F;
    info->n_reflections = p->G;
    info->precision = p->precision;
    info->device_bytes = (int64_t)(p->bytes + p->ws.bytes);
    info->last_evaluated = p->last_evaluated;
    info->n_phases = p->n_phases;
    info->last_refine_pairs = p->last_refine_pairs;
    info->k0 = p->k0;
    return ACOM_OK;
}

acom_status acom_plan_get_zone_axes(acom_plan p, double* dst) {
    if (!p || !dst) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    std::memcpy(dst, p->za_host.data(), sizeof(double) * p->za_host.size());
    return ACOM_OK;
}

acom_status acom_plan_get_spectra(acom_plan p, float* dst, void* cuda_stream) {
    if (!p || !dst) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    launch_spectra_export(p->Pr, p->Pi, p->Z, p->F, p->Spad, p->S, dst, (cudaStream_t)cuda_stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ACOM_OK : cuda_error(e, "get_spectra");
}

static acom_status check_peaks(const acom_peaks_csr* pk) {
    if (!pk) return set_error(ACOM_ERR_INVALID_ARG, "null peaks");
    if (pk->n_patterns < 0) return set_error(ACOM_ERR_INVALID_ARG, "n_patterns < 0");
    if (pk->n_patterns > 0 && (!pk->row_ptr || !pk->qx || !pk->qy || !pk->I))
        return set_error(ACOM_ERR_INVALID_ARG, "null peak array");
    return ACOM_OK;
}

static acom_status read_error_word(acom_plan_s* p, cudaStream_t st) {
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "match");
    prof_resolve();
    if (herr & kErrTimeout) return set_error(ACOM_ERR_TIMEOUT, "device wait timed out");
    if (herr & (kErrRowPtr | kErrNonFinite | kErrTooManyPeaks)) {
        std::string m = "bad peak data:";
        if (herr & kErrRowPtr) m += " row_ptr not starting at 0 or decreasing;";
        if (herr & kErrNonFinite) m += " non-finite qx/qy/I;";
        if (herr & kErrTooManyPeaks) m += " more than 1024 peaks in a pattern;";
        return set_error(ACOM_ERR_BAD_INPUT, m);
    }
    return ACOM_OK;
}


acom_status acom_polar_spectra(acom_plan p, const acom_peaks_csr* peaks, float* dst, float* xnorm,
                               void* cuda_stream) {
    g_last_error.clear();
    if (!p || !dst) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    acom_status s = check_peaks(peaks);
    if (s != ACOM_OK) return s;
    const int64_t B = peaks->n_patterns;
    if (B == 0) return ACOM_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int chunk = (int)std::min<int64_t>(B, 1024);
    s = ensure_workspace(p, chunk, false, true, st);
    if (s != ACOM_OK) return s;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
    launch_check_row0(peaks->row_ptr, p->err, st);
    RasterGeom geo{p->S, p->Spad, p->N, p->F, (float)p->dq, (float)p->delta, (float)p->gamma_pow, 0};
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, B - c0);
        PatternSource src{nullptr, 0, peaks->row_ptr + c0, peaks->qx, peaks->qy, peaks->I, nb,
                          (float)p->gamma_pow, (float)p->omega};
        RasterOut ro;
        ro.re = p->ws.Xr;
        ro.im = p->ws.Xi;
        ro.sumsq = p->ws.xnorm2;
        launch_raster_patterns(geo, src, ro, p->err, st);
        launch_spectra_export(p->ws.Xr, p->ws.Xi, nb, p->F, p->Spad, p->S,
                              dst + 2 * c0 * (int64_t)p->S * p->F, st);
        if (xnorm) {
            cudaMemcpyAsync(xnorm + c0, p->ws.xnorm2, sizeof(float) * nb, cudaMemcpyDeviceToDevice, st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "polar_spectra launch");
    s = read_error_word(p, st);
    return s;
}

// Rounding constant of the FP32 contraction: |c_f(computed) - c_f| <= kappa
// ||P^_f|| ||X^_f|| (dot products of 2S terms, complex combination, sqrt).
static float kappa_fp32(const acom_plan_s* p) {
    return (float)((3.0 * (p->Spad + 2) + 2.0 * p->F) * std::ldexp(1.0, -24));
}

// BF16 operands: each product carries at most 2^-7 relative rounding, and
// |Pr|+|Pi| <= sqrt(2)|P^| (same for X^) gives 2^-6 ||P^_f|| ||X^_f|| for the
// complex spectrum; the tensor-core FP32 accumulation is charged 8x the FP32
// dot-product term.
static float kappa_bf16(const acom_plan_s* p) {
    return (float)(std::ldexp(1.0, -6) +
                   (3.0 * (p->Spad + 2) + 2.0 * p->F) * std::ldexp(1.0, -21));
}

// FP16 operands: relative rounding 2^-11 per operand gives 2^-10 per product
// and 2^-9 for the complex spectrum, as for BF16; values below the normal range
// are charged separately by the select kernel (an absolute term per pattern).
static float kappa_fp16(const acom_plan_s* p) {
    return (float)(std::ldexp(1.0, -9) +
                   (3.0 * (p->Spad + 2) + 2.0 * p->F) * std::ldexp(1.0, -21));
}

// E4M3 operands: relative rounding 2^-4 per operand, 2^-3 per product and
// 2^-2 for the complex spectrum; values below the normal range are charged
// by the select kernel's absolute term (eta 2^-6)
static float kappa_fp8(const acom_plan_s* p) {
    return (float)(std::ldexp(1.0, -2) +
                   (3.0 * (p->Spad + 2) + 2.0 * p->F) * std::ldexp(1.0, -21));
}

static float kappa_tc(const acom_plan_s* p) {
    return p->precision == ACOM_PREC_FP8    ? kappa_fp8(p)
           : p->precision == ACOM_PREC_FP16 ? kappa_fp16(p)
                                            : kappa_bf16(p);
}

// the FP16 raster rows of a chunk into the E4M3 operand (FP8 plans)
static void convert_fp8(acom_plan_s* p, const Workspace& ws, cudaStream_t st) {
    if (p->precision != ACOM_PREC_FP8) return;
    const int64_t n = (int64_t)p->F * ws.PTs * 128 * p->Spad;
    launch_half_to_e4m3(ws.XB, ws.XB8, n, kFp8Shift, st);
}

// Everything acom_match does up to the read of the error word: validation,
// workspace, launches.  With capture set (stream capture in progress) the
// workspace must already fit and no profiling events are recorded.
static acom_status match_enqueue(acom_plan p, const acom_peaks_csr* peaks,
                                 const acom_match_opts* opts, acom_result* out,
                                 cudaStream_t st, bool capture, bool* empty) {
    *empty = false;
    if (!p || !out) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    acom_status s = check_peaks(peaks);
    if (s != ACOM_OK) return s;
    const int64_t B = peaks->n_patterns;
    if (B > 0 && (!out->za_idx || !out->phi3_bin || !out->mirror || !out->score))
        return set_error(ACOM_ERR_INVALID_ARG, "result: za_idx, phi3_bin, mirror, score required");
    if (B == 0) {
        *empty = true;
        return ACOM_OK;
    }
    const int refine = opts ? opts->refine : 1;
    const bool exhaustive = opts && opts->exhaustive;
    const int rescore_top = opts && !exhaustive ? opts->rescore_top : 0;
    if (rescore_top < 0) return set_error(ACOM_ERR_INVALID_ARG, "rescore_top must be >= 0");
    const int tile_order = opts ? opts->tile_order : 0;
    if (tile_order < 0 || tile_order > 1)
        return set_error(ACOM_ERR_INVALID_ARG, "tile_order must be 0 or 1");
    const int cta_pairs = opts ? opts->cta_pairs : 0;
    if (cta_pairs < 0 || cta_pairs > 1)
        return set_error(ACOM_ERR_INVALID_ARG, "cta_pairs must be 0 or 1");
    if (exhaustive && (out->runner_za || out->runner_score || out->runner_orient))
        return set_error(ACOM_ERR_UNSUPPORTED, "runner-up outputs need certified pruning");
    if (!exhaustive && p->Z > 16384)
        return set_error(ACOM_ERR_UNSUPPORTED, "pruned mode supports at most 16384 zone axes");
    int chunk = opts && opts->chunk > 0 ? opts->chunk : (exhaustive ? 1024 : 8192);
    if (chunk > 65536) return set_error(ACOM_ERR_INVALID_ARG, "chunk must be <= 65536");
    chunk = (int)std::min<int64_t>(chunk, B);
    const bool fp32_contraction = exhaustive || p->precision == ACOM_PREC_FP32;
    if (capture && !(p->ws.chunk >= chunk && (!exhaustive || p->ws.Chat) &&
                     (!fp32_contraction || p->ws.Xr)))
        return set_error(ACOM_ERR_INVALID_ARG,
                         "match_async under stream capture: the workspace is not sized yet "
                         "(run acom_match once with the same chunk and mode first)");
    s = ensure_workspace(p, chunk, exhaustive, fp32_contraction, st);
    if (s != ACOM_OK) return s;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
    cudaMemsetAsync(p->ws.n_eval, 0, sizeof(int), st);
    launch_check_row0(peaks->row_ptr, p->err, st);
    RasterGeom geo{p->S, p->Spad, p->N, p->F, (float)p->dq, (float)p->delta, (float)p->gamma_pow, 0};
    const int wchunk = p->ws.chunk;
    Workspace& w = p->ws;
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, B - c0);
        const bool tc = !exhaustive && tc_precision(p->precision);
        float* xscale = tc && p->precision != ACOM_PREC_BF16 ? w.xscale : nullptr;
        PatternSource src{tc ? w.XB : nullptr, w.PTs, peaks->row_ptr + c0, peaks->qx,
                          peaks->qy, peaks->I, nb, (float)p->gamma_pow, (float)p->omega,
                          xscale ? 1 : 0, xscale, p->k0};
        RasterOut ro;
        ro.re = fp32_contraction ? w.Xr : nullptr;
        ro.im = fp32_contraction ? w.Xi : nullptr;
        ro.sre = w.Xsr;
        ro.sim = w.Xsi;
        ro.sumsq = w.xnorm2;
        ro.fnorm = w.xfn;
        ro.srange = w.srange;
        // select reads only the rows the pattern's tents reach
        ro.rmask = exhaustive ? nullptr : w.rmask;
        launch_raster_patterns(geo, src, ro, p->err, st);
        if (exhaustive) {
            cudaMemsetAsync(w.best, 0, sizeof(unsigned long long) * nb, st);
            launch_contract_fp32(p, w.Xr, w.Xi, nb, w.Chat, wchunk, st);
            launch_idft_argmax_fp32(p, w.Chat, nb, wchunk, w.za_scores, w.best, st);
            launch_refine(p, w.Chat, nb, wchunk, w.za_scores, w.best, w.xnorm2, refine, *out, c0,
                          st);
            if (out->za_scores)
                cudaMemcpyAsync(out->za_scores + c0 * (int64_t)p->Z, w.za_scores,
                                sizeof(float) * (size_t)nb * p->Z, cudaMemcpyDeviceToDevice, st);
            if (out->phase || out->phase_score)
                launch_phase_outputs(p, w.za_scores, nb, *out, c0, st);
        } else {
            if (tc) {
                convert_fp8(p, w, st);
                launch_contract_bound_tc(p, w.map_x, w.PTs, nb, w.U, st, xscale, tile_order,
                                         cta_pairs);
            } else {
                launch_contract_bound_fp32(p, w.Xr, w.Xi, nb, w.U, st);
            }
            launch_select_exact(p, w.Xsr, w.Xsi, w.U, w.xfn, w.srange, w.rmask, p->pfmax,
                                w.xnorm2, nb, tc ? kappa_tc(p) : kappa_fp32(p), refine, *out,
                                c0, w.n_eval, st, xscale, rescore_top, w.oin);
            if (out->phi3 || out->orient)
                launch_orient_compose(p, w.oin, nb, refine, *out, c0, st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "match launch");
    // error word and evaluations into the plan's pinned words
    cudaMemcpyAsync(p->host_words, p->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(p->host_words + 1, p->ws.n_eval, sizeof(int), cudaMemcpyDeviceToHost, st);
    p->async_exhaustive_evals = exhaustive ? (int64_t)B * p->Z : -1;
    return ACOM_OK;
}

// Status of the words the last enqueued match copied to pinned memory.
static acom_status finish_words(acom_plan_s* p, cudaStream_t st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "match");
    prof_resolve();
    const int herr = p->host_words[0];
    p->last_evaluated =
        p->async_exhaustive_evals >= 0 ? p->async_exhaustive_evals : (int64_t)p->host_words[1];
    if (herr & kErrTimeout) return set_error(ACOM_ERR_TIMEOUT, "device wait timed out");
    if (herr & (kErrRowPtr | kErrNonFinite | kErrTooManyPeaks)) {
        std::string m = "bad peak data:";
        if (herr & kErrRowPtr) m += " row_ptr not starting at 0 or decreasing;";
        if (herr & kErrNonFinite) m += " non-finite qx/qy/I;";
        if (herr & kErrTooManyPeaks) m += " more than 1024 peaks in a pattern;";
        return set_error(ACOM_ERR_BAD_INPUT, m);
    }
    return ACOM_OK;
}

acom_status acom_match(acom_plan p, const acom_peaks_csr* peaks, const acom_match_opts* opts,
                       acom_result* out, void* cuda_stream) {
    g_last_error.clear();
    cudaStream_t st = (cudaStream_t)cuda_stream;
    bool empty = false;
    acom_status s = match_enqueue(p, peaks, opts, out, st, false, &empty);
    if (s != ACOM_OK || empty) return s;
    return finish_words(p, st);
}

acom_status acom_match_async(acom_plan p, const acom_peaks_csr* peaks,
                             const acom_match_opts* opts, acom_result* out, void* cuda_stream) {
    g_last_error.clear();
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool capture = cap != cudaStreamCaptureStatusNone;
    prof_suppress(capture);
    bool empty = false;
    acom_status s = match_enqueue(p, peaks, opts, out, st, capture, &empty);
    prof_suppress(false);
    return s;
}

acom_status acom_sync(acom_plan p, void* cuda_stream) {
    g_last_error.clear();
    if (!p) return set_error(ACOM_ERR_INVALID_ARG, "null plan");
    return finish_words(p, (cudaStream_t)cuda_stream);
}

acom_status acom_bounds(acom_plan p, const acom_peaks_csr* peaks, float* dst, void* cuda_stream) {
    g_last_error.clear();
    if (!p || !dst) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    acom_status s = check_peaks(peaks);
    if (s != ACOM_OK) return s;
    const int64_t B = peaks->n_patterns;
    if (B == 0) return ACOM_OK;
    const int chunk = (int)std::min<int64_t>(B, 8192);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool tc = tc_precision(p->precision);
    s = ensure_workspace(p, chunk, false, !tc, st);
    if (s != ACOM_OK) return s;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
    launch_check_row0(peaks->row_ptr, p->err, st);
    RasterGeom geo{p->S, p->Spad, p->N, p->F, (float)p->dq, (float)p->delta, (float)p->gamma_pow, 0};
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, B - c0);
        float* xscale = tc && p->precision != ACOM_PREC_BF16 ? p->ws.xscale : nullptr;
        PatternSource src{tc ? p->ws.XB : nullptr, p->ws.PTs, peaks->row_ptr + c0, peaks->qx,
                          peaks->qy, peaks->I, nb, (float)p->gamma_pow, (float)p->omega,
                          xscale ? 1 : 0, xscale, p->k0};
        RasterOut ro;
        ro.re = tc ? nullptr : p->ws.Xr;
        ro.im = tc ? nullptr : p->ws.Xi;
        ro.sumsq = p->ws.xnorm2;
        launch_raster_patterns(geo, src, ro, p->err, st);
        float* U = dst + c0 * (int64_t)p->Z;
        if (tc) {
            convert_fp8(p, p->ws, st);
            launch_contract_bound_tc(p, p->ws.map_x, p->ws.PTs, nb, U, st, xscale);
        } else {
            launch_contract_bound_fp32(p, p->ws.Xr, p->ws.Xi, nb, U, st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "bounds launch");
    return read_error_word(p, st);
}

acom_status acom_refine(acom_plan p, const acom_peaks_csr* peaks, const acom_refine_opts* opts,
                        float* orient, const float* orient_alt, float* score, uint8_t* start,
                        void* cuda_stream) {
    g_last_error.clear();
    if (!p || !orient) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    acom_status s = check_peaks(peaks);
    if (s != ACOM_OK) return s;
    acom_refine_opts o = opts ? *opts : acom_refine_defaults();
    if (o.steps < 0 || o.steps > 1000 || !(o.rho_start > 0) || !(o.rho_end > 0) ||
        !std::isfinite(o.rho_start) || !std::isfinite(o.rho_end) || !(o.damping >= 0) ||
        !std::isfinite(o.damping) || !(o.max_step_deg > 0) || !std::isfinite(o.max_step_deg))
        return set_error(ACOM_ERR_INVALID_ARG,
                         "refine opts: steps 0..1000, rho > 0, damping >= 0, max_step_deg > 0");
    if (peaks->n_patterns == 0) return ACOM_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s = refine_table(p, st);
    if (s != ACOM_OK) return s;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
    cudaMemsetAsync(p->refine_pairs, 0, sizeof(unsigned long long), st);
    launch_check_row0(peaks->row_ptr, p->err, st);
    launch_refine_orient(p, peaks, o.steps, o.rho_start, o.rho_end, o.damping,
                         (float)(o.max_step_deg * M_PI / 180.0), o.twin ? 1 : 0, orient,
                         orient_alt, score, start, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "refine launch");
    unsigned long long pairs = 0;
    cudaMemcpyAsync(&pairs, p->refine_pairs, sizeof(pairs), cudaMemcpyDeviceToHost, st);
    s = read_error_word(p, st);
    p->last_refine_pairs = (int64_t)pairs;
    return s;
}

acom_status acom_kinematical_score_strain(acom_plan p, const acom_peaks_csr* peaks,
                                          const float* orient, const float* r,
                                          const float* strain, float rho, float* score,
                                          float* grad, float* gn, float* strain_grad,
                                          void* cuda_stream) {
    g_last_error.clear();
    if (!p || !orient) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    acom_status s = check_peaks(peaks);
    if (s != ACOM_OK) return s;
    if (!(rho > 0) || !std::isfinite(rho)) return set_error(ACOM_ERR_INVALID_ARG, "rho must be > 0");
    if (peaks->n_patterns == 0) return ACOM_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s = refine_table(p, st);
    if (s != ACOM_OK) return s;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
    launch_check_row0(peaks->row_ptr, p->err, st);
    launch_kin_score(p, peaks, orient, r, strain, rho, score, grad, gn, strain_grad, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "score launch");
    return read_error_word(p, st);
}

acom_status acom_kinematical_score(acom_plan p, const acom_peaks_csr* peaks, const float* orient,
                                   const float* r, float rho, float* score, float* grad,
                                   float* gn, void* cuda_stream) {
    return acom_kinematical_score_strain(p, peaks, orient, r, nullptr, rho, score, grad, gn,
                                         nullptr, cuda_stream);
}

acom_refine_opts acom_refine_defaults(void) {
    acom_refine_opts o;
    o.steps = 20;
    o.rho_start = 0.15f;
    o.rho_end = 0.03f;
    o.damping = 0.3f;
    o.max_step_deg = 1.0f;
    o.twin = 1;
    return o;
}

acom_status acom_match_multi(acom_plan p, const acom_peaks_csr* peaks,
                             const acom_match_opts* opts, int32_t n_matches, float r_del,
                             acom_result* results, void* cuda_stream) {
    g_last_error.clear();
    if (!p || !results) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    acom_status s = check_peaks(peaks);
    if (s != ACOM_OK) return s;
    if (n_matches < 1 || n_matches > kMaxMatches)
        return set_error(ACOM_ERR_INVALID_ARG, "n_matches must be 1..8");
    if (!(r_del >= 0.0f) || !(r_del < (float)p->delta))
        return set_error(ACOM_ERR_INVALID_ARG, "r_del must be in [0, delta)");
    const int64_t B = peaks->n_patterns;
    for (int j = 0; j < n_matches; ++j)
        if (B > 0 && (!results[j].za_idx || !results[j].phi3_bin || !results[j].mirror ||
                      !results[j].score))
            return set_error(ACOM_ERR_INVALID_ARG,
                             "each result needs za_idx, phi3_bin, mirror and score");
    if (B == 0) return ACOM_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s = refine_table(p, st);
    if (s != ACOM_OK) return s;
    int64_t nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, peaks->row_ptr + B, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "match_multi: reading row_ptr");
    if (nnz < 0) return set_error(ACOM_ERR_BAD_INPUT, "bad peak data: row_ptr decreasing");
    // working copy of the peaks: deletion changes it between matches
    float *wx = nullptr, *wy = nullptr, *wI = nullptr;
    const size_t bytes = sizeof(float) * (size_t)(nnz > 0 ? nnz : 1);
    if ((e = pool_alloc(reinterpret_cast<void**>(&wx), bytes, st)) != cudaSuccess ||
        (e = pool_alloc(reinterpret_cast<void**>(&wy), bytes, st)) != cudaSuccess ||
        (e = pool_alloc(reinterpret_cast<void**>(&wI), bytes, st)) != cudaSuccess) {
        pool_free(wx, st);
        pool_free(wy, st);
        pool_free(wI, st);
        return cuda_error(e, "match_multi: working peaks");
    }
    auto release = [&]() {
        pool_free(wx, st);
        pool_free(wy, st);
        pool_free(wI, st);
    };
    if (nnz > 0) {
        cudaMemcpyAsync(wx, peaks->qx, sizeof(float) * nnz, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(wy, peaks->qy, sizeof(float) * nnz, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(wI, peaks->I, sizeof(float) * nnz, cudaMemcpyDeviceToDevice, st);
    }
    acom_peaks_csr work{B, peaks->row_ptr, wx, wy, wI};
    for (int j = 0; j < n_matches; ++j) {
        s = acom_match(p, &work, opts, &results[j], cuda_stream);
        if (s != ACOM_OK) {
            release();
            return s;
        }
        launch_delete_peaks(p, &work, results[j], r_del, 1e-3f, st);
    }
    // the full pattern's correlation at every match
    const int chunk = (int)std::min<int64_t>(B, 8192);
    s = ensure_workspace(p, chunk, false, false, st);
    if (s != ACOM_OK) {
        release();
        return s;
    }
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
    RasterGeom geo{p->S, p->Spad, p->N, p->F, (float)p->dq, (float)p->delta, (float)p->gamma_pow, 0};
    for (int64_t c0 = 0; c0 < B; c0 += chunk) {
        const int nb = (int)std::min<int64_t>(chunk, B - c0);
        PatternSource src{nullptr, p->ws.PTs, peaks->row_ptr + c0, peaks->qx, peaks->qy, peaks->I, nb,
                          (float)p->gamma_pow, (float)p->omega};
        RasterOut ro;
        ro.sre = p->ws.Xsr;
        ro.sim = p->ws.Xsi;
        ro.sumsq = p->ws.xnorm2;
        ro.fnorm = p->ws.xfn;
        ro.srange = p->ws.srange;
        launch_raster_patterns(geo, src, ro, p->err, st);
        launch_score_at(p, p->ws.Xsr, p->ws.Xsi, p->ws.srange, p->ws.xnorm2, nb, results, n_matches,
                        c0, st);
    }
    e = cudaGetLastError();
    release();
    if (e != cudaSuccess) return cuda_error(e, "match_multi launch");
    return read_error_word(p, st);
}

acom_status acom_autotune(acom_plan p, const acom_peaks_csr* peaks, const acom_match_opts* base,
                          acom_tune_result* best, acom_tune_result* trials, void* cuda_stream) {
    g_last_error.clear();
    if (!p || !peaks || !best) return set_error(ACOM_ERR_INVALID_ARG, "null argument");
    if (peaks->n_patterns <= 0) return set_error(ACOM_ERR_INVALID_ARG, "empty sample");
    const int64_t B = peaks->n_patterns;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // results of the trial matches go to scratch owned by this call
    int32_t *za = nullptr, *kb = nullptr;
    uint8_t* mi = nullptr;
    float* sc = nullptr;
    cudaError_t e;
    if ((e = pool_alloc(reinterpret_cast<void**>(&za), sizeof(int32_t) * B, st)) != cudaSuccess ||
        (e = pool_alloc(reinterpret_cast<void**>(&kb), sizeof(int32_t) * B, st)) != cudaSuccess ||
        (e = pool_alloc(reinterpret_cast<void**>(&mi), B, st)) != cudaSuccess ||
        (e = pool_alloc(reinterpret_cast<void**>(&sc), sizeof(float) * B, st)) != cudaSuccess) {
        pool_free(za, st);
        pool_free(kb, st);
        pool_free(mi, st);
        pool_free(sc, st);
        return cuda_error(e, "autotune scratch");
    }
    acom_result r{};
    r.za_idx = za;
    r.phi3_bin = kb;
    r.mirror = mi;
    r.score = sc;
    acom_match_opts o = base ? *base : acom_match_opts{1, 0, 0, 0, 0, 0};
    const int chunks[3] = {8192, 16384, 32768};
    const bool tc = tc_precision(p->precision) && !o.exhaustive;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    acom_status s = ACOM_OK;
    best->ms = -1.0f;
    int n = 0;
    for (int ci = 0; ci < 3 && s == ACOM_OK; ++ci)
        for (int order = 0; order < 2 && s == ACOM_OK; ++order)
            for (int pairs = 0; pairs < 2 && s == ACOM_OK; ++pairs) {
            o.chunk = chunks[ci];
            o.tile_order = order;
            o.cta_pairs = tc ? pairs : 0;
            s = acom_match(p, peaks, &o, &r, cuda_stream);           // warm-up, sizes the workspace
            if (s != ACOM_OK) break;
            cudaEventRecord(t0, st);
            s = acom_match(p, peaks, &o, &r, cuda_stream);
            cudaEventRecord(t1, st);
            cudaEventSynchronize(t1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            const acom_tune_result tr{o.chunk, order, o.cta_pairs, ms};
            if (trials) trials[n] = tr;
            ++n;
            if (best->ms < 0.f || ms < best->ms) *best = tr;
        }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    pool_free(za, st);
    pool_free(kb, st);
    pool_free(mi, st);
    pool_free(sc, st);
    cudaStreamSynchronize(st);
    return s;
}

}  // extern "C"
