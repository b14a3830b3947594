// Internal declarations shared by the translation units of libacom.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/acom.h"

namespace acom {

constexpr int kMaxPeaks = 1024;     // peaks per pattern held on chip
constexpr int kMaxPhi = 720;        // in-plane bins (F <= 361)
constexpr int kMaxShells = 512;
constexpr int kRasterThreads = 256;  // 8 warps: one shell per warp per group
constexpr int kShellGroup = 8;

// device error word bits
constexpr int kErrRowPtr = 1;       // row_ptr[0] != 0 or decreasing
constexpr int kErrNonFinite = 2;    // qx, qy or I not finite
constexpr int kErrTooManyPeaks = 4; // more than kMaxPeaks peaks in a pattern
constexpr int kErrTimeout = 8;      // a bounded device wait gave up

// Parameters of the sparse polar raster shared by plan and pattern sources.
// Row stride (in floats) of the shell-major spectra [item][Spad][Fs]: F
// rounded up to a multiple of 4, so every row starts on a 16-byte boundary and
// the exact evaluation can load four frequencies at once.  Pad entries are 0.
__host__ __device__ inline int shell_row_stride(int F) { return (F + 3) & ~3; }

// Device memory of plans and match workspaces: stream-ordered allocations from
// one pool per device that keeps freed blocks for reuse (api.cu).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);

struct RasterGeom {
    int S, Spad, N, F;
    float dq;          // shells q_s = (s + 1) dq
    float delta;
    float gamma_pow;   // radial power
    int shell_power;   // 1: multiply rows by q_s^gamma_pow (plan); 0: peaks carry q_m^gamma
};

// Outputs of the raster + transform kernel (every pointer optional but one).
struct RasterOut {
    float* re = nullptr;       // [item][F][Spad] (frequency-major rows of shells)
    float* im = nullptr;
    float* sre = nullptr;      // [item][Spad][Fs] (shell-major rows of frequencies, Fs = shell_row_stride(F))
    float* sim = nullptr;
    float* sumsq = nullptr;    // [item] sum of squares of the polar image
    float* fnorm = nullptr;    // [item][F] ||X^_f|| over shells
    int2* srange = nullptr;    // [item] first and one-past-last shell with a non-zero row
    // [item][Spad / 32] bit s: some peak's tent reached shell s.  When given, the
    // shell-major rows (sre, sim) are written only for shell pairs with such a
    // shell, and a reader must skip every row whose bit is clear (those rows
    // are exactly zero and their memory is left as it was).
    uint32_t* rmask = nullptr;
};

struct PlanSource {            // reflections rotated into each zone-axis frame
    const double* g;           // [G][3] crystal Cartesian
    const double* amp;         // [G] |F|^omega
    const double* frames;      // [Z][9] row-major R = Rz(phi1) Rx(theta2)
    int G;
    double lambda;
};

struct PatternSource {         // one chunk of CSR patterns
    void* xb;                  // optional BF16 [F][PTs][128][Spad] output (16-row groups: 8 re, 8 im)
    int PTs;
    const int64_t* row_ptr;    // global row_ptr, already offset to the chunk start
    const float* qx;
    const float* qy;
    const float* I;
    int64_t n_items;
    float gamma_pow, omega;
    int xb_fp16 = 0;           // xb holds FP16 of 2^e_b X^ instead of BF16 of X^
    float* xscale = nullptr;   // [n_items] 2^e_b of each pattern (with xb_fp16)
    int xb_k0 = 0;             // the contraction reads xb from this shell on: 16-shell
                               // tiles wholly below it are not written
};

// FP16 operands of the tensor-core contraction: each pattern's spectrum is
// stored as FP16(2^e X^) with 2^e B <= 2^14, B an a-priori bound on |X^_sf|
// (X >= 0, so |X^_sf| <= X^_s0 = sum_j X(s, j) <= sum_m w_m n_m, n_m the most
// bins a peak's tent can cover), and the plan's as FP16(2^k P^) with
// 2^k sqrt(N) <= 2^14 (||P_z|| = 1 and P >= 0 bound |P^_zsf| by sqrt(N)).
// The bound U is divided by 2^(e+k) again; both scales are powers of two, so
// scaling and unscaling are exact.
constexpr float kFp16Target = 16384.0f;
// Absolute error of an FP16 operand below the normal range (|x| < 2^-14),
// whether the value is rounded to a subnormal or flushed to zero
constexpr double kFp16Eta = 6.103515625e-05;   // 2^-14
// E4M3 operands: the FP16 operands times 2^-6 (|x| <= 2^8 < 448, exact), so
// the pattern and plan scales are the FP16 ones times 2^-6; below E4M3's
// normal range (2^-6) an operand is off by at most 2^-6
constexpr float kFp8Shift = 0.015625f;          // 2^-6
constexpr double kFp8Eta = 0.015625;            // 2^-6

// 2^k of the plan's FP16 spectra: the largest power of two with 2^k sqrt(N) <= 2^14
inline float fp16_plan_scale(int N) {
    double s = 1.0;
    while (2.0 * s * std::sqrt((double)N) <= kFp16Target) s *= 2.0;
    while (s * std::sqrt((double)N) > kFp16Target) s *= 0.5;
    return (float)s;
}

// What the select kernel hands the orientation kernel for one pattern: the
// winner (axis z, bin + mirror * N), the correlation at bins k - 1, k, k + 1
// and the score-weighted sum of the neighbour axes within 0.9 of the best.
struct OrientIn {
    double w[3];
    float c3[3];
    int z, km, pad;
};

// Workspace for one chunk of patterns.
struct Workspace {
    int chunk = 0;                 // capacity in patterns
    float* Xr = nullptr;           // [chunk][F][Spad] (FP32 contraction only)
    float* Xi = nullptr;
    float* Xsr = nullptr;          // [chunk][Spad][Fs] (exact evaluation)
    float* Xsi = nullptr;
    float* xnorm2 = nullptr;       // [chunk]
    float* Chat = nullptr;         // [4][F][chunk][Zp] (exhaustive mode only)
    float* U = nullptr;            // [chunk][Z] spectral bounds
    void* XB = nullptr;            // BF16 [F][PTs][128][Spad] (tensor-core operand, 16-row groups: 8 re, 8 im)
    int PTs = 0;                   // pattern tiles of 64 in XB
    alignas(64) unsigned char map_x[128];   // TMA map of XB
    float* xfn = nullptr;          // [chunk][F] ||X^_bf|| over shells
    int* n_eval = nullptr;         // axes evaluated exactly in the last match
    int2* srange = nullptr;        // [chunk] non-zero shell range of each pattern
    uint32_t* rmask = nullptr;     // [chunk][Spad / 32] shells each pattern's tents reach
    unsigned long long* best = nullptr;  // [chunk] packed (score, index)
    float* za_scores = nullptr;    // [chunk][Z]
    float* xscale = nullptr;       // [chunk] 2^e of each pattern's FP16 spectrum
    void* XB8 = nullptr;           // E4M3 copy of XB (FP8 plans)
    OrientIn* oin = nullptr;       // [chunk] winners for the orientation kernel
    size_t bytes = 0;
};

// phases of one plan (acom_plan_concat)
constexpr int kMaxPhases = 8;
// matches per pattern of acom_match_multi
constexpr int kMaxMatches = 8;

// precisions whose contraction runs on the tensor cores
inline bool tc_precision(int precision) {
    return precision == ACOM_PREC_BF16 || precision == ACOM_PREC_FP16 ||
           precision == ACOM_PREC_FP8;
}
// bytes per tensor-core operand element
inline int tc_elem_bytes(int precision) { return precision == ACOM_PREC_FP8 ? 1 : 2; }
// make_bf16_map / launch_plan_to_bf16 operand kind: 0 BF16, 1 FP16, 2 E4M3
inline int tc_kind(int precision) {
    return precision == ACOM_PREC_FP8 ? 2 : (precision == ACOM_PREC_FP16 ? 1 : 0);
}

}  // namespace acom

struct acom_plan_s {
    int device = 0;
    int Z = 0, S = 0, N = 0, F = 0, Spad = 0, Zp = 0, G = 0;
    double delta = 0, gamma_pow = 1, omega = 1, lambda = 0, q_max = 0, sigma_exc = 0;
    double step_deg = 0, dq = 0;
    int precision = ACOM_PREC_FP32;
    std::vector<double> za_host;      // [Z][3]
    // device memory
    float* Pr = nullptr;              // [Zp][F][Spad], zero rows beyond Z
    float* Pi = nullptr;
    float* Psr = nullptr;             // [Zp][Spad][Fs] (exact evaluation)
    float* Psi = nullptr;
    double* za = nullptr;             // [Z][3]
    double* frames = nullptr;         // [Z][9]
    int* nbr_ptr = nullptr;           // [Z + 1]
    int* nbr_idx = nullptr;
    double* refl_g = nullptr;         // [G][3]
    double* refl_amp = nullptr;       // [G]
    int* err = nullptr;               // device error word
    float* pfmax = nullptr;           // [F] max over axes of ||P^_zf|| over shells
    float pscale = 1.0f;              // 2^k of the FP16 plan spectra (1 otherwise)
    uint32_t* smask = nullptr;        // [Zp][Spad / 32] bit s: shell row s of the axis not zero
    // tensor-core operand, BF16 / FP16 / E4M3 of 2^k P^: [F][Zp / 128][256][Spad],
    // each 128-axis tile's real rows followed by its imaginary rows, so that one
    // TMA box of 256 rows is the whole B operand of an MMA
    void* Pb = nullptr;
    alignas(64) unsigned char map_p[128];   // TMA map of Pb (boxes of 256 rows)
    alignas(64) unsigned char map_p128[128];  // the same with boxes of 128 rows (CTA pairs)
    // first shell of the tensor-core contraction's K range: the lowest shell
    // (rounded down to a multiple of 16) where some axis' plan row is not
    // zero; the products below it are zero for every axis and pattern
    int k0 = 0;
    float4* refl_tab = nullptr;       // [G] FP32 (g, |g|^gamma |F_g|^omega) for refinement
    unsigned long long* refine_pairs = nullptr;  // (reflection, peak) pairs of the last refine
    int64_t last_refine_pairs = 0;
    int n_phases = 1;                 // crystal structures (phases) in this plan
    std::vector<int> phase_off_host;  // [n_phases + 1] first axis of each phase, then Z
    int* phase_off = nullptr;         // the same on the device
    int64_t last_evaluated = 0;       // axes evaluated exactly in the last match
    int* host_words = nullptr;        // pinned [2]: error word and evaluations of the last
                                      // match (read by acom_sync / acom_match)
    int64_t async_exhaustive_evals = -1;  // exhaustive: evaluations of the last match
    size_t bytes = 0;
    acom::Workspace ws;
};

namespace acom {

// ---- per-kernel timing and launch count (profile.cu) ----
enum KernelClass {
    kKReflections, kKRasterPlan, kKScale, kKRasterPatterns, kKContract, kKIdft, kKRefine,
    kKMisc, kKContractBf16, kKIdftBf16, kKRescore, kKSelect, kKRefineOrient, kKCount
};
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st);
void prof_resolve();
void prof_suppress(bool on);   // this thread's launches record no events (no event creation)

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per kernel, device and
// size: repeated launches make no host attribute call (stream capture).
// Process-global, not thread-safe.
inline void set_max_dynamic_smem(const void* func, size_t bytes) {
    struct Done {
        const void* f;
        int dev;
        size_t bytes;
    };
    static std::vector<Done> done;
    int dev = 0;
    cudaGetDevice(&dev);
    for (auto& d : done)
        if (d.f == func && d.dev == dev) {
            if (d.bytes >= bytes) return;
            cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            d.bytes = bytes;
            return;
        }
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done.push_back({func, dev, bytes});
}

// ---- error reporting (api.cu) ----
acom_status set_error(acom_status s, const std::string& msg);
acom_status cuda_error(cudaError_t e, const char* what);
void clear_error();                 // acom_last_error() returns "" afterwards
void count_allocation();            // one device or pinned allocation requested
// device check that row_ptr[0] == 0 (sets kErrRowPtr in err); allocates nothing
void launch_check_row0(const int64_t* row_ptr, int* err, cudaStream_t st);

// ---- launchers (defined in the .cu files) ----
// plan.cu
acom_status build_plan_device(acom_plan_s* p, const acom_crystal* crystal, cudaStream_t st);
// raster.cu
void launch_raster_plan(const RasterGeom& geo, const PlanSource& src, int Z,
                        const RasterOut& out, int* err, cudaStream_t st);
void launch_raster_patterns(const RasterGeom& geo, const PatternSource& src,
                            const RasterOut& out, int* err, cudaStream_t st);
void launch_scale_rows(float* re, float* im, const float* sumsq, int items, int row_elems,
                       cudaStream_t st);
void launch_spectra_export(const float* re, const float* im, int items, int F, int Spad, int S,
                           float* dst, cudaStream_t st);
size_t raster_smem_bytes(int N, int F);
// match_fp32.cu
void launch_contract_fp32(const acom_plan_s* p, const float* Xr, const float* Xi, int nb,
                          float* Chat, int chunk, cudaStream_t st);
void launch_idft_argmax_fp32(const acom_plan_s* p, const float* Chat, int nb, int chunk,
                             float* za_scores, unsigned long long* best, cudaStream_t st);
// match_prune.cu
void launch_contract_bound_fp32(const acom_plan_s* p, const float* Xr, const float* Xi, int nb,
                                float* U, cudaStream_t st);
void launch_plan_fnorm_max(const acom_plan_s* p, float* out, cudaStream_t st);
// p->smask from the plan's shell-major spectra (p->smask allocated, Zp x Spad/32)
void launch_plan_shell_mask(const acom_plan_s* p, cudaStream_t st);
// match_tc.cu
acom_status make_bf16_map(void* map_storage, const void* base, uint64_t rows, uint64_t cols,
                          int kind = 0, int box_rows = 128);
void launch_half_to_e4m3(const void* src, void* dst, int64_t n, float mul, cudaStream_t st);
// budget in clock cycles of the tensor-core contraction's pipeline waits (0: default)
void set_wait_cycles(long long cycles);
// xscale: per-pattern 2^e of FP16 pattern spectra (nullptr: BF16, no scale)
// cta_pairs: 0 one CTA per MMA (cta_group::1), 1 CTA pairs (cta_group::2)
void launch_contract_bound_tc(const acom_plan_s* p, const void* map_x, int pt_stride, int nb,
                              float* U, cudaStream_t st, const float* xscale = nullptr,
                              int tile_order = 0, int cta_pairs = 0);
// the plan's FP32 spectra Pr, Pi [Zp][F][Spad] -> the merged operand p->Pb:
// BF16 of P^ (kind 0), FP16 (1) or E4M3 (2) of scale * P^
void launch_plan_to_operand(const float* Pr, const float* Pi, int Zp, int F, int Spad, void* dst,
                            cudaStream_t st, int kind, float scale);
void launch_orient_compose(const acom_plan_s* p, const OrientIn* oin, int nb, int refine,
                           acom_result out, int64_t off, cudaStream_t st);
void launch_select_exact(const acom_plan_s* p, const float* Xsr, const float* Xsi, const float* U,
                         const float* xfn, const int2* srange, const uint32_t* rmask,
                         const float* pfmax, const float* xnorm2, int nb,
                         float kappa, int refine, acom_result out, int64_t off, int* n_eval,
                         cudaStream_t st, const float* xscale, int rescore_top, OrientIn* oin);
// refine.cu: continuous refinement on the plan's reflections
acom_status refine_table(acom_plan_s* p, cudaStream_t st);
void launch_refine_orient(const acom_plan_s* p, const acom_peaks_csr* pk, int steps,
                          float rho_start, float rho_end, float damping, float max_step, int twin,
                          float* orient, const float* orient_alt, float* score, uint8_t* start_out,
                          cudaStream_t st);
void launch_kin_score(const acom_plan_s* p, const acom_peaks_csr* pk, const float* orient,
                      const float* r, const float* strain, float rho, float* score, float* grad,
                      float* gn, float* strain_grad, cudaStream_t st);
// multimatch.cu: peak deletion after a match, full-pattern score at a match
void launch_delete_peaks(const acom_plan_s* p, const acom_peaks_csr* work, const acom_result& r,
                         float r_del, float d_min, cudaStream_t st);
void launch_score_at(const acom_plan_s* p, const float* Xsr, const float* Xsi, const int2* srange,
                     const float* xnorm2, int nb, const acom_result* res, int n_matches,
                     int64_t off, cudaStream_t st);
// exhaustive mode: phase of each winner and each phase's best score
void launch_phase_outputs(const acom_plan_s* p, const float* za_scores, int nb, acom_result out,
                          int64_t off, cudaStream_t st);
void launch_refine(const acom_plan_s* p, const float* Chat, int nb, int chunk,
                   const float* za_scores, const unsigned long long* best, const float* xnorm2,
                   int refine, acom_result out, int64_t out_offset, cudaStream_t st);

// Order-preserving map of a float to an unsigned key: larger float -> larger key.
__host__ __device__ inline unsigned int float_order_key(float v) {
    unsigned int u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(v);
#else
    memcpy(&u, &v, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ inline float float_from_order_key(unsigned int k) {
    unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float v;
#ifdef __CUDA_ARCH__
    v = __uint_as_float(u);
#else
    memcpy(&v, &u, 4);
#endif
    return v;
}

// Packed (score, index) key: max over keys = max score, then lowest index.
__host__ __device__ inline unsigned long long pack_best(float score, unsigned int index) {
    return ((unsigned long long)float_order_key(score) << 32) |
           (unsigned long long)(0xffffffffu - index);
}

}  // namespace acom
