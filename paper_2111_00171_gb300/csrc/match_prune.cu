// Certified pruning of the correlation step.
//
// For a zone axis z and a pattern b the correlations over phi3 are inverse
// transforms of the spectra c_f = sum_s FFT{P}^*_sf FFT{X}_sf (direct) and of
// its mirror counterpart, so for every bin k
//
//   C[k] = (1/N) sum_f w_f Re(c_f e^{2 pi i f k / N}) <= (1/N) sum_f w_f |c_f|
//
// (w_0 = w_{N/2} = 1, else 2).  The contraction kernels reduce every (z, b)
// pair to U = (1/N) sum_f w_f max(|c_f^dir|, |c_f^mir|), which bounds both
// correlations at once, while the spectra are on chip; the full
// correlation of an axis is then evaluated (in FP32) only while its bound can
// still beat the best score found so far.  Rounding of the contraction is
// covered by a margin E_b = kappa (1/N) sum_f w_f max_z ||P^_zf|| ||X^_bf||,
// which bounds |c_f(computed) - c_f(exact)| for every axis through
// Cauchy-Schwarz over the shells.  The winner is the same as that of the
// exhaustive evaluation (up to FP32 ties).
#include <math_constants.h>

#include <cmath>

#include "acom_internal.cuh"
#include "fft_warp.cuh"

namespace acom {

// ---------------------------------------------------------------------------
// FP32 contraction with the bound epilogue.  CTA tile: 64 zone axes x 64
// patterns, all frequencies; thread tile 4 x 4 pairs.
// ---------------------------------------------------------------------------
constexpr int kBz = 64, kBb = 64, kBk = 16;

__global__ void __launch_bounds__(256)
k_contract_bound_fp32(const float* __restrict__ Pr, const float* __restrict__ Pi,
                      const float* __restrict__ Xr, const float* __restrict__ Xi, int F, int N,
                      int Spad, int Z, int nb, float* __restrict__ U) {
    __shared__ __align__(16) float sPr[kBk][kBz + 4];
    __shared__ __align__(16) float sPi[kBk][kBz + 4];
    __shared__ __align__(16) float sXr[kBk][kBb + 4];
    __shared__ __align__(16) float sXi[kBk][kBb + 4];
    const int z0 = blockIdx.x * kBz, b0 = blockIdx.y * kBb;
    const int t = threadIdx.x, tz = t & 15, tb = t >> 4;
    const int lr = t >> 2, lc = (t & 3) * 4;
    const bool bvalid = (b0 + lr) < nb;
    float Ud[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Ud[i][j] = 0.f;

    for (int f = 0; f < F; ++f) {
        float A[4][4], B[4][4], C[4][4], D[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) A[i][j] = B[i][j] = C[i][j] = D[i][j] = 0.f;
        const int64_t prow = ((int64_t)(z0 + lr) * F + f) * Spad;
        const int64_t xrow = ((int64_t)(b0 + lr) * F + f) * Spad;
        for (int s0 = 0; s0 < Spad; s0 += kBk) {
            float4 pr = *reinterpret_cast<const float4*>(Pr + prow + s0 + lc);
            float4 pi = *reinterpret_cast<const float4*>(Pi + prow + s0 + lc);
            float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), xi = xr;
            if (bvalid) {
                xr = *reinterpret_cast<const float4*>(Xr + xrow + s0 + lc);
                xi = *reinterpret_cast<const float4*>(Xi + xrow + s0 + lc);
            }
            __syncthreads();
            sPr[lc + 0][lr] = pr.x; sPr[lc + 1][lr] = pr.y; sPr[lc + 2][lr] = pr.z; sPr[lc + 3][lr] = pr.w;
            sPi[lc + 0][lr] = pi.x; sPi[lc + 1][lr] = pi.y; sPi[lc + 2][lr] = pi.z; sPi[lc + 3][lr] = pi.w;
            sXr[lc + 0][lr] = xr.x; sXr[lc + 1][lr] = xr.y; sXr[lc + 2][lr] = xr.z; sXr[lc + 3][lr] = xr.w;
            sXi[lc + 0][lr] = xi.x; sXi[lc + 1][lr] = xi.y; sXi[lc + 2][lr] = xi.z; sXi[lc + 3][lr] = xi.w;
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kBk; ++kk) {
                float4 a_r = *reinterpret_cast<const float4*>(&sPr[kk][tz * 4]);
                float4 a_i = *reinterpret_cast<const float4*>(&sPi[kk][tz * 4]);
                float4 b_r = *reinterpret_cast<const float4*>(&sXr[kk][tb * 4]);
                float4 b_i = *reinterpret_cast<const float4*>(&sXi[kk][tb * 4]);
                const float ar[4] = {a_r.x, a_r.y, a_r.z, a_r.w};
                const float ai[4] = {a_i.x, a_i.y, a_i.z, a_i.w};
                const float br[4] = {b_r.x, b_r.y, b_r.z, b_r.w};
                const float bi[4] = {b_i.x, b_i.y, b_i.z, b_i.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        A[i][j] = fmaf(ar[i], br[j], A[i][j]);
                        B[i][j] = fmaf(ai[i], bi[j], B[i][j]);
                        C[i][j] = fmaf(ar[i], bi[j], C[i][j]);
                        D[i][j] = fmaf(ai[i], br[j], D[i][j]);
                    }
            }
        }
        const float w = (f == 0 || 2 * f == N) ? 1.f : 2.f;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // max(|c_dir|, |c_mir|)^2 = p + 2 |AB - CD|, p = A^2 + B^2 + C^2 + D^2
                const float a_ = A[i][j], b_ = B[i][j], c_ = C[i][j], d_ = D[i][j];
                const float p = fmaf(a_, a_, fmaf(b_, b_, fmaf(c_, c_, d_ * d_)));
                const float q = fmaf(a_, b_, -c_ * d_);
                Ud[i][j] = fmaf(w, sqrtf(fmaf(2.0f, fabsf(q), p)), Ud[i][j]);
            }
    }
    const float invN = 1.0f / (float)N;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = b0 + tb * 4 + j;
        if (b >= nb) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int z = z0 + tz * 4 + i;
            if (z < Z) U[(int64_t)b * Z + z] = Ud[i][j] * invN;
        }
    }
}

void launch_contract_bound_fp32(const acom_plan_s* p, const float* Xr, const float* Xi, int nb,
                                float* U, cudaStream_t st) {
    dim3 grid(p->Zp / kBz, (nb + kBb - 1) / kBb);
    prof_begin(kKContract, st);
    k_contract_bound_fp32<<<grid, 256, 0, st>>>(p->Pr, p->Pi, Xr, Xi, p->F, p->N, p->Spad, p->Z,
                                                nb, U);
    prof_end(kKContract, st);
}

// ---------------------------------------------------------------------------
// max over zone axes of ||P^_zf||_2 (over shells), per frequency, times
// 1.0001 for the rounding of the norm itself: one warp per (axis, frequency)
// row, lanes over the shells; the maximum of non-negative floats by an
// integer atomicMax on their bit patterns (out cleared to +0 first)
__global__ void k_plan_fnorm_max(const float* __restrict__ Pr, const float* __restrict__ Pi,
                                 int Z, int F, int Spad, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= (int64_t)Z * F) return;
    const int f = (int)(row % F);
    const float* pr = Pr + row * Spad;
    const float* pi = Pi + row * Spad;
    float a = 0.f;
    for (int s = lane; s < Spad; s += 32) a = fmaf(pr[s], pr[s], fmaf(pi[s], pi[s], a));
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) atomicMax(reinterpret_cast<int*>(out) + f, __float_as_int(sqrtf(a) * 1.0001f));
}

// bit s of word [z][s / 32]: shell row s of axis z (re or im) has a non-zero
// entry; one warp per row
__global__ void k_plan_shell_mask(const float* __restrict__ Pr, const float* __restrict__ Pi,
                                  int64_t rows, int Spad, int Fs, uint32_t* __restrict__ mask) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    bool nz = false;
    for (int f = lane; f < Fs; f += 32) nz |= Pr[row * Fs + f] != 0.f || Pi[row * Fs + f] != 0.f;
    if (__any_sync(0xffffffffu, nz) && lane == 0) {
        const int64_t z = row / Spad;
        const int s = (int)(row - z * Spad);
        atomicOr(mask + z * (Spad >> 5) + (s >> 5), 1u << (s & 31));
    }
}

void launch_plan_shell_mask(const acom_plan_s* p, cudaStream_t st) {
    const int64_t rows = (int64_t)p->Zp * p->Spad;
    cudaMemsetAsync(p->smask, 0, sizeof(uint32_t) * (size_t)p->Zp * (p->Spad / 32), st);
    prof_begin(kKMisc, st);
    k_plan_shell_mask<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(
        p->Psr, p->Psi, rows, p->Spad, shell_row_stride(p->F), p->smask);
    prof_end(kKMisc, st);
}

void launch_plan_fnorm_max(const acom_plan_s* p, float* out, cudaStream_t st) {
    const int64_t rows = (int64_t)p->Z * p->F;
    cudaMemsetAsync(out, 0, sizeof(float) * (size_t)p->F, st);
    prof_begin(kKMisc, st);
    k_plan_fnorm_max<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(p->Pr, p->Pi, p->Z, p->F, p->Spad,
                                                                   out);
    prof_end(kKMisc, st);
}

// ---------------------------------------------------------------------------
// Selection and exact evaluation.  Persistent CTAs take the patterns in turn.
// The candidate axes of a pattern are evaluated in batches of up to kBatch:
//  * spectra: thread (shell part, candidate, frequency quad) runs down its
//    share of the pattern's non-zero shells with 16-byte loads of the
//    shell-major rows (four frequencies at once; the pattern's rows are shared
//    by the candidates through L1) and accumulates the four real products;
//    the shell parts are summed in shared memory;
//  * transform: one warp per candidate takes the inverse transform along phi3
//    of c_dir + i c_mir (both correlations are real, so one complex transform
//    carries both) and the argmax over (phi3, mirror);
//  * selection: a block-wide top-K of the pending bounds, two barriers.
// ---------------------------------------------------------------------------
constexpr int kSelThreads = 256;
constexpr int kSelWarps = kSelThreads / 32;
constexpr int kBatch = 8;

struct SelState {
    float T;             // best exact score so far
    unsigned Tidx;       // (z * 2 + mirror) * N + k of the best
    int bz, bk, bm;      // its axis, bin and mirror flag
    int nc;              // candidates of the current main batch
    int nref;            // candidates of the current refinement batch (a field of
                         // its own: thread 0 fills it right after the main loop's
                         // last barrier, while slower threads may still read nc)
    int q;               // next neighbour to consider (refinement batches)
    float best3[3];      // winning correlation at bins k - 1, k, k + 1
    float Emax;          // rounding margin of the bounds
    float next_u;        // bound of the best pending axis after a batch's picks
    float Tp[kMaxPhases];  // best exact score so far of each phase
    int ru_z;            // runner-up: best evaluated axis outside the winner's
    float ru_v;          // grid neighbourhood (-1: none), and its score
};

struct SelSmem {
    float2* tw;      // [N] (cos, sin)(2 pi i / N)
    float2* y;       // [kBatch][N] spectra of the batch, transformed in place
    float2* yt;      // [kBatch][N] transform ping-pong (shares space with part)
    float4* part;    // [items][4] partial (A, B, C, D) of a shell part
    float* U;        // [Z] bound, replaced by the exact score once evaluated
    uint8_t* ev;     // [Z] 0 pending, 1 evaluated, 2 in the current batch
    uint16_t* kb;    // [Z] bin + mirror * N of each evaluated axis' maximum
    float* wv;       // [kSelWarps][kBatch] per-warp top-K values
    int* wi;         // [kSelWarps][kBatch] and axes
    int* cand;       // [kBatch]
    float* res;      // [kBatch][5] best value, its index bits, values at k - 1, k, k + 1
    float* red;      // [2][kSelWarps]
    int* poff;       // [kMaxPhases + 1] first axis of each phase, then Z
    uint32_t* pmask; // [Spad / 32] shells the pattern's tents reach: its rows that may
                     // be non-zero, and the only ones the raster wrote
    uint16_t* slist; // [kBatch][Spad] shells of each candidate: pattern and plan rows both
                     // not zero
    int* slen;       // [kBatch]
    // N = 360: the spectra rows hold frequency f at perm[f] (the prime-factor
    // transform's input order), and the transform leaves bin k at pout[k]
    uint16_t* perm;
    uint16_t* pout;
    SelState* st;
};

// Phase of axis z: the last p with poff[p] <= z.
__device__ __forceinline__ int phase_of(const int* poff, int nph, int z) {
    int p = 0;
    while (p + 1 < nph && z >= poff[p + 1]) ++p;
    return p;
}

__device__ inline bool better(float v, unsigned i, float bv, unsigned bi) {
    return v > bv || (v == bv && i < bi);
}

__device__ inline void warp_argmax(float& v, unsigned& i) {
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const unsigned oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
}

// The up to K pending axes (ev == 0) of largest bound with U rel + Emax >= thr
// (with per_phase, thr is the best score so far of the axis' own phase), in
// decreasing bound (ties: lowest axis), into cand and st->nc; marks them
// ev = 2.  Each warp takes its K best by repeated argmax over entries strictly
// below its previous pick; warp 0 merges the warps' lists the same way.
__device__ void block_topk(SelSmem& sm, int Z, int K, float thr, float rel, float Emax,
                           bool per_phase, int nph, bool want_next = false) {
    // with want_next, one more round finds the best pending axis after the K
    // picks (K < kBatch): its bound goes to st->next_u (-inf: none), unpicked
    const int Kr = K + (want_next ? 1 : 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float lv = CUDART_INF_F;
    unsigned li = 0u;                       // previous pick (nothing is above it)
    for (int r = 0; r < Kr; ++r) {
        float v = -CUDART_INF_F;
        unsigned zi = 0xffffffffu;
        for (int z = warp * 32 + lane; z < Z; z += kSelThreads) {
            if (sm.ev[z] != 0) continue;
            const float u = sm.U[z];
            const float tz = per_phase ? sm.st->Tp[phase_of(sm.poff, nph, z)] : thr;
            if (u * rel + Emax < tz || !better(lv, li, u, (unsigned)z)) continue;
            if (better(u, (unsigned)z, v, zi)) {
                v = u;
                zi = (unsigned)z;
            }
        }
        warp_argmax(v, zi);
        if (lane == 0) {
            sm.wv[warp * kBatch + r] = v;
            sm.wi[warp * kBatch + r] = (int)zi;
        }
        if (zi == 0xffffffffu) {
            for (int r2 = r + 1 + lane; r2 < Kr; r2 += 32) sm.wi[warp * kBatch + r2] = -1;
            break;
        }
        lv = v;
        li = zi;
    }
    __syncthreads();
    if (warp == 0) {
        const int ne = kSelWarps * Kr;
        lv = CUDART_INF_F;
        li = 0u;
        int n = 0;
        float next = -CUDART_INF_F;
        for (int r = 0; r < Kr; ++r) {
            float v = -CUDART_INF_F;
            unsigned zi = 0xffffffffu;
            for (int e = lane; e < ne; e += 32) {
                const int w = e / Kr, j = e - w * Kr;
                const int z = sm.wi[w * kBatch + j];
                if (z < 0) continue;
                const float u = sm.wv[w * kBatch + j];
                if (better(lv, li, u, (unsigned)z) && better(u, (unsigned)z, v, zi)) {
                    v = u;
                    zi = (unsigned)z;
                }
            }
            warp_argmax(v, zi);
            if (zi == 0xffffffffu) break;
            if (r == K) {                    // the best axis after the picks
                next = v;
                break;
            }
            if (lane == 0) {
                sm.cand[n] = (int)zi;
                sm.ev[zi] = 2;
            }
            ++n;
            lv = v;
            li = zi;
        }
        if (lane == 0) {
            sm.st->nc = n;
            sm.st->next_u = next;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void fma4(float4& acc, const float4 p, const float4 x) {
    acc.x = fmaf(p.x, x.x, acc.x);
    acc.y = fmaf(p.y, x.y, acc.y);
    acc.z = fmaf(p.z, x.z, acc.z);
    acc.w = fmaf(p.w, x.w, acc.w);
}

struct SelectArgs {
    const float *Psr, *Psi, *Xsr, *Xsi;   // FP32 spectra, shell-major [.][Spad][Fs]
    const float* U;                   // [nb][Z] bounds
    const float* xfn;                 // [nb][F] ||X^_bf||
    const int2* srange;               // [nb] non-zero shell range
    const uint32_t* rmask;            // [nb][Spad / 32] shells the pattern's tents reach
    const float* pfmax;               // [F] max_z ||P^_zf||
    const float* xnorm2;              // [nb] ||X||^2
    const double* za;                 // [Z][3]
    const double* frames;             // [Z][9]
    const int* nbr_ptr;
    const int* nbr_idx;
    const int* phase_off;             // [n_phases + 1]
    int n_phases;
    int Z, F, N, S, Spad, nb, refine;
    float kappa;                      // contraction rounding constant
    FftRadix rad;                     // inverse-transform factorisation
    acom_result out;
    int64_t off;
    int* n_eval;                      // optional: total axes evaluated
    const float* xscale;              // [nb] 2^e of FP16 pattern spectra, or nullptr
    float inv_pscale;                 // 2^-k of the plan operand's scale
    float xs_mul;                     // the pattern operand holds xscale * xs_mul times X^
    float eta;                        // absolute error of an operand below its normal range
    int rescore_top;                  // > 0: evaluate only the top axes by bound (no certificate)
    const uint32_t* smask;            // [Zp][Spad / 32] non-zero plan shells
    OrientIn* oin;                    // [nb] the winners, for k_orient_compose
    float eta_rs = 0.f;               // eta sqrt(Spad), from the host (FP64 there)
};

// Spectra c_dir + i c_mir of the batch's candidate axes, scaled by 1/N, into
// the rows y[c] (both halves of the conjugate-symmetric spectrum), stored as
// their complex conjugates.
template <bool PFA>
__device__ void batch_spectra(const SelectArgs& a, int64_t b, int nc, int s_lo, int s_hi,
                              SelSmem& sm) {
    const int F = a.F, N = a.N, Fq = shell_row_stride(F) >> 2;
    const int items = nc * Fq;
    const int len = s_hi - s_lo;
    int h = kSelThreads / items;
    h = h < 1 ? 1 : (h > 8 ? 8 : h);
    if (h > len) h = len > 1 ? len : 1;
    const int total = items * h;
    // each candidate's shells: rows of both the pattern and the axis not zero
    // (a product with a zero row is exactly 0 and is skipped); warp c lists
    // candidate c in increasing shell order
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, MW = a.Spad >> 5;
        for (int c = warp; c < nc; c += kSelWarps) {
            const uint32_t* pm = a.smask + (int64_t)sm.cand[c] * MW;
            const uint32_t m = lane < MW ? (sm.pmask[lane] & pm[lane]) : 0u;
            const int cnt = __popc(m);
            int off = cnt;                              // inclusive scan over the lanes
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, off, o);
                if (lane >= o) off += v;
            }
            const int tot = __shfl_sync(0xffffffffu, off, 31);
            off -= cnt;
            uint16_t* L = sm.slist + c * a.Spad;
            uint32_t mm = m;
            while (mm) {
                const int bit = __ffs(mm) - 1;
                mm &= mm - 1;
                L[off++] = (uint16_t)(32 * lane + bit);
            }
            if (lane == 0) sm.slen[c] = tot;
        }
        __syncthreads();
    }
    const int64_t blk = (int64_t)a.Spad * Fq;       // float4 per pattern or axis
    const float4* xr0 = reinterpret_cast<const float4*>(a.Xsr) + b * blk;
    const float4* xi0 = reinterpret_cast<const float4*>(a.Xsi) + b * blk;
    for (int idx = threadIdx.x; idx < total; idx += kSelThreads) {
        const int hh = idx / items, rem = idx - hh * items;
        const int c = rem / Fq, fq = rem - c * Fq;
        const uint16_t* L = sm.slist + c * a.Spad;
        const int ln = sm.slen[c];
        const int sa = (ln * hh) / h, se = (ln * (hh + 1)) / h;   // positions in the list
        const int64_t pb = (int64_t)sm.cand[c] * blk + fq;
        const float4* pr = reinterpret_cast<const float4*>(a.Psr) + pb;
        const float4* pi = reinterpret_cast<const float4*>(a.Psi) + pb;
        const float4* xr = xr0 + fq;
        const float4* xi = xi0 + fq;
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f), B = A, C = A, D = A;
        int i = sa;
        for (; i + 1 < se; i += 2) {
            const int o0 = L[i] * Fq, o1 = L[i + 1] * Fq;
            const float4 x1a = __ldg(xr + o0), x2a = __ldg(xi + o0);
            const float4 x1b = __ldg(xr + o1), x2b = __ldg(xi + o1);
            const float4 p1a = __ldg(pr + o0), p2a = __ldg(pi + o0);
            const float4 p1b = __ldg(pr + o1), p2b = __ldg(pi + o1);
            fma4(A, p1a, x1a);
            fma4(B, p2a, x2a);
            fma4(C, p1a, x2a);
            fma4(D, p2a, x1a);
            fma4(A, p1b, x1b);
            fma4(B, p2b, x2b);
            fma4(C, p1b, x2b);
            fma4(D, p2b, x1b);
        }
        if (i < se) {
            const int o0 = L[i] * Fq;
            const float4 x1 = __ldg(xr + o0), x2 = __ldg(xi + o0);
            const float4 p1 = __ldg(pr + o0), p2 = __ldg(pi + o0);
            fma4(A, p1, x1);
            fma4(B, p2, x2);
            fma4(C, p1, x2);
            fma4(D, p2, x1);
        }
        float4* q = sm.part + 4 * idx;
        q[0] = A;
        q[1] = B;
        q[2] = C;
        q[3] = D;
    }
    __syncthreads();
    const float invN = 1.0f / (float)N;
    for (int e = threadIdx.x; e < nc * F; e += kSelThreads) {
        const int c = e / F, f = e - c * F, l = f & 3;
        float A = 0.f, B = 0.f, C = 0.f, D = 0.f;
        for (int hh = 0; hh < h; ++hh) {
            const float* q = reinterpret_cast<const float*>(sm.part + 4 * (hh * items + c * Fq + (f >> 2)));
            A += q[l];
            B += q[4 + l];
            C += q[8 + l];
            D += q[12 + l];
        }
        const float dre = (A + B) * invN, dim = (C - D) * invN;
        const float mre = (A - B) * invN, mim = -(C + D) * invN;
        // stored conjugated: the inverse transform runs as a forward one
        float2* y = sm.y + c * N;
        y[PFA ? (int)sm.perm[f] : f] = make_float2(dre - mim, -(dim + mre));
        if (f > 0 && 2 * f < N) y[PFA ? (int)sm.perm[N - f] : N - f] = make_float2(dre + mim, dim - mre);
    }
    __syncthreads();
}

// One warp per candidate: C_dir[k] + i C_mir[k] = sum_f y_f exp(2 pi i f k / N),
// taken as the conjugate of the forward transform of conj(y) (the rows hold
// conj(y)); the argmax over
// (k, mirror) with the correlation at k - 1, k, k + 1 goes to res[c].
template <bool PFA>
__device__ void batch_transforms(const SelectArgs& a, int nc, SelSmem& sm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, N = a.N;
    for (int c = warp; c < nc; c += kSelWarps) {
        float2* row = sm.y + c * N;
        float2* alt = sm.yt + c * N;
        const float2* out;
        const uint16_t* pout = sm.pout;     // PFA: bin k at out[pout[k]]
        if constexpr (PFA) {
            warp_pfa360(row, nullptr, lane);
            out = row;
        } else if (a.rad.n > 0) {
            out = warp_fft_fixed(row, alt, N, a.rad, sm.tw, lane);
        } else {
            for (int k = lane; k < N; k += 32) {
                float2 acc = make_float2(0.f, 0.f);
                int idx = 0;
                for (int f = 0; f < N; ++f) {
                    const float2 t = cmul_conj(row[f], sm.tw[idx]);
                    acc.x += t.x;
                    acc.y += t.y;
                    idx += k;
                    if (idx >= N) idx -= N;
                }
                alt[k] = acc;
            }
            __syncwarp();
            out = alt;
        }
        float bv = -CUDART_INF_F;
        unsigned bi = 0xffffffffu;
        for (int k = lane; k < N; k += 32) {
            const float2 v = out[PFA ? (int)pout[k] : k];
            if (better(v.x, (unsigned)k, bv, bi)) {
                bv = v.x;
                bi = (unsigned)k;
            }
            if (better(-v.y, (unsigned)(N + k), bv, bi)) {
                bv = -v.y;
                bi = (unsigned)(N + k);
            }
        }
        warp_argmax(bv, bi);
        if (lane == 0) {
            const int m = (int)(bi / (unsigned)N), k = (int)bi - m * N;
            const int km = (k + N - 1) % N, kp = (k + 1) % N;
            const float2 ym = out[PFA ? (int)pout[km] : km], y0 = out[PFA ? (int)pout[k] : k],
                         yp = out[PFA ? (int)pout[kp] : kp];
            float* r = sm.res + 5 * c;
            r[0] = bv;
            r[1] = __uint_as_float(bi);
            r[2] = m ? -ym.y : ym.x;
            r[3] = m ? -y0.y : y0.x;
            r[4] = m ? -yp.y : yp.x;
        }
        __syncwarp();
    }
    __syncthreads();
}

// Record the batch's exact scores; with update, fold them into the best.
// Every score also updates its phase's best.
__device__ void fold_batch(int nc, int N, bool update, int nph, SelSmem& sm) {
    if (threadIdx.x == 0) {
        SelState& st = *sm.st;
        for (int c = 0; c < nc; ++c) {
            const int z = sm.cand[c];
            const float* r = sm.res + 5 * c;
            const float bv = r[0];
            float& tp = st.Tp[phase_of(sm.poff, nph, z)];
            tp = bv > tp ? bv : tp;
            const unsigned bi = __float_as_uint(r[1]);
            const unsigned gidx = (unsigned)z * 2u * (unsigned)N + bi;
            if (update && better(bv, gidx, st.T, st.Tidx)) {
                st.T = bv;
                st.Tidx = gidx;
                st.bz = z;
                st.bm = (int)(bi / (unsigned)N);
                st.bk = (int)(bi - (unsigned)st.bm * N);
                st.best3[0] = r[2];
                st.best3[1] = r[3];
                st.best3[2] = r[4];
            }
            sm.U[z] = bv;
            sm.kb[z] = (uint16_t)bi;
            sm.ev[z] = 1;
        }
    }
    __syncthreads();
}

__device__ inline void matmul3d(const double* a, const double* b, double* c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

// Outputs of the winner (warp 0).  For the orientation, the score-weighted
// sum of the neighbour axes within 0.9 of the best (the lanes take the
// neighbours and a butterfly sums them, so every lane holds the same FP64
// sum) and the correlation at bins k - 1, k, k + 1 go to oin[b]; the FP64
// composition runs in k_orient_compose, one thread per pattern, so that it
// does not hold up the block.
__device__ __noinline__ void write_outputs(const SelectArgs& a, int64_t b, const SelSmem& sm,
                                           bool want_ref, int lane) {
    const SelState& st = *sm.st;
    const int N = a.N, bz = st.bz, bk = st.bk, bm = st.bm;
    const float T = st.T;
    const int64_t o = a.off + b;
    const float score = T == -CUDART_INF_F ? 0.f : T;
    double a0 = 0, a1 = 0, a2 = 0;
    if (want_ref && a.refine) {
        for (int q = a.nbr_ptr[bz] + lane; q < a.nbr_ptr[bz + 1]; q += 32) {
            const int z2 = a.nbr_idx[q];
            if (!sm.ev[z2]) continue;             // its true score is below 0.9 of the best
            const float sc = sm.U[z2];
            if (sc >= 0.9f * T) {
                a0 += (double)sc * a.za[3 * z2];
                a1 += (double)sc * a.za[3 * z2 + 1];
                a2 += (double)sc * a.za[3 * z2 + 2];
            }
        }
        for (int w = 16; w > 0; w >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, w);
            a1 += __shfl_xor_sync(0xffffffffu, a1, w);
            a2 += __shfl_xor_sync(0xffffffffu, a2, w);
        }
    }
    if (lane != 0) return;
    a.out.za_idx[o] = bz;
    a.out.phi3_bin[o] = bk;
    a.out.mirror[o] = (uint8_t)bm;
    a.out.score[o] = score;
    if (a.out.phase) a.out.phase[o] = phase_of(sm.poff, a.n_phases, bz);
    if (a.out.runner_za || a.out.runner_score || a.out.runner_orient) {
        // the runner-up's grid orientation frame Rz(-2 pi k / N) [Ry(pi)] in
        // FP32 (a start for refinement); the winner's grid orientation when
        // there is no runner-up
        const int rz = st.ru_z;
        const int z = rz >= 0 ? rz : bz;
        const int kbz = rz >= 0 ? (int)sm.kb[rz] : bk + bm * N;
        const int mm = kbz >= N ? 1 : 0, kk = kbz - mm * N;
        if (a.out.runner_za) a.out.runner_za[o] = rz;
        if (a.out.runner_score) a.out.runner_score[o] = rz >= 0 ? st.ru_v : 0.f;
        if (a.out.runner_orient) {
            float sp, cp;
            sincospif(-2.0f * (float)kk / (float)N, &sp, &cp);
            const double* Fz = a.frames + 9 * z;
            for (int i = 0; i < 3; ++i) {
                const float f0 = (float)Fz[3 * i], f1 = (float)Fz[3 * i + 1], f2 = (float)Fz[3 * i + 2];
                float c0 = f0 * cp + f1 * sp, c1 = f1 * cp - f0 * sp, c2 = f2;
                if (mm) {
                    c0 = -c0;
                    c2 = -c2;
                }
                a.out.runner_orient[9 * o + 3 * i] = c0;
                a.out.runner_orient[9 * o + 3 * i + 1] = c1;
                a.out.runner_orient[9 * o + 3 * i + 2] = c2;
            }
        }
    }
    if (a.out.phase_score)
        for (int p = 0; p < a.n_phases; ++p)      // a phase left unevaluated: all-zero image
            a.out.phase_score[o * a.n_phases + p] = st.Tp[p] == -CUDART_INF_F ? 0.f : st.Tp[p];
    if (a.out.score_cos) {
        const float xn = sqrtf(a.xnorm2[b]);
        a.out.score_cos[o] = xn > 0.f ? score / xn : 0.f;
    }
    if (!want_ref) return;
    OrientIn& r = a.oin[b];
    r.w[0] = a0;
    r.w[1] = a1;
    r.w[2] = a2;
    r.c3[0] = st.best3[0];
    r.c3[1] = st.best3[1];
    r.c3[2] = st.best3[2];
    r.z = bz;
    r.km = bk + bm * N;
}

// Orientation of each winner, one thread per pattern: parabolic phi3 offset
// from the correlation at k - 1, k, k + 1; the zone axis refined toward the
// normalised score-weighted neighbour sum; m = T frame Rz(phi3) [Ry(pi)]
// composed in FP64.
__global__ void k_orient_compose(const OrientIn* __restrict__ oin, int nb, int N, int refine,
                                 const double* __restrict__ za, const double* __restrict__ frames,
                                 acom_result out, int64_t off) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const OrientIn r = oin[b];
    const int bz = r.z, bm = r.km >= N ? 1 : 0, bk = r.km - bm * N;
    const int64_t o = off + b;
    double dk = 0.0, wref[3];
    if (refine) {
        const double cm = r.c3[0], c0 = r.c3[1], cp = r.c3[2];
        const double den = cm - 2.0 * c0 + cp;
        if (den < 0.0) {
            dk = (cm - cp) / (2.0 * den);
            dk = dk > 0.5 ? 0.5 : (dk < -0.5 ? -0.5 : dk);
        }
        const double a0 = r.w[0], a1 = r.w[1], a2 = r.w[2];
        const double nrm = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        wref[0] = nrm > 0 ? a0 / nrm : za[3 * bz];
        wref[1] = nrm > 0 ? a1 / nrm : za[3 * bz + 1];
        wref[2] = nrm > 0 ? a2 / nrm : za[3 * bz + 2];
    } else {
        wref[0] = za[3 * bz];
        wref[1] = za[3 * bz + 1];
        wref[2] = za[3 * bz + 2];
    }
    const double phi3 = -2.0 * CUDART_PI * ((double)bk + dk) / (double)N;
    if (out.phi3) out.phi3[o] = (float)phi3;
    if (!out.orient) return;
    double Rz[9], m1[9], m2[9], Tm[9];
    double c3, s3;
    sincos(phi3, &s3, &c3);
    Rz[0] = c3; Rz[1] = -s3; Rz[2] = 0; Rz[3] = s3; Rz[4] = c3; Rz[5] = 0; Rz[6] = 0; Rz[7] = 0; Rz[8] = 1;
    matmul3d(frames + 9 * bz, Rz, m1);
    if (bm) {
        for (int i = 0; i < 3; ++i) {
            m1[3 * i] = -m1[3 * i];
            m1[3 * i + 2] = -m1[3 * i + 2];
        }
    }
    const double u0 = za[3 * bz], u1 = za[3 * bz + 1], u2 = za[3 * bz + 2];
    double ax0 = u1 * wref[2] - u2 * wref[1];
    double ax1 = u2 * wref[0] - u0 * wref[2];
    double ax2 = u0 * wref[1] - u1 * wref[0];
    const double sn = sqrt(ax0 * ax0 + ax1 * ax1 + ax2 * ax2);
    const double cs = u0 * wref[0] + u1 * wref[1] + u2 * wref[2];
    for (int i = 0; i < 9; ++i) Tm[i] = (i % 4 == 0) ? 1.0 : 0.0;
    if (sn > 1e-15) {
        ax0 /= sn; ax1 /= sn; ax2 /= sn;
        const double K[9] = {0, -ax2, ax1, ax2, 0, -ax0, -ax1, ax0, 0};
        double K2[9];
        matmul3d(K, K, K2);
        for (int i = 0; i < 9; ++i) Tm[i] += sn * K[i] + (1.0 - cs) * K2[i];
    }
    matmul3d(Tm, m1, m2);
    for (int i = 0; i < 9; ++i) out.orient[9 * o + i] = (float)m2[i];
}

void launch_orient_compose(const acom_plan_s* p, const OrientIn* oin, int nb, int refine,
                           acom_result out, int64_t off, cudaStream_t st) {
    if (nb <= 0) return;
    prof_begin(kKRefine, st);
    k_orient_compose<<<(nb + 127) / 128, 128, 0, st>>>(oin, nb, p->N, refine, p->za, p->frames,
                                                       out, off);
    prof_end(kKRefine, st);
}

__host__ __device__ inline size_t sel_items(int F) {
    const int Fq = shell_row_stride(F) >> 2;
    return (size_t)(kSelThreads > kBatch * Fq ? kSelThreads : kBatch * Fq);
}

// PFA: N = 360 with the prime-factor inverse transform, compiled alone (the
// radix transforms' code stays out of this kernel).  FULL: per-phase
// certificates, top-K rescoring or the runner-up may be asked for; without
// them the kernel carries only the one-certificate search and the winner's
// neighbours (a smaller kernel runs faster).
template <bool PFA, bool FULL>
__global__ void __launch_bounds__(kSelThreads, 3) k_select_exact(SelectArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Z = a.Z, F = a.F, N = a.N;
    SelSmem sm;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = smem_raw + off;
        off += (bytes + 15) & ~(size_t)15;
        return p;
    };
    sm.tw = reinterpret_cast<float2*>(take(sizeof(float2) * N));
    sm.y = reinterpret_cast<float2*>(take(sizeof(float2) * kBatch * N));
    {
        const size_t pb = sizeof(float4) * 4 * sel_items(F), yb = sizeof(float2) * kBatch * N;
        unsigned char* shared_area = take(pb > yb ? pb : yb);
        sm.part = reinterpret_cast<float4*>(shared_area);
        sm.yt = reinterpret_cast<float2*>(shared_area);
    }
    sm.U = reinterpret_cast<float*>(take(sizeof(float) * Z));
    sm.wv = reinterpret_cast<float*>(take(sizeof(float) * kSelWarps * kBatch));
    sm.wi = reinterpret_cast<int*>(take(sizeof(int) * kSelWarps * kBatch));
    sm.cand = reinterpret_cast<int*>(take(sizeof(int) * kBatch));
    sm.res = reinterpret_cast<float*>(take(sizeof(float) * 5 * kBatch));
    sm.red = reinterpret_cast<float*>(take(sizeof(float) * 2 * kSelWarps));
    sm.poff = reinterpret_cast<int*>(take(sizeof(int) * (kMaxPhases + 1)));
    sm.pmask = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (a.Spad >> 5)));
    sm.slist = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * kBatch * a.Spad));
    sm.slen = reinterpret_cast<int*>(take(sizeof(int) * kBatch));
    sm.perm = sm.pout = nullptr;
    if (PFA) {
        sm.perm = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * 360));
        sm.pout = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * 360));
    }
    sm.st = reinterpret_cast<SelState*>(take(sizeof(SelState)));
    sm.ev = take(Z);
    sm.kb = reinterpret_cast<uint16_t*>(take(sizeof(uint16_t) * Z));
    const int nph = a.n_phases;
    for (int i = threadIdx.x; i <= nph; i += kSelThreads) sm.poff[i] = a.phase_off[i];
    // with per-phase scores requested, every phase's best is certified
    const bool per_phase = FULL && a.out.phase_score != nullptr && nph > 1;
    const int rescore_top = FULL ? a.rescore_top : 0;

    for (int i = threadIdx.x; i < N; i += kSelThreads) {
        if constexpr (PFA) {
            sm.perm[i] = (uint16_t)pfa360_in(i);
            sm.pout[i] = (uint16_t)pfa360_out(i);
        } else {
            double s, c;
            sincospi(2.0 * (double)i / (double)N, &s, &c);
            sm.tw[i] = make_float2((float)c, (float)s);
        }
    }
    const float rel = 1.0f + 1e-5f;     // FP32 accumulation of U and of the scores
    const bool want_ref = (a.out.phi3 != nullptr) || (a.out.orient != nullptr);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int64_t b = blockIdx.x; b < a.nb; b += gridDim.x) {
        for (int z = threadIdx.x; z < Z; z += kSelThreads) {
            sm.U[z] = a.U[b * Z + z];
            sm.ev[z] = 0;
        }
        // the shells some peak's tent reached (recorded by the raster, which
        // wrote only those rows; every other row of the pattern is zero)
        for (int w = threadIdx.x; w < (a.Spad >> 5); w += kSelThreads)
            sm.pmask[w] = a.rmask[b * (a.Spad >> 5) + w];
        // E_b: rounding margin valid for every axis (its partial sums load
        // together with the bounds, before the first barrier).  FP16 operands add an
        // absolute term for values below the normal range: an operand x is off
        // by at most 2^-11 |x| + eta, so a dot product over Spad shells of
        // 2^e X^ and 2^k P^ gains eta sqrt(Spad) (2^e ||X^_bf|| + 2^k ||P^_zf||)
        // + Spad eta^2, i.e. after dividing by 2^(e+k)
        //   eta sqrt(Spad) (||X^_bf|| 2^-k + ||P^_zf|| 2^-e + sqrt(Spad) eta 2^-(e+k)),
        // charged four times for the four real products of c_f
        const float inv_sc = a.xscale ? 1.0f / (a.xscale[b] * a.xs_mul) : 0.f;
        const float tiny = a.eta_rs * inv_sc * a.inv_pscale;
        float e = 0.f, ea = 0.f;
        for (int f = threadIdx.x; f < F; f += kSelThreads) {
            const float w = (f == 0 || 2 * f == N) ? 1.f : 2.f;
            e = fmaf(w * a.pfmax[f], a.xfn[b * F + f], e);
            ea = fmaf(w, a.xfn[b * F + f] * a.inv_pscale + a.pfmax[f] * inv_sc + tiny, ea);
        }
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            ea += __shfl_xor_sync(0xffffffffu, ea, o);
        }
        if (lane == 0) {
            sm.red[warp] = e;
            sm.red[kSelWarps + warp] = ea;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f, ta = 0.f;
            for (int w = 0; w < kSelWarps; ++w) {
                t += sm.red[w];
                ta += sm.red[kSelWarps + w];
            }
            SelState& st = *sm.st;
            const float abs_term =
                a.xscale ? 4.0f * a.eta_rs * ta : 0.f;
            st.Emax = (a.kappa * t + abs_term) / (float)N * 1.01f;
            st.T = -CUDART_INF_F;
            st.Tidx = 0xffffffffu;
            st.bz = st.bk = st.bm = 0;
            st.best3[0] = st.best3[1] = st.best3[2] = 0.f;
            for (int p = 0; p < kMaxPhases; ++p) st.Tp[p] = -CUDART_INF_F;
        }
        __syncthreads();
        const float Emax = sm.st->Emax;
        const int2 sr = a.srange[b];
        int evals = 0;
        // Three stages share one evaluation site (one copy of the batch code):
        //  0 search: batches in decreasing bound, the first the 2 largest
        //    bounds, later ones every axis whose bound can still reach the best
        //    exact score (rescore_top: the top axes by bound only);
        //  1 the winner's grid neighbours that may reach 0.9 of the best (their
        //    exact scores weight the orientation refinement);
        //  2 the runner-up: the best axis outside the winner and its grid
        //    neighbours (bit 4 of ev marks them meanwhile), certified like the
        //    winner.
        const bool single = !per_phase && rescore_top == 0;
        const bool want_ru = FULL && (a.out.runner_za || a.out.runner_score || a.out.runner_orient);
        int stage = 0, batch = 0;
        for (;;) {
            int nc = 0;
            bool update = false;
            if (stage == 0) {
                const int left = rescore_top - evals;
                if (rescore_top == 0 || left > 0) {
                    const float thr =
                        (batch == 0 || rescore_top > 0) ? -CUDART_INF_F : sm.st->T;
                    const int K = rescore_top > 0 ? (left < kBatch ? left : kBatch)
                                                  : (batch == 0 ? 2 : kBatch);
                    // the first batch also finds the best bound after its picks:
                    // when that cannot reach the batch's best score, no later batch
                    // would find a candidate and the search ends without a scan
                    block_topk(sm, Z, K, thr, rel, Emax,
                               per_phase && batch > 0 && rescore_top == 0, nph,
                               single && batch == 0);
                    nc = sm.st->nc;
                }
                update = true;
            } else if (stage == 1) {
                // thread 0 gathers the next batch of neighbours; all threads run it
                const float T = sm.st->T;
                if (threadIdx.x == 0) {
                    const int qe = a.nbr_ptr[sm.st->bz + 1];
                    int q = sm.st->q, n = 0;
                    for (; q < qe && n < kBatch; ++q) {
                        const int z2 = a.nbr_idx[q];
                        if (sm.ev[z2] || sm.U[z2] * rel + Emax < 0.9f * T) continue;
                        sm.cand[n++] = z2;
                        sm.ev[z2] = 2;
                    }
                    sm.st->q = q;
                    sm.st->nref = n;
                }
                __syncthreads();
                nc = sm.st->nref;
            } else if (FULL && stage == 2) {
                // the best evaluated axis outside the neighbourhood so far
                float v = -CUDART_INF_F;
                unsigned zi = 0xffffffffu;
                for (int z = threadIdx.x; z < Z; z += kSelThreads)
                    if (sm.ev[z] == 1 && better(sm.U[z], (unsigned)z, v, zi)) {
                        v = sm.U[z];
                        zi = (unsigned)z;
                    }
                warp_argmax(v, zi);
                if (lane == 0) {
                    sm.wv[warp * kBatch] = v;
                    sm.wi[warp * kBatch] = (int)zi;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    float bv = -CUDART_INF_F;
                    unsigned bi = 0xffffffffu;
                    for (int w = 0; w < kSelWarps; ++w)
                        if (better(sm.wv[w * kBatch], (unsigned)sm.wi[w * kBatch], bv, bi)) {
                            bv = sm.wv[w * kBatch];
                            bi = (unsigned)sm.wi[w * kBatch];
                        }
                    sm.st->ru_z = bi == 0xffffffffu ? -1 : (int)bi;
                    sm.st->ru_v = bv;
                }
                __syncthreads();
                const bool have = sm.st->ru_z >= 0;
                // an all-zero image: every axis ties at 0, nothing to certify
                if (!(have && sm.st->T == 0.f && sm.st->Tidx == 0u)) {
                    block_topk(sm, Z, have ? kBatch : 2, have ? sm.st->ru_v : -CUDART_INF_F,
                               rel, Emax, false, nph);
                    nc = sm.st->nc;
                }
            } else {
                break;
            }
            if (nc > 0) {
                batch_spectra<PFA>(a, b, nc, sr.x, sr.y, sm);
                batch_transforms<PFA>(a, nc, sm);
                fold_batch(nc, N, update, nph, sm);
                evals += nc;
            }
            bool next = nc == 0;
            if (stage == 0 && nc > 0) {
                ++batch;
                // an all-zero image: every axis ties at 0 and the lowest index has won
                if (sm.st->T == 0.f && sm.st->Tidx == 0u) next = true;
                if (single && batch == 1 && sm.st->next_u * rel + Emax < sm.st->T) next = true;
            }
            if (!next) continue;
            // the next stage that applies
            const int bz = sm.st->bz;
            if (stage == 2) {
                for (int q = a.nbr_ptr[bz] + threadIdx.x; q < a.nbr_ptr[bz + 1]; q += kSelThreads)
                    sm.ev[a.nbr_idx[q]] &= 3;
                if (threadIdx.x == 0) sm.ev[bz] &= 3;
                __syncthreads();
                stage = 3;
                continue;
            }
            if (stage == 0 && want_ref && a.refine && sm.st->T > 0.f) {
                __syncthreads();                 // every thread has read nc
                if (threadIdx.x == 0) sm.st->q = a.nbr_ptr[bz];
                stage = 1;
                continue;
            }
            if (want_ru) {
                for (int q = a.nbr_ptr[bz] + threadIdx.x; q < a.nbr_ptr[bz + 1]; q += kSelThreads)
                    sm.ev[a.nbr_idx[q]] |= 4;
                if (threadIdx.x == 0) sm.ev[bz] |= 4;
                __syncthreads();
                stage = 2;
                continue;
            }
            stage = 3;
        }
        if (a.out.za_scores)
            for (int z = threadIdx.x; z < Z; z += kSelThreads)
                a.out.za_scores[(a.off + b) * Z + z] = sm.ev[z] ? sm.U[z] : sm.U[z] * rel + Emax;
        if (warp == 0) {
            if (lane == 0 && a.n_eval) atomicAdd(a.n_eval, evals);
            write_outputs(a, b, sm, want_ref, lane);
        }
        __syncthreads();
    }
}

// Exhaustive mode: each phase's best score, the maximum of the exact per-axis
// scores over its axes, and the phase of the winning axis.  One warp per
// pattern.
__global__ void k_phase_outputs(const float* __restrict__ za_scores, int Z, int nb,
                                const int* __restrict__ poff, int nph, acom_result out,
                                int64_t off) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= nb) return;
    const int64_t o = off + b;
    if (out.phase && lane == 0) out.phase[o] = phase_of(poff, nph, out.za_idx[o]);
    if (!out.phase_score) return;
    for (int p = 0; p < nph; ++p) {
        float m = -CUDART_INF_F;
        for (int z = poff[p] + lane; z < poff[p + 1]; z += 32) m = fmaxf(m, za_scores[b * Z + z]);
        for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
        if (lane == 0) out.phase_score[o * nph + p] = m;
    }
}

void launch_phase_outputs(const acom_plan_s* p, const float* za_scores, int nb, acom_result out,
                          int64_t off, cudaStream_t st) {
    if (nb <= 0) return;
    prof_begin(kKMisc, st);
    k_phase_outputs<<<(nb + 3) / 4, 128, 0, st>>>(za_scores, p->Z, nb, p->phase_off, p->n_phases,
                                                   out, off);
    prof_end(kKMisc, st);
}

size_t select_smem_bytes(int Z, int N, int F, int Spad) {
    auto r16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t pb = sizeof(float4) * 4 * sel_items(F), yb = sizeof(float2) * kBatch * (size_t)N;
    return r16(sizeof(float2) * N) + r16(sizeof(float2) * kBatch * (size_t)N) + r16(pb > yb ? pb : yb) +
           r16(sizeof(float) * Z) + 2 * r16(sizeof(float) * kSelWarps * kBatch) +
           r16(sizeof(int) * kBatch) + r16(sizeof(float) * 5 * kBatch) +
           r16(sizeof(float) * 2 * kSelWarps) + r16(sizeof(int) * (kMaxPhases + 1)) +
           r16(sizeof(uint32_t) * (Spad >> 5)) + r16(sizeof(uint16_t) * kBatch * Spad) +
           r16(sizeof(int) * kBatch) +
           (N == 360 ? 2 * r16(sizeof(uint16_t) * 360) : 0) +
           r16(sizeof(SelState)) + r16(Z) + r16(sizeof(uint16_t) * Z);
}

void launch_select_exact(const acom_plan_s* p, const float* Xsr, const float* Xsi, const float* U,
                         const float* xfn, const int2* srange, const uint32_t* rmask,
                         const float* pfmax, const float* xnorm2, int nb,
                         float kappa, int refine, acom_result out, int64_t off, int* n_eval,
                         cudaStream_t st, const float* xscale, int rescore_top, OrientIn* oin) {
    SelectArgs a{p->Psr, p->Psi, Xsr, Xsi, U, xfn, srange, rmask, pfmax, xnorm2, p->za, p->frames,
                 p->nbr_ptr,
                 p->nbr_idx, p->phase_off, p->n_phases, p->Z, p->F, p->N, p->S, p->Spad, nb, refine, kappa,
                 fft_radices(p->N), out, off, n_eval, xscale, 1.0f / p->pscale,
                 p->precision == ACOM_PREC_FP8 ? kFp8Shift : 1.0f,
                 (float)(p->precision == ACOM_PREC_FP8 ? kFp8Eta : kFp16Eta), rescore_top,
                 p->smask, oin};
    a.eta_rs = (float)((double)a.eta * std::sqrt((double)p->Spad));
    const size_t smem = select_smem_bytes(p->Z, p->N, p->F, p->Spad);
    const bool pfa = p->N == 360;
    const bool full = (out.phase_score != nullptr && p->n_phases > 1) || rescore_top > 0 ||
                      out.runner_za || out.runner_score || out.runner_orient;
    const void* kern = pfa ? (full ? (const void*)k_select_exact<true, true>
                                   : (const void*)k_select_exact<true, false>)
                           : (full ? (const void*)k_select_exact<false, true>
                                   : (const void*)k_select_exact<false, false>);
    set_max_dynamic_smem(kern, smem);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSelThreads, smem);
    int64_t grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (grid > nb) grid = nb;
    if (grid <= 0) return;
    prof_begin(kKSelect, st);
    void* args[] = {(void*)&a};
    cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kSelThreads), args, smem, st);
    prof_end(kKSelect, st);
}

}  // namespace acom
