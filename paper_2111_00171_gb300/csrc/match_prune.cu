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
// max over zone axes of ||P^_zf||_2 (over shells), per frequency
// ---------------------------------------------------------------------------
__global__ void k_plan_fnorm_max(const float* __restrict__ Pr, const float* __restrict__ Pi,
                                 int Z, int F, int Spad, float* __restrict__ out) {
    const int f = blockIdx.x;
    __shared__ float red[256];
    float mx = 0.f;
    for (int z = threadIdx.x; z < Z; z += blockDim.x) {
        const int64_t o = ((int64_t)z * F + f) * Spad;
        float a = 0.f;
        for (int s = 0; s < Spad; ++s) a = fmaf(Pr[o + s], Pr[o + s], fmaf(Pi[o + s], Pi[o + s], a));
        mx = fmaxf(mx, sqrtf(a));
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0] * 1.0001f;   // rounding of the norm itself
}

void launch_plan_fnorm_max(const acom_plan_s* p, float* out, cudaStream_t st) {
    prof_begin(kKMisc, st);
    k_plan_fnorm_max<<<p->F, 256, 0, st>>>(p->Pr, p->Pi, p->Z, p->F, p->Spad, out);
    prof_end(kKMisc, st);
}

// ---------------------------------------------------------------------------
// Selection and exact evaluation, one CTA per pattern.  Candidate axes are
// evaluated in batches of up to kBatch per pass over the pattern's spectrum:
// one thread per frequency runs down the shells (spectra stored shell-major,
// so the loads of a warp are contiguous) and accumulates the four real
// products for every candidate of the batch.
// ---------------------------------------------------------------------------
constexpr int kSelThreads = 192;
constexpr int kBatch = 8;

struct SelSmem {
    float* U;        // [Z] bound, replaced by the exact score once evaluated
    uint8_t* ev;     // [Z] 0 pending, 1 evaluated, 2 in the current batch
    float2* tw;      // [N] (cos, sin) of 2 pi i / N
    float2* y;       // [kBatch][N] spectra c_dir + i c_mir of the batch
    float2* tmp;     // [N] transform ping-pong
    float* red_v;    // [32]
    int* red_i;      // [32]
    int* cand;       // [kBatch]
};

constexpr int kMaxRadix = 12;
struct Radix {
    int n;                 // number of stages (0: no factorisation, direct transform)
    int r[kMaxRadix];      // radices 4, 2, 3, 5
};

__device__ inline bool better(float v, unsigned i, float bv, unsigned bi) {
    return v > bv || (v == bv && i < bi);
}

// block-wide argmax of (value, index) with the lowest index on ties
__device__ void block_argmax(float& v, unsigned& i, float* red_v, int* red_i) {
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, v, o);
        unsigned oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red_v[warp] = v;
        red_i[warp] = (int)i;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? red_v[lane] : -CUDART_INF_F;
        i = lane < nw ? (unsigned)red_i[lane] : 0xffffffffu;
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, v, o);
            unsigned oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (better(ov, oi, v, i)) {
                v = ov;
                i = oi;
            }
        }
        if (lane == 0) {
            red_v[0] = v;
            red_i[0] = (int)i;
        }
    }
    __syncthreads();
    v = red_v[0];
    i = (unsigned)red_i[0];
    __syncthreads();
}

// Spectra c_dir + i c_mir (both correlations are real, so one complex
// transform carries both) of the nc candidate axes of the batch, scaled by 1/N.
template <int KB>
__device__ void batch_spectra(const float* __restrict__ Psr, const float* __restrict__ Psi,
                              const float* __restrict__ Xsr, const float* __restrict__ Xsi,
                              int64_t b, int nc, int F, int N, int s_lo, int s_hi, int Spad,
                              SelSmem& sm) {
    const float invN = 1.0f / (float)N;
    const int pstride = Spad * F;
    const float* xr = Xsr + b * (int64_t)pstride;
    const float* xi = Xsi + b * (int64_t)pstride;
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
        float A[KB], B[KB], C[KB], D[KB];
        int off[KB];
#pragma unroll
        for (int c = 0; c < KB; ++c) {
            A[c] = B[c] = C[c] = D[c] = 0.f;
            off[c] = (c < nc ? sm.cand[c] : sm.cand[0]) * pstride + f;
        }
        // rows of shells outside [s_lo, s_hi) are zero in the pattern spectrum
        int s = s_lo;
        for (; s + 1 < s_hi; s += 2) {
            const int o0 = s * F, o1 = o0 + F;
            const float x1a = xr[o0 + f], x2a = xi[o0 + f], x1b = xr[o1 + f], x2b = xi[o1 + f];
#pragma unroll
            for (int c = 0; c < KB; ++c) {
                if (c < nc) {
                    const float p1a = Psr[off[c] + o0], p2a = Psi[off[c] + o0];
                    const float p1b = Psr[off[c] + o1], p2b = Psi[off[c] + o1];
                    A[c] = fmaf(p1a, x1a, fmaf(p1b, x1b, A[c]));
                    B[c] = fmaf(p2a, x2a, fmaf(p2b, x2b, B[c]));
                    C[c] = fmaf(p1a, x2a, fmaf(p1b, x2b, C[c]));
                    D[c] = fmaf(p2a, x1a, fmaf(p2b, x1b, D[c]));
                }
            }
        }
        if (s < s_hi) {
            const int o0 = s * F;
            const float x1 = xr[o0 + f], x2 = xi[o0 + f];
#pragma unroll
            for (int c = 0; c < KB; ++c) {
                if (c < nc) {
                    const float p1 = Psr[off[c] + o0], p2 = Psi[off[c] + o0];
                    A[c] = fmaf(p1, x1, A[c]);
                    B[c] = fmaf(p2, x2, B[c]);
                    C[c] = fmaf(p1, x2, C[c]);
                    D[c] = fmaf(p2, x1, D[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < KB; ++c) {
            if (c < nc) {
                const float dre = (A[c] + B[c]) * invN, dim = (C[c] - D[c]) * invN;
                const float mre = (A[c] - B[c]) * invN, mim = -(C[c] + D[c]) * invN;
                float2* y = sm.y + c * N;
                y[f] = make_float2(dre - mim, dim + mre);
                if (f > 0 && 2 * f < N) y[N - f] = make_float2(dre + mim, mre - dim);
            }
        }
    }
    __syncthreads();
}

// In-place (through sm.tmp) inverse transform of y: returns the buffer that
// holds C_dir[k] + i C_mir[k].  Stockham mixed radix when N factors into
// 4, 2, 3, 5, otherwise direct.
__device__ float2* inverse_transform(float2* y, int N, const Radix& rad, SelSmem& sm) {
    float2* src = y;
    float2* dst = sm.tmp;
    if (rad.n > 0) {
        int Ns = 1;
        for (int stg = 0; stg < rad.n; ++stg) {
            const int R = rad.r[stg];
            const int NR = N / R;
            const int tstep = N / (Ns * R);
            for (int j = threadIdx.x; j < NR; j += blockDim.x) {
                const int jm = j % Ns;
                float2 v[5];
#pragma unroll
                for (int r = 0; r < 5; ++r) {
                    if (r < R) {
                        const float2 x = src[j + r * NR];
                        const float2 t = sm.tw[r * jm * tstep];
                        v[r] = make_float2(x.x * t.x - x.y * t.y, x.x * t.y + x.y * t.x);
                    }
                }
                const int idxD = (j / Ns) * Ns * R + jm;
#pragma unroll
                for (int mo = 0; mo < 5; ++mo) {
                    if (mo < R) {
                        float2 o = v[0];
#pragma unroll
                        for (int r = 1; r < 5; ++r) {
                            if (r < R) {
                                const float2 t = sm.tw[((r * mo) % R) * NR];
                                o.x = fmaf(v[r].x, t.x, fmaf(-v[r].y, t.y, o.x));
                                o.y = fmaf(v[r].x, t.y, fmaf(v[r].y, t.x, o.y));
                            }
                        }
                        dst[idxD + mo * Ns] = o;
                    }
                }
            }
            __syncthreads();
            float2* t2 = src;
            src = dst;
            dst = t2;
            Ns *= R;
        }
        return src;
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        int idx = 0;
        for (int f = 0; f < N; ++f) {
            const float2 x = src[f], t = sm.tw[idx];
            acc.x = fmaf(x.x, t.x, fmaf(-x.y, t.y, acc.x));
            acc.y = fmaf(x.x, t.y, fmaf(x.y, t.x, acc.y));
            idx += k;
            if (idx >= N) idx -= N;
        }
        dst[k] = acc;
    }
    __syncthreads();
    return dst;
}

__device__ inline void matmul3d(const double* a, const double* b, double* c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

struct SelectArgs {
    const float *Psr, *Psi, *Xsr, *Xsi;   // FP32 spectra, shell-major [.][Spad][F]
    const float* U;                   // [nb][Z] bounds
    const float* xfn;                 // [nb][F] ||X^_bf||
    const int2* srange;               // [nb] non-zero shell range
    const float* pfmax;               // [F] max_z ||P^_zf||
    const float* xnorm2;              // [nb] ||X||^2
    const double* za;                 // [Z][3]
    const double* frames;             // [Z][9]
    const int* nbr_ptr;
    const int* nbr_idx;
    int Z, F, N, S, Spad, nb, refine;
    float kappa;                      // contraction rounding constant
    Radix rad;                        // inverse-transform factorisation
    acom_result out;
    int64_t off;
    int* n_eval;                      // optional: total axes evaluated
};

// Evaluate the axes listed in sm.cand[0..nc) in full; record each exact score
// in sm.U and fold the best into (T, Tidx, bz, bk, bm, best3).
__device__ void evaluate_batch(const SelectArgs& a, int64_t b, int nc, SelSmem& sm, float& T,
                               unsigned& Tidx, int& bz, int& bk, int& bm, float* best3) {
    const int N = a.N;
    const int2 sr = a.srange[b];
    if (nc <= 4)
        batch_spectra<4>(a.Psr, a.Psi, a.Xsr, a.Xsi, b, nc, a.F, N, sr.x, sr.y, a.Spad, sm);
    else
        batch_spectra<kBatch>(a.Psr, a.Psi, a.Xsr, a.Xsi, b, nc, a.F, N, sr.x, sr.y, a.Spad, sm);
    for (int c = 0; c < nc; ++c) {
        const int z = sm.cand[c];
        const float2* y = inverse_transform(sm.y + c * N, N, a.rad, sm);
        float bv = -CUDART_INF_F;
        unsigned bi = 0xffffffffu;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const float2 v = y[k];
            if (better(v.x, (unsigned)k, bv, bi)) { bv = v.x; bi = (unsigned)k; }
            if (better(v.y, (unsigned)(N + k), bv, bi)) { bv = v.y; bi = (unsigned)(N + k); }
        }
        block_argmax(bv, bi, sm.red_v, sm.red_i);
        const unsigned gidx = (unsigned)z * 2u * (unsigned)N + bi;
        if (better(bv, gidx, T, Tidx)) {
            T = bv;
            Tidx = gidx;
            bz = z;
            bm = (int)(bi / (unsigned)N);
            bk = (int)(bi - (unsigned)bm * N);
            if (threadIdx.x == 0) {
                const float2 ym = y[(bk + N - 1) % N], y0 = y[bk], yp = y[(bk + 1) % N];
                best3[0] = bm ? ym.y : ym.x;
                best3[1] = bm ? y0.y : y0.x;
                best3[2] = bm ? yp.y : yp.x;
            }
        }
        if (threadIdx.x == 0) {
            sm.U[z] = bv;
            sm.ev[z] = 1;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSelThreads, 3) k_select_exact(SelectArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Z = a.Z, F = a.F, N = a.N;
    SelSmem sm;
    sm.tw = reinterpret_cast<float2*>(smem_raw);
    sm.y = sm.tw + N;
    sm.tmp = sm.y + kBatch * N;
    sm.U = reinterpret_cast<float*>(sm.tmp + N);
    sm.red_v = sm.U + Z;
    sm.red_i = reinterpret_cast<int*>(sm.red_v + 32);
    sm.cand = sm.red_i + 32;
    sm.ev = reinterpret_cast<uint8_t*>(sm.cand + kBatch);
    __shared__ float s_best3[3];
    __shared__ double s_w[3];

    const int64_t b = blockIdx.x;
    if (b >= a.nb) return;
    for (int z = threadIdx.x; z < Z; z += blockDim.x) {
        sm.U[z] = a.U[b * Z + z];
        sm.ev[z] = 0;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)i / (double)N, &s, &c);
        sm.tw[i] = make_float2((float)c, (float)s);
    }
    // E_b: rounding margin valid for every axis
    float e = 0.f;
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
        const float w = (f == 0 || 2 * f == N) ? 1.f : 2.f;
        e = fmaf(w * a.pfmax[f], a.xfn[b * F + f], e);
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) sm.red_v[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm.red_v[w];
        sm.red_v[0] = t;
    }
    __syncthreads();
    const float Emax = a.kappa * sm.red_v[0] / (float)N * 1.01f;
    const float rel = 1.0f + 1e-5f;     // FP32 accumulation of U and of the scores
    __syncthreads();

    float T = -CUDART_INF_F;            // best exact score so far
    unsigned Tidx = 0xffffffffu;        // (z * 2 + mir) * N + k of the best
    int bz = 0, bk = 0, bm = 0;
    int evals = 0;
    // batches in decreasing bound: the first takes the 4 largest bounds, later
    // ones every axis whose bound can still reach the best exact score
    for (int batch = 0;; ++batch) {
        const int cap = batch == 0 ? 4 : kBatch;
        int nc = 0;
        while (nc < cap) {
            float v = -CUDART_INF_F;
            unsigned zi = 0xffffffffu;
            for (int z = threadIdx.x; z < Z; z += blockDim.x)
                if (sm.ev[z] == 0 && better(sm.U[z], (unsigned)z, v, zi)) {
                    v = sm.U[z];
                    zi = (unsigned)z;
                }
            block_argmax(v, zi, sm.red_v, sm.red_i);
            if (zi == 0xffffffffu) break;
            if (T != -CUDART_INF_F && v * rel + Emax < T) break;     // nothing left can win
            if (threadIdx.x == 0) {
                sm.cand[nc] = (int)zi;
                sm.ev[zi] = 2;
            }
            __syncthreads();
            ++nc;
        }
        if (nc == 0) break;
        evaluate_batch(a, b, nc, sm, T, Tidx, bz, bk, bm, s_best3);
        evals += nc;
        // an all-zero image: every axis ties at 0 and the lowest index has won
        if (T == 0.f && Tidx == 0u) break;
    }
    // zone-axis neighbours that may reach 0.9 of the best need their exact score
    const bool want_ref = (a.out.phi3 != nullptr) || (a.out.orient != nullptr);
    if (want_ref && a.refine && T > 0.f) {
        int q = a.nbr_ptr[bz];
        const int qe = a.nbr_ptr[bz + 1];
        for (;;) {
            int nc = 0;
            for (; q < qe && nc < kBatch; ++q) {
                const int z2 = a.nbr_idx[q];
                if (sm.ev[z2] || sm.U[z2] * rel + Emax < 0.9f * T) continue;
                if (threadIdx.x == 0) {
                    sm.cand[nc] = z2;
                    sm.ev[z2] = 2;
                }
                ++nc;
            }
            __syncthreads();
            if (nc == 0) break;
            float Tn = T;
            unsigned Tin = Tidx;
            int z0 = bz, k0 = bk, m0 = bm;
            float dummy[3];
            evaluate_batch(a, b, nc, sm, Tn, Tin, z0, k0, m0, dummy);
            evals += nc;
        }
    }
    // outputs
    if (a.out.za_scores)
        for (int z = threadIdx.x; z < Z; z += blockDim.x)
            a.out.za_scores[(a.off + b) * Z + z] = sm.ev[z] ? sm.U[z] : sm.U[z] * rel + Emax;
    if (threadIdx.x == 0 && a.n_eval) atomicAdd(a.n_eval, evals);
    double dk = 0.0;
    if (threadIdx.x == 0 && want_ref && a.refine) {
        const double cm = s_best3[0], c0 = s_best3[1], cp = s_best3[2];
        const double den = cm - 2.0 * c0 + cp;
        if (den < 0.0) {
            dk = (cm - cp) / (2.0 * den);
            dk = dk > 0.5 ? 0.5 : (dk < -0.5 ? -0.5 : dk);
        }
        double a0 = 0, a1 = 0, a2 = 0;
        for (int q = a.nbr_ptr[bz]; q < a.nbr_ptr[bz + 1]; ++q) {
            const int z2 = a.nbr_idx[q];
            if (!sm.ev[z2]) continue;             // its true score is below 0.9 of the best
            const float sc = sm.U[z2];
            if (sc >= 0.9f * T) {
                a0 += (double)sc * a.za[3 * z2];
                a1 += (double)sc * a.za[3 * z2 + 1];
                a2 += (double)sc * a.za[3 * z2 + 2];
            }
        }
        const double nrm = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        s_w[0] = nrm > 0 ? a0 / nrm : a.za[3 * bz];
        s_w[1] = nrm > 0 ? a1 / nrm : a.za[3 * bz + 1];
        s_w[2] = nrm > 0 ? a2 / nrm : a.za[3 * bz + 2];
    }
    if (threadIdx.x != 0) return;
    const int64_t o = a.off + b;
    const float score = T == -CUDART_INF_F ? 0.f : T;
    a.out.za_idx[o] = bz;
    a.out.phi3_bin[o] = bk;
    a.out.mirror[o] = (uint8_t)bm;
    a.out.score[o] = score;
    if (a.out.score_cos) {
        const float xn = sqrtf(a.xnorm2[b]);
        a.out.score_cos[o] = xn > 0.f ? score / xn : 0.f;
    }
    if (!want_ref) return;
    double wref[3];
    if (a.refine) {
        wref[0] = s_w[0]; wref[1] = s_w[1]; wref[2] = s_w[2];
    } else {
        wref[0] = a.za[3 * bz]; wref[1] = a.za[3 * bz + 1]; wref[2] = a.za[3 * bz + 2];
    }
    const double phi3 = -2.0 * CUDART_PI * ((double)bk + dk) / (double)N;
    if (a.out.phi3) a.out.phi3[o] = (float)phi3;
    if (!a.out.orient) return;
    double Rz[9], m1[9], m2[9], Tm[9];
    double c3, s3;
    sincos(phi3, &s3, &c3);
    Rz[0] = c3; Rz[1] = -s3; Rz[2] = 0; Rz[3] = s3; Rz[4] = c3; Rz[5] = 0; Rz[6] = 0; Rz[7] = 0; Rz[8] = 1;
    matmul3d(a.frames + 9 * bz, Rz, m1);
    if (bm) {
        for (int i = 0; i < 3; ++i) {
            m1[3 * i] = -m1[3 * i];
            m1[3 * i + 2] = -m1[3 * i + 2];
        }
    }
    const double u0 = a.za[3 * bz], u1 = a.za[3 * bz + 1], u2 = a.za[3 * bz + 2];
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
    for (int i = 0; i < 9; ++i) a.out.orient[9 * o + i] = (float)m2[i];
}

size_t select_smem_bytes(int Z, int N, int F) {
    return sizeof(float2) * (kBatch + 2) * (size_t)N + sizeof(float) * ((size_t)Z + 32) +
           sizeof(int) * (32 + kBatch) + Z + 16;
}

static Radix factor_radices(int N) {
    Radix r{};
    int n = N;
    const int cand[4] = {4, 2, 3, 5};
    for (int c = 0; c < 4; ++c)
        while (n % cand[c] == 0 && r.n < kMaxRadix) {
            r.r[r.n++] = cand[c];
            n /= cand[c];
        }
    if (n != 1) r.n = 0;
    return r;
}

void launch_select_exact(const acom_plan_s* p, const float* Xsr, const float* Xsi, const float* U,
                         const float* xfn, const int2* srange, const float* pfmax,
                         const float* xnorm2, int nb,
                         float kappa, int refine, acom_result out, int64_t off, int* n_eval,
                         cudaStream_t st) {
    SelectArgs a{p->Psr, p->Psi, Xsr, Xsi, U, xfn, srange, pfmax, xnorm2, p->za, p->frames,
                 p->nbr_ptr,
                 p->nbr_idx, p->Z, p->F, p->N, p->S, p->Spad, nb, refine, kappa,
                 factor_radices(p->N), out, off, n_eval};
    const size_t smem = select_smem_bytes(p->Z, p->N, p->F);
    cudaFuncSetAttribute(k_select_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin(kKSelect, st);
    k_select_exact<<<nb, kSelThreads, smem, st>>>(a);
    prof_end(kKSelect, st);
}

}  // namespace acom
