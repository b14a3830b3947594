// FP32 CUDA-core path of the correlation step (section "Correlation Pattern
// Matching"): the per-frequency contraction over shells, the inverse
// transform along phi3 with the maximum over phi3 and mirror, and the
// sub-grid refinement of the winner.
//
// Contraction.  For every frequency f the plan spectrum P^ (zone axes x
// shells) meets the pattern spectra X^ (patterns x shells):
//   A = Pr Xr, B = Pi Xi, C = Pr Xi, D = Pi Xr   (sums over shells)
//   FFT{P}^* FFT{X}   = (A + B) + i (C - D)          (direct)
//   FFT{P}^* FFT{X}^* = (A - B) - i (C + D)          (mirror)
// The four real products are shared by both correlations.  Results go to a
// scratch array [4][F][chunk][Zp] (re/im of direct, re/im of mirror).
//
// Inverse transform.  For a real correlation of even length N with spectrum
// c_f (f = 0..N/2), C[k] = (1/N) sum_f w_f (Re c_f cos(2 pi f k/N)
// - Im c_f sin(2 pi f k/N)), w_0 = w_{N/2} = 1, else 2.  With
// u_k = sum_f w_f Re c_f cos, v_k = sum_f w_f Im c_f sin (k = 0..N/2):
// C[k] = (u_k - v_k)/N and C[N-k] = (u_k + v_k)/N, so half of the bins give
// all of them.
#include <math_constants.h>

#include <cmath>

#include "acom_internal.cuh"

namespace acom {

constexpr int kCtZ = 64, kCtB = 64, kCtK = 16;

__global__ void __launch_bounds__(256)
k_contract_fp32(const float* __restrict__ Pr, const float* __restrict__ Pi,
                const float* __restrict__ Xr, const float* __restrict__ Xi, int F, int Spad,
                int Zp, int nb, int chunk, float* __restrict__ Chat) {
    __shared__ __align__(16) float sPr[kCtK][kCtZ + 4];
    __shared__ __align__(16) float sPi[kCtK][kCtZ + 4];
    __shared__ __align__(16) float sXr[kCtK][kCtB + 4];
    __shared__ __align__(16) float sXi[kCtK][kCtB + 4];
    const int z0 = blockIdx.x * kCtZ, b0 = blockIdx.y * kCtB, f = blockIdx.z;
    const int t = threadIdx.x, tz = t & 15, tb = t >> 4;
    float A[4][4], B[4][4], C[4][4], D[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) A[i][j] = B[i][j] = C[i][j] = D[i][j] = 0.f;

    const int lr = t >> 2, lc = (t & 3) * 4;
    const int64_t prow = ((int64_t)(z0 + lr) * F + f) * Spad;
    const bool bvalid = (b0 + lr) < nb;
    const int64_t xrow = ((int64_t)(b0 + lr) * F + f) * Spad;
    for (int s0 = 0; s0 < Spad; s0 += kCtK) {
        float4 pr = *reinterpret_cast<const float4*>(Pr + prow + s0 + lc);
        float4 pi = *reinterpret_cast<const float4*>(Pi + prow + s0 + lc);
        float4 xr = make_float4(0.f, 0.f, 0.f, 0.f), xi = xr;
        if (bvalid) {
            xr = *reinterpret_cast<const float4*>(Xr + xrow + s0 + lc);
            xi = *reinterpret_cast<const float4*>(Xi + xrow + s0 + lc);
        }
        sPr[lc + 0][lr] = pr.x; sPr[lc + 1][lr] = pr.y; sPr[lc + 2][lr] = pr.z; sPr[lc + 3][lr] = pr.w;
        sPi[lc + 0][lr] = pi.x; sPi[lc + 1][lr] = pi.y; sPi[lc + 2][lr] = pi.z; sPi[lc + 3][lr] = pi.w;
        sXr[lc + 0][lr] = xr.x; sXr[lc + 1][lr] = xr.y; sXr[lc + 2][lr] = xr.z; sXr[lc + 3][lr] = xr.w;
        sXi[lc + 0][lr] = xi.x; sXi[lc + 1][lr] = xi.y; sXi[lc + 2][lr] = xi.z; sXi[lc + 3][lr] = xi.w;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kCtK; ++kk) {
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
        __syncthreads();
    }
    const int64_t plane = (int64_t)chunk * Zp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = b0 + tb * 4 + j;
        if (b >= nb) continue;
        const int64_t base = ((int64_t)f * chunk + b) * Zp + z0 + tz * 4;
        float4 dre, dim, mre, mim;
        dre.x = A[0][j] + B[0][j]; dre.y = A[1][j] + B[1][j]; dre.z = A[2][j] + B[2][j]; dre.w = A[3][j] + B[3][j];
        dim.x = C[0][j] - D[0][j]; dim.y = C[1][j] - D[1][j]; dim.z = C[2][j] - D[2][j]; dim.w = C[3][j] - D[3][j];
        mre.x = A[0][j] - B[0][j]; mre.y = A[1][j] - B[1][j]; mre.z = A[2][j] - B[2][j]; mre.w = A[3][j] - B[3][j];
        mim.x = -(C[0][j] + D[0][j]); mim.y = -(C[1][j] + D[1][j]); mim.z = -(C[2][j] + D[2][j]); mim.w = -(C[3][j] + D[3][j]);
        *reinterpret_cast<float4*>(Chat + base) = dre;
        *reinterpret_cast<float4*>(Chat + base + (int64_t)F * plane) = dim;
        *reinterpret_cast<float4*>(Chat + base + 2 * (int64_t)F * plane) = mre;
        *reinterpret_cast<float4*>(Chat + base + 3 * (int64_t)F * plane) = mim;
    }
}

void launch_contract_fp32(const acom_plan_s* p, const float* Xr, const float* Xi, int nb,
                          float* Chat, int chunk, cudaStream_t st) {
    dim3 grid(p->Zp / kCtZ, (nb + kCtB - 1) / kCtB, p->F);
    prof_begin(kKContract, st);
    k_contract_fp32<<<grid, 256, 0, st>>>(p->Pr, p->Pi, Xr, Xi, p->F, p->Spad, p->Zp, nb, chunk,
                                          Chat);
    prof_end(kKContract, st);
}

// ---------------------------------------------------------------------------
// Inverse transform + maximum over phi3 and mirror for 32 zone axes of one
// pattern per CTA; per-pair maxima go to za_scores and the best key of the
// pattern is merged with a 64-bit atomicMax (order independent).
// ---------------------------------------------------------------------------

constexpr int kIdPairs = 32;

__device__ inline void consider(float v, unsigned idx, float& bv, unsigned& bi) {
    if (v > bv || (v == bv && idx < bi)) {
        bv = v;
        bi = idx;
    }
}

__global__ void __launch_bounds__(256)
k_idft_argmax_fp32(const float* __restrict__ Chat, int F, int N, int Z, int Zp, int chunk,
                   float* __restrict__ za_scores, unsigned long long* __restrict__ best) {
    extern __shared__ __align__(16) float smem_f[];
    float* sC = smem_f;                          // [4][F][32], weights and 1/N folded in
    float* twc = sC + 4 * F * kIdPairs;          // [N]
    float* tws = twc + N;
    __shared__ unsigned long long s_key[8];
    const int z0 = blockIdx.x * kIdPairs, b = blockIdx.y;
    const int64_t plane = (int64_t)chunk * Zp;
    const float invN = 1.0f / (float)N;
    for (int e = threadIdx.x; e < 4 * F * kIdPairs; e += blockDim.x) {
        const int c = e / (F * kIdPairs);
        const int rem = e - c * F * kIdPairs;
        const int f = rem / kIdPairs, pr = rem - f * kIdPairs;
        const float w = (f == 0 || 2 * f == N) ? invN : 2.0f * invN;
        sC[e] = w * Chat[(int64_t)c * F * plane + ((int64_t)f * chunk + b) * Zp + z0 + pr];
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)i / (double)N, &s, &c);
        twc[i] = (float)c;
        tws[i] = (float)s;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, pg = threadIdx.x >> 5;   // 4 pairs per warp
    const int K2 = N / 2 + 1;
    float bv[4];
    unsigned bi[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        bv[i] = -CUDART_INF_F;
        bi[i] = 0xffffffffu;
    }
    for (int kbase = 0; kbase < K2; kbase += 128) {
        int kk[4], idx[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            kk[j] = kbase + lane * 4 + j;
            idx[j] = 0;
        }
        float ud[4][4], vd[4][4], um[4][4], vm[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) ud[i][j] = vd[i][j] = um[i][j] = vm[i][j] = 0.f;
        int kstep[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) kstep[j] = kk[j] < K2 ? kk[j] % N : 0;
        for (int f = 0; f < F; ++f) {
            const float4 dre = *reinterpret_cast<const float4*>(sC + (0 * F + f) * kIdPairs + pg * 4);
            const float4 dim = *reinterpret_cast<const float4*>(sC + (1 * F + f) * kIdPairs + pg * 4);
            const float4 mre = *reinterpret_cast<const float4*>(sC + (2 * F + f) * kIdPairs + pg * 4);
            const float4 mim = *reinterpret_cast<const float4*>(sC + (3 * F + f) * kIdPairs + pg * 4);
            const float r_d[4] = {dre.x, dre.y, dre.z, dre.w};
            const float i_d[4] = {dim.x, dim.y, dim.z, dim.w};
            const float r_m[4] = {mre.x, mre.y, mre.z, mre.w};
            const float i_m[4] = {mim.x, mim.y, mim.z, mim.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float cs = twc[idx[j]], sn = tws[idx[j]];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ud[i][j] = fmaf(r_d[i], cs, ud[i][j]);
                    vd[i][j] = fmaf(i_d[i], sn, vd[i][j]);
                    um[i][j] = fmaf(r_m[i], cs, um[i][j]);
                    vm[i][j] = fmaf(i_m[i], sn, vm[i][j]);
                }
                idx[j] += kstep[j];
                if (idx[j] >= N) idx[j] -= N;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = kk[j];
            if (k >= K2) continue;
            const bool has_pair = (k > 0) && (2 * k < N);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                consider(ud[i][j] - vd[i][j], (unsigned)k, bv[i], bi[i]);
                consider(um[i][j] - vm[i][j], (unsigned)(N + k), bv[i], bi[i]);
                if (has_pair) {
                    consider(ud[i][j] + vd[i][j], (unsigned)(N - k), bv[i], bi[i]);
                    consider(um[i][j] + vm[i][j], (unsigned)(2 * N - k), bv[i], bi[i]);
                }
            }
        }
    }
    // reduce the 32 lanes of the warp (same pairs, different phi3 bins)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, bv[i], o);
            unsigned oi = __shfl_xor_sync(0xffffffffu, bi[i], o);
            consider(ov, oi, bv[i], bi[i]);
        }
    }
    if (lane == 0) {
        unsigned long long kmax = 0ull;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int z = z0 + pg * 4 + i;
            if (z < Z) {
                za_scores[(int64_t)b * Z + z] = bv[i];
                unsigned long long key = pack_best(bv[i], (unsigned)z * 2u * (unsigned)N + bi[i]);
                kmax = key > kmax ? key : kmax;
            }
        }
        s_key[pg] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long kmax = 0ull;
        for (int w = 0; w < 8; ++w) kmax = s_key[w] > kmax ? s_key[w] : kmax;
        if (kmax) atomicMax(best + b, kmax);
    }
}

void launch_idft_argmax_fp32(const acom_plan_s* p, const float* Chat, int nb, int chunk,
                             float* za_scores, unsigned long long* best, cudaStream_t st) {
    size_t smem = sizeof(float) * (4 * p->F * kIdPairs + 2 * p->N);
    set_max_dynamic_smem((const void*)k_idft_argmax_fp32, smem);
    dim3 grid(p->Zp / kIdPairs, nb);
    prof_begin(kKIdft, st);
    k_idft_argmax_fp32<<<grid, 256, smem, st>>>(Chat, p->F, p->N, p->Z, p->Zp, chunk, za_scores,
                                                 best);
    prof_end(kKIdft, st);
}

// ---------------------------------------------------------------------------
// Refinement (the paper reports grid results; this is the library's reading):
// phi3 from the parabola through the best bin and its two neighbours of the
// winning correlation, the zone axis as the score-weighted mean of the best
// axis and its grid neighbours scoring >= 0.9 of the best, and the
// orientation m = T(w_best -> w_ref) Rz(phi1) Rx(theta2) Rz(phi3) [Ry(pi)],
// composed in FP64.  One warp per pattern.
// ---------------------------------------------------------------------------

__device__ inline void matmul3(const double* a, const double* b, double* c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

__global__ void k_refine(const float* __restrict__ Chat, int F, int N, int Z, int Zp, int chunk,
                         int nb, const float* __restrict__ za_scores,
                         const unsigned long long* __restrict__ best,
                         const float* __restrict__ xnorm2, const double* __restrict__ za,
                         const double* __restrict__ frames, const int* __restrict__ nbr_ptr,
                         const int* __restrict__ nbr_idx, int refine, acom_result out,
                         int64_t off) {
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= nb) return;
    const int b = wid;
    const unsigned long long key = best[b];
    const unsigned idx = 0xffffffffu - (unsigned)(key & 0xffffffffull);
    const float score = float_from_order_key((unsigned)(key >> 32));
    const int z = (int)(idx / (2u * N));
    const int rem = (int)(idx - (unsigned)z * 2u * N);
    const int mir = rem / N, k = rem - mir * N;
    const bool want_ref = (out.phi3 != nullptr) || (out.orient != nullptr);
    double dk = 0.0;
    double wref[3] = {0, 0, 0};
    if (want_ref && refine) {
        // C at k-1, k, k+1 of the winning correlation
        const int64_t plane = (int64_t)chunk * Zp;
        const float* cre = Chat + (int64_t)(2 * mir) * F * plane;
        const float* cim = cre + (int64_t)F * plane;
        float acc[3] = {0.f, 0.f, 0.f};
        for (int f = lane; f < F; f += 32) {
            const int64_t o = ((int64_t)f * chunk + b) * Zp + z;
            const float re = cre[o], im = cim[o];
            const float w = (f == 0 || 2 * f == N) ? 1.f : 2.f;
            for (int d = -1; d <= 1; ++d) {
                const int kk = ((k + d) % N + N) % N;
                const int ph = (int)(((int64_t)f * kk) % N);
                double s, c;
                sincospi(2.0 * (double)ph / (double)N, &s, &c);
                acc[d + 1] += w * (re * (float)c - im * (float)s);
            }
        }
        for (int d = 0; d < 3; ++d)
            for (int o = 16; o > 0; o >>= 1) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], o);
        const double cm = acc[0], c0 = acc[1], cp = acc[2];
        const double den = cm - 2.0 * c0 + cp;
        if (den < 0.0) {
            dk = (cm - cp) / (2.0 * den);
            dk = dk > 0.5 ? 0.5 : (dk < -0.5 ? -0.5 : dk);
        }
        // score-weighted neighbour mean of the zone axis
        const float zbest = za_scores[(int64_t)b * Z + z];
        double a0 = 0, a1 = 0, a2 = 0;
        for (int q = nbr_ptr[z] + lane; q < nbr_ptr[z + 1]; q += 32) {
            const int z2 = nbr_idx[q];
            const float sc = za_scores[(int64_t)b * Z + z2];
            if (sc >= 0.9f * zbest) {
                a0 += (double)sc * za[3 * z2];
                a1 += (double)sc * za[3 * z2 + 1];
                a2 += (double)sc * za[3 * z2 + 2];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        const double nrm = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        if (nrm > 0) {
            wref[0] = a0 / nrm; wref[1] = a1 / nrm; wref[2] = a2 / nrm;
        } else {
            wref[0] = za[3 * z]; wref[1] = za[3 * z + 1]; wref[2] = za[3 * z + 2];
        }
    } else {
        wref[0] = za[3 * z]; wref[1] = za[3 * z + 1]; wref[2] = za[3 * z + 2];
    }
    if (lane != 0) return;
    const int64_t o = off + b;
    out.za_idx[o] = z;
    out.phi3_bin[o] = k;
    out.mirror[o] = (uint8_t)mir;
    out.score[o] = score;
    if (out.score_cos) {
        const float xn = sqrtf(xnorm2[b]);
        out.score_cos[o] = xn > 0.f ? score / xn : 0.f;
    }
    if (!want_ref) return;
    const double phi3 = -2.0 * CUDART_PI * ((double)k + dk) / (double)N;
    if (out.phi3) out.phi3[o] = (float)phi3;
    if (!out.orient) return;
    double Rz[9], m1[9], m2[9], T[9];
    double c3, s3;
    sincos(phi3, &s3, &c3);
    Rz[0] = c3; Rz[1] = -s3; Rz[2] = 0; Rz[3] = s3; Rz[4] = c3; Rz[5] = 0; Rz[6] = 0; Rz[7] = 0; Rz[8] = 1;
    matmul3(frames + 9 * z, Rz, m1);
    if (mir) {   // right-multiply by Ry(pi) = diag(-1, 1, -1)
        for (int i = 0; i < 3; ++i) {
            m1[3 * i] = -m1[3 * i];
            m1[3 * i + 2] = -m1[3 * i + 2];
        }
    }
    // smallest rotation taking w_best to w_ref (Rodrigues)
    const double u0 = za[3 * z], u1 = za[3 * z + 1], u2 = za[3 * z + 2];
    double ax0 = u1 * wref[2] - u2 * wref[1];
    double ax1 = u2 * wref[0] - u0 * wref[2];
    double ax2 = u0 * wref[1] - u1 * wref[0];
    const double sn = sqrt(ax0 * ax0 + ax1 * ax1 + ax2 * ax2);
    const double cs = u0 * wref[0] + u1 * wref[1] + u2 * wref[2];
    for (int i = 0; i < 9; ++i) T[i] = (i % 4 == 0) ? 1.0 : 0.0;
    if (sn > 1e-15) {
        ax0 /= sn; ax1 /= sn; ax2 /= sn;
        const double K[9] = {0, -ax2, ax1, ax2, 0, -ax0, -ax1, ax0, 0};
        double K2[9];
        matmul3(K, K, K2);
        for (int i = 0; i < 9; ++i) T[i] += sn * K[i] + (1.0 - cs) * K2[i];
    }
    matmul3(T, m1, m2);
    for (int i = 0; i < 9; ++i) out.orient[9 * o + i] = (float)m2[i];
}

void launch_refine(const acom_plan_s* p, const float* Chat, int nb, int chunk,
                   const float* za_scores, const unsigned long long* best, const float* xnorm2,
                   int refine, acom_result out, int64_t off, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (nb * 32 + threads - 1) / threads;
    if (blocks > 0) {
        prof_begin(kKRefine, st);
        k_refine<<<blocks, threads, 0, st>>>(Chat, p->F, p->N, p->Z, p->Zp, chunk, nb, za_scores,
                                             best, xnorm2, p->za, p->frames, p->nbr_ptr,
                                             p->nbr_idx, refine, out, off);
        prof_end(kKRefine, st);
    }
}

}  // namespace acom
