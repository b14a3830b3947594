// Several matches per pattern (section "Matching of Overlapping Diffraction
// Patterns"): after a match, the forward pattern of the matched orientation is
// computed and the peaks it explains are removed or weakened, then the pattern
// is matched again.  Each match is reported with the correlation of the
// original, full pattern at its (zone axis, phi3 bin, mirror).
//
// k_delete_peaks  one warp per pattern: the grid orientation of the match
//                 (frame of the axis, Rz(-2 pi k / N), Ry(pi) for a mirror
//                 match); the reflections whose Gaussian shape factor D(s_g)
//                 (Eq. 8, excitation error by Eq. 6) reaches d_min form the
//                 forward pattern; each peak within r_del of a spot is removed
//                 (moved outside every shell, intensity 0), each one within
//                 the correlation kernel size delta keeps (d - r_del) /
//                 (delta - r_del) of its intensity.  A match whose best
//                 correlation is 0 (nothing left to match) is marked -1.
// k_score_at      one warp per (pattern, match): c_f over the pattern's
//                 non-zero shells from the shell-major spectra, then the
//                 inverse transform at the one bin k: sum_f y_f exp(2 pi i f
//                 k / N) = C_dir[k] + i C_mir[k], y = (c_dir + i c_mir) / N
//                 (the spectrum the select kernel transforms).
#include <math_constants.h>

#include "acom_internal.cuh"

namespace acom {

namespace {

constexpr int kDelWarps = 4;
constexpr int kDelSpotCap = 512;               // forward spots listed at a time
constexpr float kFarAway = 1.0e4f;             // 1/A: outside every shell

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct DelArgs {
    const float4* refl;        // [G] (g, weight); only g is used here
    int G;
    const double* frames;      // [Z][9]
    int N;
    float inv_lam, s2max;      // spot when s^2 <= s2max (D(s) >= d_min)
    float r_del, delta;
    const int64_t* row_ptr;
    float *qx, *qy, *I;        // working peaks, changed in place
    int32_t* za;               // match j: -1 written where nothing was matched
    const int32_t* kbin;
    const uint8_t* mir;
    const float* score;
    int64_t nb;
};

__global__ void __launch_bounds__(kDelWarps * 32) k_delete_peaks(DelArgs a) {
    __shared__ float s_x[kDelWarps][kDelSpotCap], s_y[kDelWarps][kDelSpotCap];
    __shared__ float s_d[kDelWarps][kMaxPeaks];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* sx = s_x[warp];
    float* sy = s_y[warp];
    float* dmin = s_d[warp];
    for (int64_t b = (int64_t)blockIdx.x * kDelWarps + warp; b < a.nb;
         b += (int64_t)gridDim.x * kDelWarps) {
        if (!(a.score[b] > 0.0f)) {                 // no further orientation
            if (lane == 0) a.za[b] = -1;
            continue;
        }
        const int64_t p0 = a.row_ptr[b];
        int64_t n = a.row_ptr[b + 1] - p0;
        if (n < 0) n = 0;
        const int M = (int)(n < kMaxPeaks ? n : kMaxPeaks);
        // R = m^T, m = frame Rz(-2 pi k / N) [Ry(pi)]
        const int z = a.za[b], kk = a.kbin[b], mm = a.mir[b];
        float sp, cp;
        sincospif(-2.0f * (float)kk / (float)a.N, &sp, &cp);
        float R[9];
        for (int i = 0; i < 3; ++i) {
            const float f0 = (float)a.frames[9 * z + 3 * i], f1 = (float)a.frames[9 * z + 3 * i + 1],
                        f2 = (float)a.frames[9 * z + 3 * i + 2];
            float c0 = f0 * cp + f1 * sp, c1 = f1 * cp - f0 * sp, c2 = f2;
            if (mm) {
                c0 = -c0;
                c2 = -c2;
            }
            R[3 * 0 + i] = c0;          // m[i][0] -> R[0][i]
            R[3 * 1 + i] = c1;
            R[3 * 2 + i] = c2;
        }
        __syncwarp();
        for (int m = lane; m < M; m += 32) dmin[m] = CUDART_INF_F;
        for (int c0 = 0; c0 < a.G; c0 += kDelSpotCap) {
            const int c1 = c0 + kDelSpotCap < a.G ? c0 + kDelSpotCap : a.G;
            int ns = 0;
            for (int g0 = c0; g0 < c1; g0 += 32) {
                const int gi = g0 + lane;
                bool spot = false;
                float vx = 0.f, vy = 0.f;
                if (gi < c1) {
                    const float4 g = __ldg(a.refl + gi);
                    vx = R[0] * g.x + R[1] * g.y + R[2] * g.z;
                    vy = R[3] * g.x + R[4] * g.y + R[5] * g.z;
                    const float vz = R[6] * g.x + R[7] * g.y + R[8] * g.z;
                    const float v2 = vx * vx + vy * vy + vz * vz;
                    const float kz = vz - a.inv_lam;
                    const float nkv = sqrtf(vx * vx + vy * vy + kz * kz);
                    const float s = -(v2 - 2.0f * vz * a.inv_lam) / (2.0f * nkv);
                    spot = s * s <= a.s2max;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, spot);
                if (spot) {
                    const int at = ns + __popc(mask & ((1u << lane) - 1u));
                    sx[at] = vx;
                    sy[at] = vy;
                }
                ns += __popc(mask);
            }
            __syncwarp();
            for (int m = lane; m < M; m += 32) {
                const float x = a.qx[p0 + m], y = a.qy[p0 + m];
                float d = dmin[m];
                for (int j = 0; j < ns; ++j) {
                    const float dx = x - sx[j], dy = y - sy[j];
                    d = fminf(d, dx * dx + dy * dy);
                }
                dmin[m] = d;
            }
            __syncwarp();
        }
        for (int m = lane; m < M; m += 32) {
            const float d = sqrtf(dmin[m]);
            if (d < a.r_del) {
                a.qx[p0 + m] = kFarAway;
                a.qy[p0 + m] = kFarAway;
                a.I[p0 + m] = 0.0f;
            } else if (d < a.delta) {
                a.I[p0 + m] *= (d - a.r_del) / (a.delta - a.r_del);
            }
        }
    }
}

struct ScoreAtArgs {
    const float *Psr, *Psi;          // plan, shell-major [Zp][Spad][Fs]
    const float *Xsr, *Xsi;          // chunk, shell-major [nb][Spad][Fs]
    const int2* srange;              // [nb]
    const float* xnorm2;             // [nb]
    int F, N, Spad, Fs;
    int nb, n_matches;
    int64_t off;                     // chunk start in the result arrays
    acom_result res[kMaxMatches];
};

__global__ void __launch_bounds__(256) k_score_at(ScoreAtArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (item >= (int64_t)a.nb * a.n_matches) return;
    const int b = (int)(item / a.n_matches), j = (int)(item % a.n_matches);
    const acom_result& r = a.res[j];
    const int64_t o = a.off + b;
    const int z = r.za_idx[o];
    if (z < 0) {
        if (lane == 0) {
            r.score[o] = 0.0f;
            if (r.score_cos) r.score_cos[o] = 0.0f;
        }
        return;
    }
    const int k = r.phi3_bin[o], mirror = r.mirror[o];
    const int N = a.N, F = a.F;
    const int2 sr = a.srange[b];
    const float invN = 1.0f / (float)N;
    float ore = 0.f, oim = 0.f;
    for (int f = lane; f < F; f += 32) {
        float A = 0.f, B = 0.f, C = 0.f, D = 0.f;
        for (int s = sr.x; s < sr.y; ++s) {
            const int64_t pi = ((int64_t)z * a.Spad + s) * a.Fs + f;
            const int64_t xi = ((int64_t)b * a.Spad + s) * a.Fs + f;
            const float pr = a.Psr[pi], pim = a.Psi[pi], xr = a.Xsr[xi], xim = a.Xsi[xi];
            A = fmaf(pr, xr, A);
            B = fmaf(pim, xim, B);
            C = fmaf(pr, xim, C);
            D = fmaf(pim, xr, D);
        }
        const float dre = (A + B) * invN, dim = (C - D) * invN;
        const float mre = (A - B) * invN, mim = -(C + D) * invN;
        // y_f = (dre - mim) + i (dim + mre) at f, and its partner at N - f
        float sn, cs;
        sincospif(2.0f * (float)(((int64_t)f * k) % N) / (float)N, &sn, &cs);
        const float yr = dre - mim, yi = dim + mre;
        ore += yr * cs - yi * sn;
        oim += yr * sn + yi * cs;
        if (f > 0 && 2 * f < N) {
            const int f2 = N - f;
            sincospif(2.0f * (float)(((int64_t)f2 * k) % N) / (float)N, &sn, &cs);
            const float zr = dre + mim, zi = mre - dim;
            ore += zr * cs - zi * sn;
            oim += zr * sn + zi * cs;
        }
    }
    ore = warp_sum_f(ore);
    oim = warp_sum_f(oim);
    if (lane == 0) {
        const float Cv = mirror ? oim : ore;          // sum = C_dir + i C_mir
        r.score[o] = Cv;
        if (r.score_cos) {
            const float xn = sqrtf(a.xnorm2[b]);
            r.score_cos[o] = xn > 0.f ? Cv / xn : 0.f;
        }
    }
}

}  // namespace

void launch_delete_peaks(const acom_plan_s* p, const acom_peaks_csr* work, const acom_result& r,
                         float r_del, float d_min, cudaStream_t st) {
    DelArgs a{};
    a.refl = p->refl_tab;
    a.G = p->G;
    a.frames = p->frames;
    a.N = p->N;
    a.inv_lam = (float)(1.0 / p->lambda);
    a.s2max = (float)(2.0 * p->sigma_exc * p->sigma_exc * std::log(1.0 / (double)d_min));
    a.r_del = r_del;
    a.delta = (float)p->delta;
    a.row_ptr = work->row_ptr;
    a.qx = const_cast<float*>(work->qx);
    a.qy = const_cast<float*>(work->qy);
    a.I = const_cast<float*>(work->I);
    a.za = r.za_idx;
    a.kbin = r.phi3_bin;
    a.mir = r.mirror;
    a.score = r.score;
    a.nb = work->n_patterns;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (a.nb + kDelWarps - 1) / kDelWarps;
    const int grid = (int)(need < (int64_t)nsm * 16 ? need : (int64_t)nsm * 16);
    if (grid <= 0) return;
    prof_begin(kKMisc, st);
    k_delete_peaks<<<grid, kDelWarps * 32, 0, st>>>(a);
    prof_end(kKMisc, st);
}

void launch_score_at(const acom_plan_s* p, const float* Xsr, const float* Xsi, const int2* srange,
                     const float* xnorm2, int nb, const acom_result* res, int n_matches,
                     int64_t off, cudaStream_t st) {
    ScoreAtArgs a{};
    a.Psr = p->Psr;
    a.Psi = p->Psi;
    a.Xsr = Xsr;
    a.Xsi = Xsi;
    a.srange = srange;
    a.xnorm2 = xnorm2;
    a.F = p->F;
    a.N = p->N;
    a.Spad = p->Spad;
    a.Fs = shell_row_stride(p->F);
    a.nb = nb;
    a.n_matches = n_matches;
    a.off = off;
    for (int j = 0; j < n_matches; ++j) a.res[j] = res[j];
    const int64_t items = (int64_t)nb * n_matches;
    if (items <= 0) return;
    prof_begin(kKMisc, st);
    k_score_at<<<(unsigned)((items + 7) / 8), 256, 0, st>>>(a);
    prof_end(kKMisc, st);
}

}  // namespace acom
