// Sparse polar raster + Fourier transform along phi3.
//
// One CTA handles one item at a time: a diffraction pattern (its CSR peak
// list) or a zone axis of the orientation plan (the reflections rotated into
// that axis' frame).  Both are rasterised with the same tent
//
//   T(s, j) = max{1 - (1/delta) sqrt((r - q_s)^2 + e + wrap(phi_j - gam)^2 q_s^2), 0}
//
// which is the sparse polar image X of section "Correlation Pattern Matching"
// for a pattern peak (r = q_m, gam = gamma_m, e = 0, weight q_m^gamma
// I_m^(omega/2)) and the plan P0 of section "Generation of an Orientation
// Plan" for a reflection (r = |g'_xy|, gam = gamma_g, e = s_g^2, weight
// |V_g|^omega, rows scaled by q_s^gamma) under uniform shells.
//
// Peaks are sorted by radius, so the peaks reaching a shell are a contiguous
// run.  Each warp owns one shell: for every peak reaching it, the lanes
// evaluate the tent on 32 consecutive bins of the peak's angular window, and
// the window's contribution to X^(s, f) = sum_j X(s, j) exp(-2 pi i f j / N),
// f = 0..N/2, is added by Horner's rule (the transform is linear, so
// overlapping windows simply add; peaks are visited in a fixed order, so the
// sums are deterministic).  Eight shells are staged in shared memory and
// written in the requested layouts; ||X||^2 follows by Parseval.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math_constants.h>

#include <type_traits>

#include "acom_internal.cuh"
#include "fft_warp.cuh"

namespace acom {

// A reflection of the plan: radius, angle, weight and squared excitation error.
struct Peak {
    float r, gam, w, e;
};

// A pattern peak: no excitation error (12 bytes, so that a pattern's peak list
// takes less shared memory).
struct PeakXY {
    float r, gam, w;
    static constexpr float e = 0.f;
};

// Block-ordered compaction: returns this thread's slot among the threads with
// keep == true (in thread order) and the block total in *total.
__device__ inline int block_compact(bool keep, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < nwarps; ++w) {
            int c = s_warp[w];
            s_warp[w] = acc;
            acc += c;
        }
        s_warp[nwarps] = acc;
    }
    __syncthreads();
    int pos = s_warp[warp] + __popc(m & ((1u << lane) - 1u));
    *total = s_warp[nwarps];
    __syncthreads();
    return pos;
}

struct PatternLoader {
    using PeakT = PeakXY;
    static constexpr int kMinBlocks = 3;   // FFT raster CTAs per SM (74.5 KB of shared memory)
    PatternSource src;
    __host__ __device__ void* xb_out() const { return src.xb; }
    __device__ int xb_tiles() const { return src.PTs; }
    __host__ __device__ bool xb_half() const { return src.xb_fp16 != 0; }
    __device__ float* xscale_out() const { return src.xscale; }
    __device__ int xb_k0() const { return src.xb_k0; }
    __device__ int load(int64_t item, PeakXY* sp, int* s_warp, int* err) const {
        const int64_t b0 = src.row_ptr[item];
        const int64_t b1 = src.row_ptr[item + 1];
        int64_t cnt = b1 - b0;
        if (cnt < 0) {
            if (threadIdx.x == 0) atomicOr(err, kErrRowPtr);
            return 0;
        }
        if (cnt > kMaxPeaks) {
            if (threadIdx.x == 0) atomicOr(err, kErrTooManyPeaks);
            return 0;
        }
        const float half_omega = 0.5f * src.omega;
        for (int i = threadIdx.x; i < (int)cnt; i += blockDim.x) {
            float x = src.qx[b0 + i], y = src.qy[b0 + i], I = src.I[b0 + i];
            PeakXY pk;
            if (!(isfinite(x) && isfinite(y) && isfinite(I))) {
                atomicOr(err, kErrNonFinite);
                pk.r = 0.f; pk.gam = 0.f; pk.w = 0.f;
            } else {
                pk.r = sqrtf(x * x + y * y);
                pk.gam = atan2f(y, x);
                pk.w = powf(pk.r, src.gamma_pow) * powf(fmaxf(I, 0.f), half_omega);
            }
            sp[i] = pk;
        }
        __syncthreads();
        return (int)cnt;
    }
};

struct PlanLoader {
    using PeakT = Peak;
    static constexpr int kMinBlocks = 2;
    PlanSource src;
    float delta;
    __host__ __device__ void* xb_out() const { return nullptr; }
    __device__ int xb_tiles() const { return 0; }
    __host__ __device__ bool xb_half() const { return false; }
    __device__ float* xscale_out() const { return nullptr; }
    __device__ int xb_k0() const { return 0; }
    __device__ int load(int64_t item, Peak* sp, int* s_warp, int* err) const {
        const double* R = src.frames + 9 * item;
        double R00 = R[0], R01 = R[1], R02 = R[2], R10 = R[3], R11 = R[4], R12 = R[5],
               R20 = R[6], R21 = R[7], R22 = R[8];
        const double kz = -1.0 / src.lambda;   // beam along -z
        int count = 0;
        for (int base = 0; base < src.G; base += blockDim.x) {
            int i = base + threadIdx.x;
            bool keep = false;
            Peak pk;
            if (i < src.G) {
                double gx = src.g[3 * i], gy = src.g[3 * i + 1], gz = src.g[3 * i + 2];
                // g' = R^T g: the inverse of the zone-axis rotation
                double px = R00 * gx + R10 * gy + R20 * gz;
                double py = R01 * gx + R11 * gy + R21 * gz;
                double pz = R02 * gx + R12 * gy + R22 * gz;
                // Eq. 6 with alpha = 0: s = -g'.(2k + g') / (2 |k + g'|)
                double dot = px * px + py * py + pz * (2.0 * kz + pz);
                double nk = sqrt(px * px + py * py + (kz + pz) * (kz + pz));
                double s = -dot / (2.0 * nk);
                keep = fabs(s) < (double)delta;
                pk.r = (float)sqrt(px * px + py * py);
                pk.gam = (float)atan2(py, px);
                pk.w = (float)src.amp[i];
                pk.e = (float)(s * s);
            }
            int total;
            int pos = block_compact(keep, s_warp, &total);
            if (keep && count + pos < kMaxPeaks) sp[count + pos] = pk;
            count += total;
        }
        if (count > kMaxPeaks) {
            if (threadIdx.x == 0) atomicOr(err, kErrTooManyPeaks);
            count = kMaxPeaks;
        }
        __syncthreads();
        return count;
    }
};

size_t raster_smem_bytes(int N, int F) {
    const int W = kRasterThreads / 32;
    size_t b = 0;
    b += sizeof(Peak) * 2 * kMaxPeaks; // peaks as loaded, and sorted by radius
    b += sizeof(float2) * N;           // twiddles
    b += sizeof(float) * W * 32;       // tent values of the current window chunk
    b += sizeof(float) * 2 * W * F;    // staged spectra of a shell group
    b += sizeof(float) * F;            // per-frequency sums of |X^|^2 over shells
    b += sizeof(int) * 64;             // scratch (compaction, shell range, sums)
    return b;
}

// 2^e for the FP16 copy of pattern item's spectrum (every thread of the CTA,
// one barrier): 2^e B <= kFp16Target with B = sum_m w_m n_m >= max |X^_sf|,
// n_m = min(N, 2 delta / (max(r_m - delta, dq) dphi) + 3) the most bins a
// peak's tent covers on any shell it reaches (tents are at most 1 and X >= 0).
template <class PeakT>
__device__ float fp16_pattern_scale(const PeakT* sp, int np, const RasterGeom& geo, float dphi,
                                    int* red) {
    float b = 0.f;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const PeakT pk = sp[i];
        const float qmin = fmaxf(pk.r - geo.delta, geo.dq);
        const float n = fminf((float)geo.N, floorf(2.0f * geo.delta / (qmin * dphi)) + 3.0f);
        b = fmaf(fabsf(pk.w), n, b);
    }
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = __float_as_int(b);
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += __int_as_float(red[w]);
    if (!(tot > 0.f) || !isfinite(tot)) return 1.0f;
    int e = (int)floorf(log2f(kFp16Target / tot));
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    float sc = ldexpf(1.0f, e);
    if (sc * tot > kFp16Target) sc *= 0.5f;      // guard the log2 rounding
    return sc;
}

template <class Loader, int NF2>
__global__ void __launch_bounds__(kRasterThreads)
k_raster_dft(RasterGeom geo, Loader ld, int64_t n_items, RasterOut out, int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = geo.N, F = geo.F, S = geo.S, Spad = geo.Spad;
    constexpr int W = kRasterThreads / 32;
    using PeakT = typename Loader::PeakT;
    PeakT* sp = reinterpret_cast<PeakT*>(smem);
    PeakT* ss = sp + kMaxPeaks;                               // sorted by radius
    float2* tw = reinterpret_cast<float2*>(ss + kMaxPeaks);   // (cos, sin) of 2 pi i / N
    float* tbuf = reinterpret_cast<float*>(tw + N);
    float* st_re = tbuf + W * 32;
    float* st_im = st_re + W * F;
    float* fn2 = st_im + W * F;
    int* s_int = reinterpret_cast<int*>(fn2 + F);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double c, s;
        sincospi(2.0 * (double)i / (double)N, &s, &c);
        tw[i] = make_float2((float)c, (float)s);
    }
    __syncthreads();
    // z_f = exp(-2 pi i f / N) for this lane's frequencies f = lane + 32 g
    float zr[NF2], zi[NF2];
#pragma unroll
    for (int g = 0; g < NF2; ++g) {
        const int f = (lane + 32 * g) % N;
        zr[g] = tw[f].x;
        zi[g] = -tw[f].y;
    }
    const float delta = geo.delta, d2 = delta * delta, inv_delta = 1.0f / delta;
    const float two_pi = 2.0f * CUDART_PI_F;
    const float dphi = two_pi / (float)N;
    const float inv_dphi = (float)N / two_pi;
    const float invN = 1.0f / (float)N;
    float* my_t = tbuf + warp * 32;

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int np = ld.load(item, sp, s_int, err);
        // rank sort by (radius, index): the peaks reaching a shell are then a
        // contiguous run of the sorted list
        for (int i = threadIdx.x; i < np; i += blockDim.x) {
            const float ri = sp[i].r;
            int rank = 0;
            for (int j = 0; j < np; ++j) {
                const float rj = sp[j].r;
                rank += (rj < ri) || (rj == ri && j < i);
            }
            ss[rank] = sp[i];
        }
        for (int f = threadIdx.x; f < F; f += blockDim.x) fn2[f] = 0.f;
        if (threadIdx.x == 0) {
            s_int[40] = Spad;                // first shell with a non-zero row
            s_int[41] = 0;                   // one past the last
        }
        __syncthreads();
        const bool half = ld.xb_out() && ld.xb_half();
        float xsc = 1.0f;
        if (half) {
            xsc = fp16_pattern_scale(sp, np, geo, dphi, s_int + 56);
            if (threadIdx.x == 0) ld.xscale_out()[item] = xsc;
        }
        for (int s0 = 0; s0 < Spad; s0 += W) {
            const int s = s0 + warp;
            float ar[NF2], ai[NF2];
#pragma unroll
            for (int g = 0; g < NF2; ++g) ar[g] = ai[g] = 0.f;
            bool nonzero = false;
            if (s < S) {
                const float qs = (float)(s + 1) * geo.dq;
                const float qs2 = qs * qs;
                const float rscale = geo.shell_power ? powf(qs, geo.gamma_pow) : 1.0f;
                // sorted peaks with |r - q_s| < delta
                int lo = 0, hi = 0;
                for (int base = 0; base < np; base += 32) {
                    const int m = base + lane;
                    const float r = m < np ? ss[m].r : CUDART_INF_F;
                    lo += __popc(__ballot_sync(0xffffffffu, r <= qs - delta));
                    hi += __popc(__ballot_sync(0xffffffffu, r < qs + delta));
                }
                for (int m = lo; m < hi; ++m) {
                    const PeakT pk = ss[m];
                    const float dr = pk.r - qs;
                    const float a2 = dr * dr + pk.e;
                    if (!(a2 < d2) || pk.w == 0.f) continue;          // tent is zero on this shell
                    const float hw = sqrtf(d2 - a2) / qs;            // angular half width
                    int jlo, cnt;
                    if (hw >= CUDART_PI_F) {
                        jlo = 0;
                        cnt = N;
                    } else {
                        jlo = (int)floorf((pk.gam - hw) * inv_dphi) - 1;
                        const int jhi = (int)ceilf((pk.gam + hw) * inv_dphi) + 1;
                        cnt = min(jhi - jlo + 1, N);
                    }
                    const float wgt = pk.w * rscale;
                    jlo %= N;                                       // first bin in [0, N)
                    if (jlo < 0) jlo += N;
                    // chunks of 32 consecutive bins (mod N, which the transform
                    // sees as consecutive): tent values, then Horner's rule
                    for (int c0 = 0; c0 < cnt; c0 += 32) {
                        const int t = c0 + lane;
                        float tv = 0.f;
                        if (t < cnt) {
                            int j = jlo + t;                    // t < cnt <= N
                            if (j >= N) j -= N;
                            float d = (float)j * dphi - pk.gam;
                            d -= two_pi * floorf((d + CUDART_PI_F) / two_pi);   // wrap to [-pi, pi)
                            const float tt = 1.0f - sqrtf(a2 + d * d * qs2) * inv_delta;
                            tv = tt > 0.f ? wgt * tt : 0.f;
                        }
                        my_t[lane] = tv;
                        __syncwarp();
                        const int L = min(32, cnt - c0);
                        float hr[NF2], hi_[NF2];
#pragma unroll
                        for (int g = 0; g < NF2; ++g) hr[g] = hi_[g] = 0.f;
                        for (int p = L - 1; p >= 0; --p) {
                            const float v = my_t[p];
#pragma unroll
                            for (int g = 0; g < NF2; ++g) {
                                const float tq = fmaf(hr[g], zr[g], fmaf(-hi_[g], zi[g], v));
                                hi_[g] = fmaf(hr[g], zi[g], hi_[g] * zr[g]);
                                hr[g] = tq;
                            }
                        }
                        __syncwarp();
                        int j0 = jlo + c0;
                        if (j0 >= N) j0 -= N;
#pragma unroll
                        for (int g = 0; g < NF2; ++g) {
                            const int prod = (lane + 32 * g) * j0;
                            const int q = __float2int_rz((float)prod * invN);
                            int idx = prod - q * N;
                            if (idx >= N) idx -= N;
                            if (idx < 0) idx += N;
                            const float2 w = tw[idx];            // exp(+i theta): conjugate it
                            ar[g] = fmaf(hr[g], w.x, fmaf(hi_[g], w.y, ar[g]));
                            ai[g] = fmaf(hi_[g], w.x, fmaf(-hr[g], w.y, ai[g]));
                        }
                    }
                    nonzero = true;
                }
                if (lane == 0 && nonzero) {
                    atomicMin(&s_int[40], s);
                    atomicMax(&s_int[41], s + 1);
                }
            }
#pragma unroll
            for (int g = 0; g < NF2; ++g) {
                const int f = lane + 32 * g;
                if (f < F) {
                    st_re[warp * F + f] = ar[g];
                    st_im[warp * F + f] = ai[g];
                }
            }
            __syncthreads();
            for (int f = threadIdx.x; f < F; f += blockDim.x) {
                float acc = fn2[f];
                for (int w = 0; w < W; ++w)
                    acc = fmaf(st_re[w * F + f], st_re[w * F + f],
                               fmaf(st_im[w * F + f], st_im[w * F + f], acc));
                fn2[f] = acc;
            }
            if (ld.xb_out()) {
                // BF16 copy in the tensor-core tile layout: 64-pattern tiles whose
                // 16-row groups hold 8 patterns' real rows, then their imaginary rows
                const int64_t tile = item / 64, r = item % 64;
                for (int e = threadIdx.x; e < 2 * F; e += blockDim.x) {
                    const int f = e >> 1, c = e & 1;
                    const float* srcv = c ? st_im : st_re;
                    __align__(16) unsigned short v[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        const float x = srcv[w * F + f];
                        v[w] = half ? __half_as_ushort(__float2half_rn(x * xsc))
                                    : __bfloat16_as_ushort(__float2bfloat16_rn(x));
                    }
                    const int64_t row = ((int64_t)f * ld.xb_tiles() + tile) * 128 + (r >> 3) * 16 + c * 8 + (r & 7);
                    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned short*>(ld.xb_out()) +
                                              row * Spad + s0) = *reinterpret_cast<uint4*>(v);
                }
            }
            if (out.re) {
                const int64_t obase = item * (int64_t)F * Spad + s0;
                for (int e = threadIdx.x; e < F * W; e += blockDim.x) {
                    const int f = e / W, w = e - f * W;
                    out.re[obase + (int64_t)f * Spad + w] = st_re[w * F + f];
                    out.im[obase + (int64_t)f * Spad + w] = st_im[w * F + f];
                }
            }
            if (out.sre) {
                // whole padded rows, the pad frequencies as zeros
                const int Fs = shell_row_stride(F);
                const int64_t sbase = (item * (int64_t)Spad + s0) * Fs;
                for (int e = threadIdx.x; e < Fs * W; e += blockDim.x) {
                    const int w = e / Fs, f = e - w * Fs;
                    const bool in = f < F;
                    out.sre[sbase + (int64_t)w * Fs + f] = in ? st_re[w * F + f] : 0.f;
                    out.sim[sbase + (int64_t)w * Fs + f] = in ? st_im[w * F + f] : 0.f;
                }
            }
            __syncthreads();
        }
        if (out.fnorm)
            for (int f = threadIdx.x; f < F; f += blockDim.x)
                out.fnorm[item * (int64_t)F + f] = sqrtf(fn2[f]);
        if (threadIdx.x == 0) {
            if (out.srange) {
                const int lo = s_int[40], hi = s_int[41];
                out.srange[item] = lo < hi ? make_int2(lo, hi) : make_int2(0, 0);
            }
        }
        if (out.sumsq) {
            // Parseval: sum_j X^2 = (1/N) sum_f w_f sum_s |X^_f|^2
            float e = 0.f;
            for (int f = threadIdx.x; f < F; f += blockDim.x)
                e += ((f == 0 || 2 * f == N) ? 1.f : 2.f) * fn2[f];
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (lane == 0) st_re[warp] = e;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.f;
                for (int w = 0; w < W; ++w) t += st_re[w];
                out.sumsq[item] = t * invN;
            }
        }
        __syncthreads();
    }
}

template <class Loader, int NF2>
static void launch_raster_nf(const RasterGeom& geo, const Loader& ld, int64_t n_items,
                             const RasterOut& out, int* err, cudaStream_t st, int cls) {
    size_t smem = raster_smem_bytes(geo.N, geo.F);
    set_max_dynamic_smem((const void*)k_raster_dft<Loader, NF2>, smem);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_dft<Loader, NF2>,
                                                  kRasterThreads, smem);
    int64_t grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (grid > n_items) grid = n_items;
    prof_begin(cls, st);
    k_raster_dft<Loader, NF2><<<(unsigned)grid, kRasterThreads, smem, st>>>(
        geo, ld, n_items, out, err);
    prof_end(cls, st);
}


// ---------------------------------------------------------------------------
// FFT variant (N = 2^a 3^b 5^c): each warp rasterises two shells into the real
// and imaginary parts of one complex row of N bins and transforms it with a
// Stockham mixed-radix FFT (radices 4, 2, 3, 5); the spectra of the two real
// rows are separated by the conjugate symmetry of real transforms.
// ---------------------------------------------------------------------------

constexpr int kFftTile = 16;      // shells per 16-bit staging tile: 8 pairs, one per warp
constexpr int kFftStageWords = kFftTile / 2 + 1;   // words per staged row: 8 shell pairs + pad
constexpr int kPeakSortPerThread = (kMaxPeaks + kRasterThreads - 1) / kRasterThreads;
constexpr int kMaxFPerLane = 12;  // F <= 361 (N <= 720)

size_t raster_fft_smem_bytes(int N, int F, size_t peak_bytes) {
    const int W = kRasterThreads / 32;
    size_t b = 0;
    b += peak_bytes * kMaxPeaks;                         // peaks, sorted in place by radius
    b += sizeof(float2) * N;                             // twiddles
    b += sizeof(float2) * 2 * W * N;                     // per-warp row and transform buffer
    b += sizeof(uint32_t) * 2 * F * kFftStageWords;      // BF16 staging of a shell tile
    b += sizeof(int) * 64;                               // scratch
    if (N == 360) b += sizeof(uint16_t) * 2 * 360;       // prime-factor input, output positions
    return b;
}

// PFA: N = 360 and its prime-factor transform, compiled alone (the radix
// transforms' code stays out of this kernel), six frequencies per lane.
// XB: the tensor-core copy written, 0 none (FP32 contraction or plan), 1 BF16,
// 2 FP16 of 2^e X^ (each instance carries only its own output code).
template <class Loader, bool PFA, int XB>
__global__ void __launch_bounds__(kRasterThreads, Loader::kMinBlocks)
k_raster_fft(RasterGeom geo, Loader ld, int64_t n_items, RasterOut out, FftRadix rad,
             int* err) {
    constexpr int kFL = PFA ? 6 : kMaxFPerLane;     // frequencies per lane (F <= 32 kFL)
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = geo.N, F = geo.F, S = geo.S, Spad = geo.Spad;
    const int Fs = shell_row_stride(F);
    constexpr int W = kRasterThreads / 32;
    using PeakT = typename Loader::PeakT;
    PeakT* sp = reinterpret_cast<PeakT*>(smem);
    float2* tw = reinterpret_cast<float2*>(sp + kMaxPeaks);
    float2* zb = tw + N;
    float2* zt = zb + W * N;
    uint32_t* stage = reinterpret_cast<uint32_t*>(zt + W * N);   // [2F][kFftStageWords]
    int* s_int = reinterpret_cast<int*>(stage + 2 * F * kFftStageWords);
    // N = 360: the rows hold the bins in the prime-factor transform's input
    // order (bin j at s_perm[j]), the transform runs in place and leaves
    // frequency f at s_pout[f]
    constexpr bool pfa = PFA;
    uint16_t* s_perm = reinterpret_cast<uint16_t*>(s_int + 64);
    uint16_t* s_pout = s_perm + 360;
    float* scratch = reinterpret_cast<float*>(zb);     // after the last transform of an item

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double c, sn;
        sincospi(2.0 * (double)i / (double)N, &sn, &c);
        tw[i] = make_float2((float)c, (float)sn);
    }
    if (pfa)
        for (int i = threadIdx.x; i < 360; i += blockDim.x) {
            s_perm[i] = (uint16_t)pfa360_in(i);
            s_pout[i] = (uint16_t)pfa360_out(i);
        }
    __syncthreads();
    const float delta = geo.delta, d2 = delta * delta, inv_delta = 1.0f / delta;
    const float two_pi = 2.0f * CUDART_PI_F;
    const float dphi = two_pi / (float)N;
    const float inv_dphi = (float)N / two_pi;
    // windows narrower than this never reach an angle offset of pi, so the
    // offsets need no wrapping
    const float hw_nowrap = CUDART_PI_F - 3.0f * dphi;
    const float invN = 1.0f / (float)N;
    float2* z = zb + warp * N;
    float2* zz = zt + warp * N;
    __nv_bfloat16* xb = XB ? reinterpret_cast<__nv_bfloat16*>(ld.xb_out()) : nullptr;

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int np = ld.load(item, sp, s_int, err);
        // rank sort by (radius, index), in place: every thread holds its peaks
        // and their ranks in registers across the barrier, then stores them
        {
            PeakT mine[kPeakSortPerThread];
            int rk[kPeakSortPerThread];
#pragma unroll
            for (int k = 0; k < kPeakSortPerThread; ++k) {
                const int i = threadIdx.x + k * kRasterThreads;
                rk[k] = -1;
                if (i < np) {
                    mine[k] = sp[i];
                    const float ri = mine[k].r;
                    int rank = 0;
                    for (int j = 0; j < np; ++j) {
                        const float rj = sp[j].r;
                        rank += (rj < ri) || (rj == ri && j < i);
                    }
                    rk[k] = rank;
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kPeakSortPerThread; ++k)
                if (rk[k] >= 0) sp[rk[k]] = mine[k];
        }
        if (threadIdx.x == 0) {
            s_int[40] = Spad;
            s_int[41] = 0;
        }
        if (threadIdx.x < 16) s_int[16 + threadIdx.x] = 0;    // shells the tents reach
        __syncthreads();
        constexpr bool half = XB == 2;
        float xsc = 1.0f;
        if (half) {
            xsc = fp16_pattern_scale(sp, np, geo, dphi, s_int + 56);
            if (threadIdx.x == 0) ld.xscale_out()[item] = xsc;
        }
        float fa[kFL];                  // sum over this warp's shells of |X^_sf|^2, f = lane + 32 k
#pragma unroll
        for (int k = 0; k < kFL; ++k) fa[k] = 0.f;
        int w_lo = Spad, w_hi = 0;      // this warp's non-zero shells

        for (int t0 = 0; t0 < Spad; t0 += kFftTile) {
            // the 16-bit copy of a tile the contraction never reads is skipped
            const bool stg = XB != 0 && t0 + kFftTile > ld.xb_k0();
            // pairs warp and warp + W of the tile
            for (int pp = warp; pp < kFftTile / 2; pp += W) {
                const int sA = t0 + 2 * pp;
                // One pass over the peaks reaching either shell of the pair (radius
                // within delta of q_A or q_B): the half-warps take alternate peaks,
                // each into its own row (z, zz), and every bin of a peak's window
                // gets both shells' tents (x: shell sA, y: shell sA + 1).  The two
                // rows are summed before the transform, a fixed order.  A pair no
                // peak's radius reaches is all zero: no rows, no transform.
                bool inA_any = false, inB_any = false;
                const bool vB = sA + 1 < S;
                const float qA = (float)(sA + 1) * geo.dq, qB = (float)(sA + 2) * geo.dq;
                int lo = 0, hi = 0;
                if (sA < S) {
                    const float qhi = vB ? qB : qA;
                    for (int base = 0; base < np; base += 32) {
                        const int m = base + lane;
                        const float r = m < np ? sp[m].r : CUDART_INF_F;
                        lo += __popc(__ballot_sync(0xffffffffu, r <= qA - delta));
                        hi += __popc(__ballot_sync(0xffffffffu, r < qhi + delta));
                    }
                }
                if (hi > lo) {
                    // rows start on 16-byte boundaries (N even: 16-byte accesses)
                    if ((N & 1) == 0) {
                        float4* z4 = reinterpret_cast<float4*>(z);
                        float4* zz4 = reinterpret_cast<float4*>(zz);
                        for (int j = lane; j < N / 2; j += 32) {
                            z4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                            zz4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    } else {
                        for (int j = lane; j < N; j += 32) {
                            z[j] = make_float2(0.f, 0.f);
                            zz[j] = make_float2(0.f, 0.f);
                        }
                    }
                    __syncwarp();
                    const float qA2 = qA * qA, qB2 = qB * qB;
                    const float iqA = 1.0f / qA, iqB = 1.0f / qB;
                    const float rsA = geo.shell_power ? powf(qA, geo.gamma_pow) : 1.0f;
                    const float rsB = geo.shell_power ? powf(qB, geo.gamma_pow) : 1.0f;
                    const int half = lane >> 4, hl = lane & 15;
                    const unsigned hmask = 0xffffu << (16 * half);
                    float2* acc = half ? zz : z;
                    // every condition below is uniform over a half-warp (its lanes
                    // share the peak), so the half-warp syncs pair up; they order a
                    // bin's updates by different lanes for successive peaks
                    for (int m = lo + half; m < hi; m += 2) {
                        const PeakT pk = sp[m];
                        const float drA = pk.r - qA, drB = pk.r - qB;
                        const float a2A = fmaf(drA, drA, pk.e), a2B = fmaf(drB, drB, pk.e);
                        const bool inA = a2A < d2 && pk.w != 0.f, inB = vB && a2B < d2 && pk.w != 0.f;
                        if (!inA && !inB) continue;
                        inA_any |= inA;
                        inB_any |= inB;
                        // window half-widths (the window keeps a bin of margin on each
                        // side, and each bin's tent is tested, so an approximate root
                        // cannot drop a bin)
                        float hwA = 0.f, hwB = 0.f;
                        if (inA) asm("sqrt.approx.f32 %0, %1;" : "=f"(hwA) : "f"(d2 - a2A));
                        if (inB) asm("sqrt.approx.f32 %0, %1;" : "=f"(hwB) : "f"(d2 - a2B));
                        hwA *= iqA;
                        hwB *= iqB;
                        const float hw = fmaxf(hwA, hwB);
                        const float wA = inA ? pk.w * rsA : 0.f, wB = inB ? pk.w * rsB : 0.f;
                        if (hw < hw_nowrap) {
                            // bins jlo .. jlo + cnt - 1 around gamma; the offset of bin
                            // jlo + t is d0 + t dphi, within (-pi, pi) by the bound on hw
                            const int jlo = __float2int_rd((pk.gam - hw) * inv_dphi) - 1;
                            const int jhi = __float2int_ru((pk.gam + hw) * inv_dphi) + 1;
                            const int cnt = jhi - jlo + 1;
                            const float d0 = fmaf((float)jlo, dphi, -pk.gam);
                            int jw = jlo;
                            if (jw < 0) jw += N;
                            if (jw < 0) jw += N;
                            for (int t = hl; t < cnt; t += 16) {
                                int j = jw + t;
                                if (j >= N) j -= N;
                                const float d = fmaf((float)t, dphi, d0), dd = d * d;
                                float sa, sb;
                                asm("sqrt.approx.f32 %0, %1;" : "=f"(sa) : "f"(fmaf(dd, qA2, a2A)));
                                asm("sqrt.approx.f32 %0, %1;" : "=f"(sb) : "f"(fmaf(dd, qB2, a2B)));
                                const float ta = inA ? 1.0f - sa * inv_delta : 0.f;
                                const float tb = inB ? 1.0f - sb * inv_delta : 0.f;
                                if (ta > 0.f || tb > 0.f) {
                                    const int jj = pfa ? (int)s_perm[j] : j;
                                    float2 v = acc[jj];
                                    if (ta > 0.f) v.x = fmaf(wA, ta, v.x);
                                    if (tb > 0.f) v.y = fmaf(wB, tb, v.y);
                                    acc[jj] = v;
                                }
                            }
                        } else {
                            // a window of (nearly) the whole circle: every bin, offsets wrapped
                            for (int j = hl; j < N; j += 16) {
                                float d = fmaf((float)j, dphi, -pk.gam);
                                if (d >= CUDART_PI_F) d -= two_pi;
                                if (d < -CUDART_PI_F) d += two_pi;
                                const float dd = d * d;
                                float sa, sb;
                                asm("sqrt.approx.f32 %0, %1;" : "=f"(sa) : "f"(fmaf(dd, qA2, a2A)));
                                asm("sqrt.approx.f32 %0, %1;" : "=f"(sb) : "f"(fmaf(dd, qB2, a2B)));
                                const float ta = inA ? 1.0f - sa * inv_delta : 0.f;
                                const float tb = inB ? 1.0f - sb * inv_delta : 0.f;
                                if (ta > 0.f || tb > 0.f) {
                                    const int jj = pfa ? (int)s_perm[j] : j;
                                    float2 v = acc[jj];
                                    if (ta > 0.f) v.x = fmaf(wA, ta, v.x);
                                    if (tb > 0.f) v.y = fmaf(wB, tb, v.y);
                                    acc[jj] = v;
                                }
                            }
                        }
                        __syncwarp(hmask);
                    }
                }
                const bool anyA = __any_sync(0xffffffffu, inA_any);
                const bool anyB = __any_sync(0xffffffffu, inB_any);
                if (anyA) {
                    w_lo = min(w_lo, sA);
                    w_hi = max(w_hi, sA + 1);
                }
                if (anyB) {
                    w_lo = min(w_lo, sA + 1);
                    w_hi = max(w_hi, sA + 2);
                }
                const bool any = anyA || anyB;
                if (lane == 0 && any && out.rmask)
                    atomicOr(reinterpret_cast<unsigned*>(s_int + 16 + (sA >> 5)),
                             (anyA ? 1u << (sA & 31) : 0u) | (anyB ? 1u << ((sA + 1) & 31) : 0u));
                if (any && pfa) {
                    __syncwarp();
                    warp_pfa360(z, zz, lane);     // sums the two rows as it loads them
                } else if (any) {
                    __syncwarp();
                    if ((N & 1) == 0) {
                        float4* z4 = reinterpret_cast<float4*>(z);
                        const float4* zz4 = reinterpret_cast<const float4*>(zz);
                        for (int j = lane; j < N / 2; j += 32) {
                            const float4 u = zz4[j];
                            float4 v = z4[j];
                            v.x += u.x;
                            v.y += u.y;
                            v.z += u.z;
                            v.w += u.w;
                            z4[j] = v;
                        }
                    } else {
                        for (int j = lane; j < N; j += 32) {
                            const float2 u = zz[j];
                            float2 v = z[j];
                            v.x += u.x;
                            v.y += u.y;
                            z[j] = v;
                        }
                    }
                    __syncwarp();
                }
                const float2* Z =
                    !any ? nullptr : (pfa ? z : warp_fft_fixed(z, zz, N, rad, tw, lane));
                // real rows a (shell sA), b (shell sA + 1) from Z = FFT(a + i b):
                //   A_f = (Z_f + conj Z_{N-f}) / 2,  B_f = -i (Z_f - conj Z_{N-f}) / 2
                const int64_t srow = (item * (int64_t)Spad + sA) * Fs;
                const int pw = pp;                               // word of the pair in a staged row
#pragma unroll
                for (int k = 0; k < kFL; ++k) {
                    const int f = lane + 32 * k;
                    if (f >= Fs) break;
                    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
                    if (any && f < F) {
                        const int fc = f == 0 ? 0 : N - f;
                        const float2 zf = Z[pfa ? (int)s_pout[f] : f];
                        const float2 zc = Z[pfa ? (int)s_pout[fc] : fc];
                        ar = 0.5f * (zf.x + zc.x);
                        ai = 0.5f * (zf.y - zc.y);
                        br = 0.5f * (zf.y + zc.y);
                        bi = 0.5f * (zc.x - zf.x);
                    }
                    if (out.sre && (any || !out.rmask)) {
                        out.sre[srow + f] = ar;
                        out.sim[srow + f] = ai;
                        out.sre[srow + Fs + f] = br;
                        out.sim[srow + Fs + f] = bi;
                    }
                    if (f < F) {
                        fa[k] = fmaf(ar, ar, fmaf(ai, ai, fmaf(br, br, fmaf(bi, bi, fa[k]))));
                        if (XB == 0 && out.re) {
                            const int64_t o = (item * (int64_t)F + f) * Spad + sA;
                            out.re[o] = ar;
                            out.re[o + 1] = br;
                            out.im[o] = ai;
                            out.im[o + 1] = bi;
                        }
                        if (XB == 2 && stg) {
                            const __half2 vr = __floats2half2_rn(ar * xsc, br * xsc);
                            const __half2 vi = __floats2half2_rn(ai * xsc, bi * xsc);
                            stage[f * kFftStageWords + pw] = *reinterpret_cast<const uint32_t*>(&vr);
                            stage[(F + f) * kFftStageWords + pw] = *reinterpret_cast<const uint32_t*>(&vi);
                        } else if (XB == 1 && stg) {
                            const __nv_bfloat162 vr = __floats2bfloat162_rn(ar, br);
                            const __nv_bfloat162 vi = __floats2bfloat162_rn(ai, bi);
                            stage[f * kFftStageWords + pw] = *reinterpret_cast<const uint32_t*>(&vr);
                            stage[(F + f) * kFftStageWords + pw] = *reinterpret_cast<const uint32_t*>(&vi);
                        }
                    }
                }
                __syncwarp();
            }
            if (stg) {
                // the tile's BF16 copy in the tensor-core layout (64-pattern tiles whose
                // 16-row groups hold 8 patterns' real rows, then their imaginary rows):
                // 32 bytes (16 shells) per row
                __syncthreads();
                const int64_t tile = item / 64, r = item % 64;
                const int64_t rbase = (r >> 3) * 16 + (r & 7);
                for (int e = threadIdx.x; e < 2 * F * 2; e += blockDim.x) {
                    const int row = e >> 1, q = e & 1;
                    const int c = row >= F, f = row - c * F;
                    const uint32_t* src = stage + row * kFftStageWords + 4 * q;
                    const uint4 v = make_uint4(src[0], src[1], src[2], src[3]);
                    const int64_t grow = ((int64_t)f * ld.xb_tiles() + tile) * 128 + rbase + c * 8;
                    *reinterpret_cast<uint4*>(xb + grow * Spad + t0 + 8 * q) = v;
                }
                __syncthreads();
            }
        }
        if (w_lo < w_hi) {
            atomicMin(&s_int[40], w_lo);
            atomicMax(&s_int[41], w_hi);
        }
        __syncthreads();                 // every transform of the item is done
#pragma unroll
        for (int k = 0; k < kFL; ++k) {
            const int f = lane + 32 * k;
            if (f < F) scratch[warp * F + f] = fa[k];
        }
        __syncthreads();
        float e = 0.f;
        for (int f = threadIdx.x; f < F; f += blockDim.x) {
            float fn2 = 0.f;
            for (int w = 0; w < W; ++w) fn2 += scratch[w * F + f];
            if (out.fnorm) out.fnorm[item * (int64_t)F + f] = sqrtf(fn2);
            e += ((f == 0 || 2 * f == N) ? 1.f : 2.f) * fn2;
        }
        if (threadIdx.x == 0 && out.srange) {
            const int lo = s_int[40], hi = s_int[41];
            out.srange[item] = lo < hi ? make_int2(lo, hi) : make_int2(0, 0);
        }
        if (out.rmask && threadIdx.x < (Spad >> 5))
            out.rmask[item * (int64_t)(Spad >> 5) + threadIdx.x] = (uint32_t)s_int[16 + threadIdx.x];
        if (out.sumsq) {
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (lane == 0) s_int[48 + warp] = __float_as_int(e);
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = 0.f;
                for (int w = 0; w < W; ++w) t += __int_as_float(s_int[48 + w]);
                out.sumsq[item] = t * invN;
            }
        }
        __syncthreads();
    }
}

template <class Loader>
static bool launch_raster_fft(const RasterGeom& geo, const Loader& ld, int64_t n_items,
                              const RasterOut& out, int* err, cudaStream_t st, int cls) {
    const FftRadix rad = fft_radices(geo.N);
    if (rad.n == 0 || geo.Spad % kFftTile != 0 || geo.F > 32 * kMaxFPerLane) return false;
    const size_t smem = raster_fft_smem_bytes(geo.N, geo.F, sizeof(typename Loader::PeakT));
    if (smem > 227 * 1024) return false;
    const bool pfa = geo.N == 360;
    const int xk = ld.xb_out() ? (ld.xb_half() ? 2 : 1) : 0;
    auto pick = [&](auto pfa_c) -> const void* {
        constexpr bool P = decltype(pfa_c)::value;
        return xk == 2 ? (const void*)k_raster_fft<Loader, P, 2>
                       : (xk == 1 ? (const void*)k_raster_fft<Loader, P, 1>
                                  : (const void*)k_raster_fft<Loader, P, 0>);
    };
    const void* kern = pfa ? pick(std::true_type{}) : pick(std::false_type{});
    set_max_dynamic_smem(kern, smem);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRasterThreads, smem);
    int64_t grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (grid > n_items) grid = n_items;
    prof_begin(cls, st);
    void* args[] = {(void*)&geo, (void*)&ld, (void*)&n_items, (void*)&out, (void*)&rad, (void*)&err};
    cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kRasterThreads), args, smem, st);
    prof_end(cls, st);
    return true;
}

// frequencies per lane: the smallest compiled count covering F = N/2 + 1
template <class Loader>
static void launch_raster(const RasterGeom& geo, const Loader& ld, int64_t n_items,
                          const RasterOut& out, int* err, cudaStream_t st, int cls) {
    if (n_items <= 0) return;
    if (launch_raster_fft(geo, ld, n_items, out, err, st, cls)) return;
    const int nf2 = (geo.F + 31) / 32;
    if (nf2 <= 2)
        launch_raster_nf<Loader, 2>(geo, ld, n_items, out, err, st, cls);
    else if (nf2 <= 3)
        launch_raster_nf<Loader, 3>(geo, ld, n_items, out, err, st, cls);
    else if (nf2 <= 6)
        launch_raster_nf<Loader, 6>(geo, ld, n_items, out, err, st, cls);
    else
        launch_raster_nf<Loader, 12>(geo, ld, n_items, out, err, st, cls);
}

void launch_raster_plan(const RasterGeom& geo, const PlanSource& src, int Z,
                        const RasterOut& out, int* err, cudaStream_t st) {
    PlanLoader ld{src, geo.delta};
    launch_raster(geo, ld, Z, out, err, st, kKRasterPlan);
}

void launch_raster_patterns(const RasterGeom& geo, const PatternSource& src,
                            const RasterOut& out, int* err, cudaStream_t st) {
    PatternLoader ld{src};
    launch_raster(geo, ld, src.n_items, out, err, st, kKRasterPatterns);
}

// P = A P0 with A = 1/||P0||_2 (0 for an empty slice): the transform is
// linear, so the spectrum rows are scaled after the fact.
// rows of item y scaled by 1 / sqrt(sumsq[y]) (0 for an all-zero item);
// row_elems is a multiple of 4 (16-byte accesses), blockIdx.y is the item
__global__ void k_scale_rows(float* re, float* im, const float* sumsq, int row_elems) {
    const int item = blockIdx.y;
    const float ss = sumsq[item];
    const float a = ss > 0.f ? rsqrtf(ss) : 0.f;
    float4* r4 = reinterpret_cast<float4*>(re + (int64_t)item * row_elems);
    float4* i4 = reinterpret_cast<float4*>(im + (int64_t)item * row_elems);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < row_elems / 4; q += gridDim.x * blockDim.x) {
        float4 u = r4[q], v = i4[q];
        u.x *= a; u.y *= a; u.z *= a; u.w *= a;
        v.x *= a; v.y *= a; v.z *= a; v.w *= a;
        r4[q] = u;
        i4[q] = v;
    }
}

void launch_scale_rows(float* re, float* im, const float* sumsq, int items, int row_elems,
                       cudaStream_t st) {
    if (items <= 0) return;
    const dim3 grid((unsigned)((row_elems / 4 + 255) / 256), (unsigned)items);
    prof_begin(kKScale, st);
    k_scale_rows<<<grid, 256, 0, st>>>(re, im, sumsq, row_elems);
    prof_end(kKScale, st);
}

// [items][F][Spad] planar -> [items][S][F][2] interleaved
__global__ void k_spectra_export(const float* re, const float* im, int items, int F, int Spad,
                                 int S, float* dst) {
    int64_t total = (int64_t)items * S * F;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int f = (int)(i % F);
        int64_t t = i / F;
        int s = (int)(t % S);
        int64_t item = t / S;
        int64_t src = (item * F + f) * Spad + s;
        dst[2 * i] = re[src];
        dst[2 * i + 1] = im[src];
    }
}

void launch_spectra_export(const float* re, const float* im, int items, int F, int Spad, int S,
                           float* dst, cudaStream_t st) {
    int64_t total = (int64_t)items * S * F;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    if (blocks > 0) {
        prof_begin(kKMisc, st);
        k_spectra_export<<<blocks, 256, 0, st>>>(re, im, items, F, Spad, S, dst);
        prof_end(kKMisc, st);
    }
}

}  // namespace acom
