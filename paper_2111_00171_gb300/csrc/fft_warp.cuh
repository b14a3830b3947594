// Warp-level complex FFT (Stockham autosort, radices 4, 2, 3, 5) over a row
// in shared memory: one warp transforms one row, ping-ponging between two
// buffers, with __syncwarp between stages.  Compile-time stages for the bin
// counts used in practice (N = 72, 180, 360, 720), runtime radices otherwise.
// The twiddle table holds tw[i] = (cos, sin)(2 pi i / N).
#pragma once

#include <cuda_runtime.h>

namespace acom {

struct FftRadix {
    int n;
    int r[12];
};

__device__ __forceinline__ float2 cmul_conj(float2 x, float2 t) {   // x * conj(t)
    return make_float2(fmaf(x.x, t.x, x.y * t.y), fmaf(x.y, t.x, -x.x * t.y));
}

// forward transform of src (length N) within one warp; returns the buffer
// holding sum_j src[j] exp(-2 pi i f j / N)
__device__ inline float2* warp_fft_forward(float2* src, float2* dst, int N, const FftRadix& rad,
                                    const float2* __restrict__ tw, int lane) {
    int Ns = 1;
    for (int stg = 0; stg < rad.n; ++stg) {
        const int R = rad.r[stg];
        const int NR = N / R;
        const int tstep = N / (Ns * R);
        for (int j = lane; j < NR; j += 32) {
            const int jq = j / Ns;
            const int jm = j - jq * Ns;
            float2 v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) v[r] = cmul_conj(src[j + r * NR], tw[r * jm * tstep]);
            const int idxD = jq * Ns * R + jm;
            if (R == 4) {
                const float2 a = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
                const float2 b = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
                const float2 c = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
                const float2 d = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
                dst[idxD] = make_float2(a.x + c.x, a.y + c.y);
                dst[idxD + Ns] = make_float2(b.x + d.y, b.y - d.x);
                dst[idxD + 2 * Ns] = make_float2(a.x - c.x, a.y - c.y);
                dst[idxD + 3 * Ns] = make_float2(b.x - d.y, b.y + d.x);
            } else if (R == 2) {
                dst[idxD] = make_float2(v[0].x + v[1].x, v[0].y + v[1].y);
                dst[idxD + Ns] = make_float2(v[0].x - v[1].x, v[0].y - v[1].y);
            } else {
#pragma unroll
                for (int mo = 0; mo < 5; ++mo) {
                    if (mo < R) {
                        float2 o = v[0];
#pragma unroll
                        for (int r = 1; r < 5; ++r) {
                            if (r < R) {
                                const float2 t = cmul_conj(v[r], tw[((r * mo) % R) * NR]);
                                o.x += t.x;
                                o.y += t.y;
                            }
                        }
                        dst[idxD + mo * Ns] = o;
                    }
                }
            }
        }
        __syncwarp();
        float2* t2 = src;
        src = dst;
        dst = t2;
        Ns *= R;
    }
    return src;
}


// Compile-time Stockham stages for the bin counts used in practice: constant
// strides turn the index arithmetic into multiplies and shifts.  The rows must
// start on a 16-byte boundary (the first stage stores 16 bytes at a time).
template <int R>
__device__ __forceinline__ void dft_small(float2* v) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = make_float2(a.x + b.x, a.y + b.y);
        v[1] = make_float2(a.x - b.x, a.y - b.y);
    } else if constexpr (R == 4) {
        const float2 a = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
        const float2 b = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
        const float2 c = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
        const float2 d = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);
        v[0] = make_float2(a.x + c.x, a.y + c.y);
        v[1] = make_float2(b.x + d.y, b.y - d.x);
        v[2] = make_float2(a.x - c.x, a.y - c.y);
        v[3] = make_float2(b.x - d.y, b.y + d.x);
    } else if constexpr (R == 3) {
        // exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
        const float h = 0.8660254037844386f;
        const float2 t1 = make_float2(v[1].x + v[2].x, v[1].y + v[2].y);
        const float2 t2 = make_float2(v[1].x - v[2].x, v[1].y - v[2].y);
        const float2 m1 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
        v[0] = make_float2(v[0].x + t1.x, v[0].y + t1.y);
        v[1] = make_float2(m1.x + h * t2.y, m1.y - h * t2.x);
        v[2] = make_float2(m1.x - h * t2.y, m1.y + h * t2.x);
    } else {
        static_assert(R == 5, "radix");
        // exp(-2 pi i k / 5)
        const float c1 = 0.30901699437494745f, s1 = 0.9510565162951535f;
        const float c2 = -0.8090169943749475f, s2 = 0.5877852522924732f;
        const float2 a1 = make_float2(v[1].x + v[4].x, v[1].y + v[4].y);
        const float2 b1 = make_float2(v[1].x - v[4].x, v[1].y - v[4].y);
        const float2 a2 = make_float2(v[2].x + v[3].x, v[2].y + v[3].y);
        const float2 b2 = make_float2(v[2].x - v[3].x, v[2].y - v[3].y);
        const float2 x0 = v[0];
        const float2 m1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
        const float2 m2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
        // -i (s1 b1 + s2 b2) and -i (s2 b1 - s1 b2)
        const float2 n1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
        const float2 n2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
        v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
        v[1] = make_float2(m1.x + n1.y, m1.y - n1.x);
        v[4] = make_float2(m1.x - n1.y, m1.y + n1.x);
        v[2] = make_float2(m2.x + n2.y, m2.y - n2.x);
        v[3] = make_float2(m2.x - n2.y, m2.y + n2.x);
    }
}

template <int N, int Ns, int R>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                          const float2* __restrict__ tw, int lane) {
    constexpr int NR = N / R;
    constexpr int tstep = N / (Ns * R);
    for (int j = lane; j < NR; j += 32) {
        const int jq = j / Ns;
        const int jm = j - jq * Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 x = src[j + r * NR];
            v[r] = (Ns == 1 || r == 0) ? x : cmul_conj(x, tw[r * jm * tstep]);
        }
        dft_small<R>(v);
        const int idxD = jq * Ns * R + jm;
        if constexpr (Ns == 1 && R % 2 == 0) {
            // the first stage's outputs of a lane are consecutive: 16-byte
            // stores (half the instructions and bank wavefronts of 8-byte ones)
            float4* d4 = reinterpret_cast<float4*>(dst + idxD);
#pragma unroll
            for (int r = 0; r < R / 2; ++r)
                d4[r] = make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y);
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) dst[idxD + r * Ns] = v[r];
        }
    }
    __syncwarp();
}

template <int N, int Ns, int R, int... Rest>
__device__ __forceinline__ float2* fft_run(float2* src, float2* dst, const float2* tw, int lane) {
    fft_stage<N, Ns, R>(src, dst, tw, lane);
    if constexpr (sizeof...(Rest) == 0) {
        return dst;
    } else {
        return fft_run<N, Ns * R, Rest...>(dst, src, tw, lane);
    }
}

__device__ __forceinline__ float2* warp_fft_fixed(float2* src, float2* dst, int N,
                                                  const FftRadix& rad, const float2* tw,
                                                  int lane) {
    switch (N) {
        case 360: return fft_run<360, 1, 4, 2, 3, 3, 5>(src, dst, tw, lane);
        case 180: return fft_run<180, 1, 4, 3, 3, 5>(src, dst, tw, lane);
        case 72: return fft_run<72, 1, 4, 2, 3, 3>(src, dst, tw, lane);
        case 720: return fft_run<720, 1, 4, 4, 3, 3, 5>(src, dst, tw, lane);
        default: return warp_fft_forward(src, dst, N, rad, tw, lane);
    }
}

// radices of N in the order 4, 2, 3, 5; n = 0 when N has another factor
inline FftRadix fft_radices(int N) {
    FftRadix r{};
    int n = N;
    const int cand[4] = {4, 2, 3, 5};
    for (int c = 0; c < 4; ++c)
        while (n % cand[c] == 0 && r.n < 12) {
            r.r[r.n++] = cand[c];
            n /= cand[c];
        }
    if (n != 1) r.n = 0;
    return r;
}

}  // namespace acom
