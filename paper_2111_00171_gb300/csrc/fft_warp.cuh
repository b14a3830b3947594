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

// ---------------------------------------------------------------------------
// N = 360 as a prime-factor (Good-Thomas) transform over 8 x 9 x 5, factors
// pairwise coprime, so no twiddle factors between the stages.  The row holds
// the input permuted: bin j at
//   pfa360_in(j) = 45 n1 + 5 n2 + n3,  n1 = 5j mod 8, n2 = 7j mod 9, n3 = 3j mod 5,
// the unique (n1, n2, n3) with j = (45 n1 + 40 n2 + 72 n3) mod 360.  With
// w_M = exp(-2 pi i / M),
//   X[f] = sum_{n1,n2,n3} x[n1, n2, n3] w_8^(n1 f) w_9^(n2 f) w_5^(n3 f)
// because w_360^(45 n1 f) = w_8^(n1 f) and so on, and w_8^(n1 f) depends on f
// mod 8 only: the transform is a DFT of length 8 along n1, 9 along n2 and 5
// along n3, computed in place (each small DFT writes the positions it read),
// and X[f] ends at pfa360_out(f) = 45 (f mod 8) + 5 (f mod 9) + (f mod 5).
// ---------------------------------------------------------------------------
__host__ __device__ inline int pfa360_in(int j) {
    return 45 * ((5 * j) % 8) + 5 * ((7 * j) % 9) + (3 * j) % 5;
}
__host__ __device__ inline int pfa360_out(int f) { return 45 * (f % 8) + 5 * (f % 9) + f % 5; }

__device__ __forceinline__ void dft8(float2* v) {
    // split into even and odd outputs: b_k = v_k + v_(k+4) gives X_(2m) = DFT4(b)_m,
    // c_k = (v_k - v_(k+4)) w_8^k gives X_(2m+1) = DFT4(c)_m
    const float r2 = 0.7071067811865476f;     // sqrt(1/2)
    float2 b[4], c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        b[k] = make_float2(v[k].x + v[k + 4].x, v[k].y + v[k + 4].y);
        c[k] = make_float2(v[k].x - v[k + 4].x, v[k].y - v[k + 4].y);
    }
    c[1] = make_float2(r2 * (c[1].x + c[1].y), r2 * (c[1].y - c[1].x));     // (1 - i) / sqrt 2
    c[2] = make_float2(c[2].y, -c[2].x);                                  // -i
    c[3] = make_float2(-r2 * (c[3].x - c[3].y), -r2 * (c[3].x + c[3].y)); // -(1 + i) / sqrt 2
    dft_small<4>(b);
    dft_small<4>(c);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        v[2 * m] = b[m];
        v[2 * m + 1] = c[m];
    }
}

__device__ __forceinline__ void dft9(float2* v) {
    // 9 = 3 x 3 (Cooley-Tukey): input 3 n1 + n2, output k1 + 3 k2, twiddles w_9^(n2 k1)
    const float2 w1 = make_float2(0.766044443118978f, 0.6427876096865393f);     // (cos, sin)(2 pi / 9)
    const float2 w2 = make_float2(0.17364817766693041f, 0.984807753012208f);    // 4 pi / 9
    const float2 w4 = make_float2(-0.9396926207859083f, 0.3420201433256689f);   // 8 pi / 9
    float2 y[3][3];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
        y[n2][0] = v[n2];
        y[n2][1] = v[3 + n2];
        y[n2][2] = v[6 + n2];
        dft_small<3>(y[n2]);
    }
    y[1][1] = cmul_conj(y[1][1], w1);
    y[1][2] = cmul_conj(y[1][2], w2);
    y[2][1] = cmul_conj(y[2][1], w2);
    y[2][2] = cmul_conj(y[2][2], w4);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        float2 t[3] = {y[0][k1], y[1][k1], y[2][k1]};
        dft_small<3>(t);
        v[k1] = t[0];
        v[k1 + 3] = t[1];
        v[k1 + 6] = t[2];
    }
}

// In-place forward transform of the permuted row z (360 complex values, z +
// zz when zz is given: the two rows are summed as the first stage loads them).
// One warp; z must not be read by other warps meanwhile.
__device__ __forceinline__ void warp_pfa360(float2* z, const float2* zz, int lane) {
    for (int d = lane; d < 45; d += 32) {           // length 8 along n1: stride 45
        float2 v[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            v[n1] = z[45 * n1 + d];
            if (zz) {
                const float2 u = zz[45 * n1 + d];
                v[n1].x += u.x;
                v[n1].y += u.y;
            }
        }
        dft8(v);
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) z[45 * k1 + d] = v[k1];
    }
    __syncwarp();
    for (int d = lane; d < 40; d += 32) {           // length 9 along n2: stride 5
        const int base = 45 * (d / 5) + d % 5;
        float2 v[9];
#pragma unroll
        for (int n2 = 0; n2 < 9; ++n2) v[n2] = z[base + 5 * n2];
        dft9(v);
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) z[base + 5 * k2] = v[k2];
    }
    __syncwarp();
    for (int d = lane; d < 72; d += 32) {           // length 5 along n3: stride 1
        float2 v[5];
#pragma unroll
        for (int n3 = 0; n3 < 5; ++n3) v[n3] = z[5 * d + n3];
        dft_small<5>(v);
#pragma unroll
        for (int k3 = 0; k3 < 5; ++k3) z[5 * d + k3] = v[k3];
    }
    __syncwarp();
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
