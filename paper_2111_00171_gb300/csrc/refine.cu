// Continuous orientation refinement: the kinematical correlation score of a
// pattern with an orientation, its gradient, and damped Gauss-Newton ascent.
//
//   S(R) = sum_m sum_g a_m b_g exp(-|p_m - (R g)_xy|^2 / (2 rho^2)) / ||b||
//
// R the crystal-to-lab rotation (R = m^T), p_m the peak positions, a_m =
// q_m^gamma I_m^(omega/2) the peak weights of the polar image, b_g =
// |g|^gamma |F_g|^omega D(s_g)^(omega/2) the same weight for the kinematical
// intensity |F_g|^2 D(s_g) of reflection g (D the Gaussian shape factor of
// Eq. 8, s_g the excitation error of R g by Eq. 6 with the beam along -z).
// The paper matches on the grid only; this score turns the orientation into a
// continuous variable (its plan correlation with a Gaussian spot of width rho
// in place of the tent and the predicted weights normalised like a plan slice).
//
// Gradient: for R -> Exp(w) R, d(R g)/dw_j = e_j x (R g), so
// dS/dw = sum_g (R g) x dS/d(R g).  For an axis-angle r about a base rotation
// (R = Exp(r) R0), dS/dr = J(r)^T dS/dw with J the left Jacobian of SO(3).
// Gauss-Newton matrix: for each product of Gaussian factors, the outer
// products of the derivatives of their arguments (positions over rho^2, the
// excitation error over sigma_e^2 = 2 sigma^2 / omega), weighted by the term.
//
// One warp per pattern.  The lanes compute the excitation factor of their
// reflections and ballot the ones that contribute into a list; each lane then
// takes its share of the list (the last, partial round split by peaks) and
// sums over the peaks (in a whole round every lane reads the same peak from
// shared memory); one butterfly reduction per evaluation gives every lane the
// same totals.  Every lane takes the same 3x3 step in FP32 and nine lanes
// compose the rotation in FP64, one element each (kept in shared memory with
// its FP32 copy, which the score reads).  A reflection whose excitation
// factor is below e^-18 of its weight is skipped (its share of S is below
// FP32 resolution).
#include <math_constants.h>

#include "acom_internal.cuh"

namespace acom {

namespace {

constexpr int kRefWarps = 8;                    // patterns per block
constexpr int kRefPeakSmem = 128;               // peaks per pattern kept in shared memory
constexpr float kExcCut = 18.0f;                // skip when s^2 / (2 sigma_e^2) > kExcCut
constexpr int kRefActCap = 512;                 // contributing reflections listed at a time

struct RefArgs {
    const float4* refl;        // [G] (g_x, g_y, g_z, |g|^gamma |F_g|^omega)
    int G;
    const int64_t* row_ptr;
    const float *qx, *qy, *I;
    int64_t nb;
    float gamma_pow, omega;
    float inv_lam;             // 1 / lambda
    float se2;                 // sigma_e^2 = 2 sigma^2 / omega (inf for omega = 0)
    // refinement
    int steps;
    float rho_start, rho_end, damping, max_step;
    int twin;
    // score mode
    const float* r;            // [nb][3] axis-angle about orient, or nullptr
    const float* strain;       // [nb][6] reciprocal-lattice strain (xx xy xz yy yz zz), or nullptr
    float* strain_grad;        // [nb][6] dS/de, or nullptr
    float rho;
    // in / out
    float* orient;             // [nb][9] m (sample to crystal), row major
    const float* orient_alt;   // [nb][9] second start, or nullptr
    float* score;              // [nb] or nullptr
    float* grad;               // [nb][3] or nullptr (score mode)
    float* gn;                 // [nb][6] or nullptr (score mode)
    uint8_t* start_out;        // [nb] winning start (bit 0 twin, bit 1 alt), or nullptr
    unsigned long long* pairs; // (reflection, peak) pairs summed, or nullptr
    int* err;
};

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float peak_weight(float x, float y, float I, float gamma_pow,
                                             float omega) {
    const float q = sqrtf(x * x + y * y);
    const float qg = gamma_pow == 1.0f ? q : (gamma_pow == 0.0f ? 1.0f : powf(q, gamma_pow));
    float iw;
    if (omega == 0.0f) iw = 1.0f;                       // I^0 = 1
    else if (!(I > 0.0f)) iw = 0.0f;                    // negative intensities weigh 0
    else iw = omega == 1.0f ? sqrtf(I) : powf(I, 0.5f * omega);
    return qg * iw;
}

struct Acc {
    float C, nb2;
    float g1[3], g2[3];
    float h[6];          // xx, xy, xz, yy, yz, zz
    float e1[6], e2[6];  // strain: sym(R^T dC/dv g^T), sym(b R^T db/dv g^T) (xx xy xz yy yz zz)
};

// g + e g for the symmetric strain e (xx xy xz yy yz zz)
__device__ __forceinline__ void strained(const float e[6], float& x, float& y, float& z) {
    const float x0 = x, y0 = y, z0 = z;
    x = x0 + e[0] * x0 + e[1] * y0 + e[2] * z0;
    y = y0 + e[1] * x0 + e[3] * y0 + e[4] * z0;
    z = z0 + e[2] * x0 + e[4] * y0 + e[5] * z0;
}

// Adds reflection g's terms over peaks m0 .. m1 - 1 to acc.  Every term is
// linear in the three peak sums except ||b||^2 and the b db/dv parts, which
// do not depend on the peaks: with `once` they are added too (a reflection
// whose peaks are split between lanes adds them in one lane only).  STRAIN:
// the reflection sits at R (I + e) g (reading: lattice strain moves the spots,
// the amplitudes keep their unstrained values), and dS/de is accumulated.
template <bool STRAIN>
__device__ __forceinline__ void add_reflection(const RefArgs& a, const float R[9], const float e[6],
                                               float4 g, float inv_r2, float l2_half_inv_r2,
                                               bool exc, float inv_se2, int64_t p0, int m0,
                                               int m1, bool once, const float* px,
                                               const float* py, const float* pa, Acc& acc) {
    float gx = g.x, gy = g.y, gz = g.z;
    if (STRAIN) strained(e, gx, gy, gz);
    const float vx = R[0] * gx + R[1] * gy + R[2] * gz;
    const float vy = R[3] * gx + R[4] * gy + R[5] * gz;
    const float vz = R[6] * gx + R[7] * gy + R[8] * gz;
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float kz = vz - a.inv_lam;
    const float nkv2 = vx * vx + vy * vy + kz * kz;
    const float nkv = sqrtf(nkv2);
    const float s = -(v2 - 2.0f * vz * a.inv_lam) / (2.0f * nkv);
    const float b = exc ? g.w * expf(-0.5f * s * s * inv_se2) : g.w;
    // ds/dv = -(k + v) (|k + v| + s) / |k + v|^2
    const float f = -(nkv + s) / nkv2;
    const float dsx = f * vx, dsy = f * vy, dsz = f * kz;
    float sE = 0.f, sEx = 0.f, sEy = 0.f;
    const int Ms = m1 < kRefPeakSmem ? m1 : kRefPeakSmem;
#pragma unroll 4
    for (int m = m0; m < Ms; ++m) {              // a whole round: every lane reads the same peak
        const float dx = px[m] - vx, dy = py[m] - vy;
        const float e = pa[m] * exp2f(-(dx * dx + dy * dy) * l2_half_inv_r2);
        sE += e;
        sEx = fmaf(e, dx, sEx);
        sEy = fmaf(e, dy, sEy);
    }
    for (int m = m0 > kRefPeakSmem ? m0 : kRefPeakSmem; m < m1; ++m) {
        const float x = a.qx[p0 + m], y = a.qy[p0 + m];
        const float w = peak_weight(x, y, a.I[p0 + m], a.gamma_pow, a.omega);
        const float dx = x - vx, dy = y - vy;
        const float e = w * exp2f(-(dx * dx + dy * dy) * l2_half_inv_r2);
        sE += e;
        sEx = fmaf(e, dx, sEx);
        sEy = fmaf(e, dy, sEy);
    }
    const float W = b * sE;
    acc.C += W;
    if (once) acc.nb2 = fmaf(b, b, acc.nb2);
    const float c = exc ? -s * inv_se2 * b : 0.0f;             // db/ds
    const float dbx = c * dsx, dby = c * dsy, dbz = c * dsz;    // db/dv
    const float dcx = b * sEx * inv_r2 + sE * dbx;
    const float dcy = b * sEy * inv_r2 + sE * dby;
    const float dcz = sE * dbz;
    if (STRAIN) {
        // dv/de_kl = R (basis_kl) g with the unstrained g: with u = R^T dC/dv,
        // dC/de_kl = u_k g_l + u_l g_k (k != l), u_k g_k (k = l); the same for
        // the b db/dv part of the quotient rule
        const float u1x = R[0] * dcx + R[3] * dcy + R[6] * dcz;
        const float u1y = R[1] * dcx + R[4] * dcy + R[7] * dcz;
        const float u1z = R[2] * dcx + R[5] * dcy + R[8] * dcz;
        const float bo = once ? b : 0.0f;
        const float u2x = bo * (R[0] * dbx + R[3] * dby + R[6] * dbz);
        const float u2y = bo * (R[1] * dbx + R[4] * dby + R[7] * dbz);
        const float u2z = bo * (R[2] * dbx + R[5] * dby + R[8] * dbz);
        acc.e1[0] += u1x * g.x;
        acc.e1[1] += u1x * g.y + u1y * g.x;
        acc.e1[2] += u1x * g.z + u1z * g.x;
        acc.e1[3] += u1y * g.y;
        acc.e1[4] += u1y * g.z + u1z * g.y;
        acc.e1[5] += u1z * g.z;
        acc.e2[0] += u2x * g.x;
        acc.e2[1] += u2x * g.y + u2y * g.x;
        acc.e2[2] += u2x * g.z + u2z * g.x;
        acc.e2[3] += u2y * g.y;
        acc.e2[4] += u2y * g.z + u2z * g.y;
        acc.e2[5] += u2z * g.z;
    }
    acc.g1[0] += vy * dcz - vz * dcy;
    acc.g1[1] += vz * dcx - vx * dcz;
    acc.g1[2] += vx * dcy - vy * dcx;
    if (once) {
        acc.g2[0] += b * (vy * dbz - vz * dby);
        acc.g2[1] += b * (vz * dbx - vx * dbz);
        acc.g2[2] += b * (vx * dby - vy * dbx);
    }
    // position part: jx = (0, vz, -vy), jy = (-vz, 0, vx)
    const float wp = W * inv_r2;
    acc.h[0] += wp * (vz * vz);
    acc.h[2] -= wp * (vz * vx);
    acc.h[3] += wp * (vz * vz);
    acc.h[4] -= wp * (vz * vy);
    acc.h[5] += wp * (vx * vx + vy * vy);
    if (exc) {                                   // excitation part: js = v x ds/dv
        const float jsx = vy * dsz - vz * dsy, jsy = vz * dsx - vx * dsz,
                    jsz = vx * dsy - vy * dsx;
        const float we = W * inv_se2;
        acc.h[0] += we * jsx * jsx;
        acc.h[1] += we * jsx * jsy;
        acc.h[2] += we * jsx * jsz;
        acc.h[3] += we * jsy * jsy;
        acc.h[4] += we * jsy * jsz;
        acc.h[5] += we * jsz * jsz;
    }
}

// S, dS/dw and the Gauss-Newton matrix of the warp's pattern at rotation R
// (identical in every lane).  The reflections that contribute are listed in
// the warp's act[] buffer kRefActCap at a time; the whole rounds of the list
// give lane l entries l, l + 32, ... with all their peaks, and the rem < 32
// entries left over are split into 32 / rem chunks of peaks each, one chunk
// per lane, so that the last round does not leave most lanes idle; the
// per-lane sums are then added by a butterfly.  Peaks: the first kRefPeakSmem
// in (px, py, pa), the rest read from global memory.
template <bool STRAIN>
__device__ void score_at(const RefArgs& a, const float R[9], const float e[6], float rho,
                         int64_t p0, int M, const float* px, const float* py, const float* pa,
                         int* act, float& S, float grad[3], float H[6], float de[6]) {
    const int lane = threadIdx.x & 31;
    const float inv_r2 = 1.0f / (rho * rho);
    // exp(-x / (2 rho^2)) = 2^(-x log2(e) / (2 rho^2)): the spot Gaussian as one
    // base-2 exponential of a pre-scaled argument
    const float l2_half_inv_r2 = 0.5f * inv_r2 * 1.4426950408889634f;
    const bool exc = a.omega > 0.0f;
    const float inv_se2 = exc ? 1.0f / a.se2 : 0.0f;
    Acc acc{};
    for (int c0 = 0; c0 < a.G; c0 += kRefActCap) {
        // list the contributing reflections of [c0, c0 + kRefActCap)
        int n = 0;
        const int c1 = c0 + kRefActCap < a.G ? c0 + kRefActCap : a.G;
        for (int g0 = c0; g0 < c1; g0 += 32) {
            const int gi = g0 + lane;
            bool active = false;
            if (gi < c1) {
                const float4 g = __ldg(a.refl + gi);
                float gx = g.x, gy = g.y, gz = g.z;
                if (STRAIN) strained(e, gx, gy, gz);
                const float vx = R[0] * gx + R[1] * gy + R[2] * gz;
                const float vy = R[3] * gx + R[4] * gy + R[5] * gz;
                const float vz = R[6] * gx + R[7] * gy + R[8] * gz;
                const float v2 = vx * vx + vy * vy + vz * vz;
                const float kz = vz - a.inv_lam;
                const float nkv = sqrtf(vx * vx + vy * vy + kz * kz);
                const float s = -(v2 - 2.0f * vz * a.inv_lam) / (2.0f * nkv);
                active = g.w > 0.0f && (!exc || 0.5f * s * s * inv_se2 <= kExcCut);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, active);
            if (active) act[n + __popc(mask & ((1u << lane) - 1u))] = gi;
            n += __popc(mask);
        }
        __syncwarp();
        if (a.pairs && lane == 0) atomicAdd(a.pairs, (unsigned long long)n * (unsigned long long)M);
        const int whole = n & ~31;
        for (int j = lane; j < whole; j += 32)
            add_reflection<STRAIN>(a, R, e, __ldg(a.refl + act[j]), inv_r2, l2_half_inv_r2, exc,
                                   inv_se2, p0, 0, M, true, px, py, pa, acc);
        const int rem = n - whole;
        if (rem > 0) {
            const int cps = 32 / rem;                // chunks per left-over reflection
            if (lane < rem * cps) {
                const int j = whole + lane / cps, c = lane - (lane / cps) * cps;
                add_reflection<STRAIN>(a, R, e, __ldg(a.refl + act[j]), inv_r2, l2_half_inv_r2,
                                       exc, inv_se2, p0, (M * c) / cps, (M * (c + 1)) / cps,
                                       c == 0, px, py, pa, acc);
            }
        }
        __syncwarp();
    }
    acc.C = warp_sum(acc.C);
    acc.nb2 = warp_sum(acc.nb2);
    for (int i = 0; i < 3; ++i) {
        acc.g1[i] = warp_sum(acc.g1[i]);
        acc.g2[i] = warp_sum(acc.g2[i]);
    }
    for (int i = 0; i < 6; ++i) acc.h[i] = warp_sum(acc.h[i]);
    if (STRAIN)
        for (int i = 0; i < 6; ++i) {
            acc.e1[i] = warp_sum(acc.e1[i]);
            acc.e2[i] = warp_sum(acc.e2[i]);
        }
    if (!(acc.nb2 > 0.0f)) {
        S = 0.0f;
        grad[0] = grad[1] = grad[2] = 0.0f;
        for (int i = 0; i < 6; ++i) H[i] = 0.0f;
        if (STRAIN)
            for (int i = 0; i < 6; ++i) de[i] = 0.0f;
        return;
    }
    const float nb = sqrtf(acc.nb2);
    const float inv_nb = 1.0f / nb;
    S = acc.C * inv_nb;
    const float q = acc.C * inv_nb * inv_nb * inv_nb;
    for (int i = 0; i < 3; ++i) grad[i] = acc.g1[i] * inv_nb - q * acc.g2[i];
    for (int i = 0; i < 6; ++i) H[i] = acc.h[i] * inv_nb;
    if (STRAIN)
        for (int i = 0; i < 6; ++i) de[i] = acc.e1[i] * inv_nb - q * acc.e2[i];
}

// Rotation by |w| about w (Rodrigues), FP64, row major.  Below 0.05 rad the
// factors sin(t)/t and (1 - cos t)/t^2 come from their Taylor series to t^4
// (remainder under 1e-11 relative there, near 1e-14 at 1 degree), which
// avoids FP64 transcendentals in the per-step update.
__device__ void exp_so3(const double w[3], double E[9]) {
    const double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double t = sqrt(t2);
    double A, B;
    if (t < 0.05) {
        A = 1.0 - t2 * (1.0 / 6.0 - t2 * (1.0 / 120.0));
        B = 0.5 - t2 * (1.0 / 24.0 - t2 * (1.0 / 720.0));
    } else {
        A = sin(t) / t;
        B = (1.0 - cos(t)) / (t * t);
    }
    const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double k2 = 0;
            for (int l = 0; l < 3; ++l) k2 += K[3 * i + l] * K[3 * l + j];
            E[3 * i + j] = (i == j ? 1.0 : 0.0) + A * K[3 * i + j] + B * k2;
        }
}

// The same rotation in FP32 for the per-step update: sin(t)/t and
// (1 - cos t)/t^2 = 2 sin^2(t/2) / t^2 (no cancellation), by their Taylor
// series to t^4 below 0.05 rad.  The step's rotation is composed onto the
// FP64 orientation, so its FP32 rounding (~1e-7 per step) does not accumulate
// into the FP64 result beyond the steps' count.
__device__ void exp_so3f(const float w[3], float E[9]) {
    const float t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const float t = sqrtf(t2);
    float A, B;
    if (t < 0.05f) {
        A = 1.0f - t2 * (1.0f / 6.0f - t2 * (1.0f / 120.0f));
        B = 0.5f - t2 * (1.0f / 24.0f - t2 * (1.0f / 720.0f));
    } else {
        const float sh = sinf(0.5f * t);
        A = sinf(t) / t;
        B = 2.0f * sh * sh / t2;
    }
    const float K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float k2 = 0;
            for (int l = 0; l < 3; ++l) k2 += K[3 * i + l] * K[3 * l + j];
            E[3 * i + j] = (i == j ? 1.0f : 0.0f) + A * K[3 * i + j] + B * k2;
        }
}

// w = (H + damping diag(H) + 1e-12 tr(H) I)^-1 g, at most max_step in norm.
__device__ void lm_step(const float H[6], const float g[3], float damping, float max_step,
                        float w[3]) {
    const float tr = H[0] + H[3] + H[5];
    w[0] = w[1] = w[2] = 0.0f;
    if (!(tr > 0.0f)) return;
    const float e = 1e-12f * tr;
    const float a = H[0] * (1.0f + damping) + e, b = H[1], c = H[2];
    const float d = H[3] * (1.0f + damping) + e, f = H[4];
    const float k = H[5] * (1.0f + damping) + e;
    // adjugate of the symmetric matrix [[a b c] [b d f] [c f k]]
    const float A00 = d * k - f * f, A01 = c * f - b * k, A02 = b * f - c * d;
    const float A11 = a * k - c * c, A12 = b * c - a * f, A22 = a * d - b * b;
    const float det = a * A00 + b * A01 + c * A02;
    if (!(fabsf(det) > 0.0f)) return;
    const float id = 1.0f / det;
    w[0] = (A00 * g[0] + A01 * g[1] + A02 * g[2]) * id;
    w[1] = (A01 * g[0] + A11 * g[1] + A12 * g[2]) * id;
    w[2] = (A02 * g[0] + A12 * g[1] + A22 * g[2]) * id;
    const float n = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (n > max_step) {
        const float sc = max_step / n;
        w[0] *= sc;
        w[1] *= sc;
        w[2] *= sc;
    }
}

__device__ __forceinline__ void load9(const float* Rf, float R[9]) {
    __syncwarp();
    for (int i = 0; i < 9; ++i) R[i] = Rf[i];
}

// One refinement run from Rd (FP64 in the warp's shared memory, with its FP32
// copy Rf).  Every lane holds the same score, gradient and matrix, so every
// lane takes the same step; lanes 0..8 compose one element of Exp(w) Rd each
// in FP64 (FP64 instructions are scarce on this GPU: nine lanes issue three
// multiply-adds where one lane issued a hundred).
__device__ float refine_run(const RefArgs& a, double* Rd, float* Rf, int64_t p0, int M,
                            const float* px, const float* py, const float* pa, int* act) {
    const int lane = threadIdx.x & 31;
    float R[9], S, g[3], H[6];
    for (int t = 0; t < a.steps; ++t) {
        const float rho = a.steps > 1
                              ? a.rho_start * powf(a.rho_end / a.rho_start,
                                                   (float)t / (float)(a.steps - 1))
                              : a.rho_end;
        load9(Rf, R);
        score_at<false>(a, R, nullptr, rho, p0, M, px, py, pa, act, S, g, H, nullptr);
        float w[3], E[9];
        lm_step(H, g, a.damping, a.max_step, w);
        exp_so3f(w, E);
        double v = 0.0;
        if (lane < 9) {
            const int i = lane / 3, j = lane - 3 * (lane / 3);
            v = (double)E[3 * i] * Rd[j] + (double)E[3 * i + 1] * Rd[3 + j] +
                (double)E[3 * i + 2] * Rd[6 + j];
        }
        __syncwarp();
        if (lane < 9) {
            Rd[lane] = v;
            Rf[lane] = (float)v;
        }
    }
    load9(Rf, R);
    score_at<false>(a, R, nullptr, a.rho_end, p0, M, px, py, pa, act, S, g, H, nullptr);
    return S;
}

// Peaks of pattern b into the warp's shared arrays; returns the count, or -1
// (and sets the error word) for an invalid row.
__device__ int load_peaks(const RefArgs& a, int64_t b, int64_t& p0, float* px, float* py,
                          float* pa) {
    const int lane = threadIdx.x & 31;
    p0 = a.row_ptr[b];
    const int64_t p1 = a.row_ptr[b + 1];
    const int64_t n = p1 - p0;
    if (n < 0 || n > kMaxPeaks) {
        if (lane == 0) atomicOr(a.err, n < 0 ? kErrRowPtr : kErrTooManyPeaks);
        return -1;
    }
    const int M = (int)n;
    bool bad = false;
    for (int m = lane; m < M; m += 32) {
        const float x = a.qx[p0 + m], y = a.qy[p0 + m], I = a.I[p0 + m];
        bad |= !isfinite(x) || !isfinite(y) || !isfinite(I);
        if (m < kRefPeakSmem) {
            px[m] = x;
            py[m] = y;
            pa[m] = peak_weight(x, y, I, a.gamma_pow, a.omega);
        }
    }
    if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) atomicOr(a.err, kErrNonFinite);
        return -1;
    }
    __syncwarp();
    return M;
}

__global__ void __launch_bounds__(kRefWarps * 32, 3) k_refine(RefArgs a) {
    __shared__ float s_px[kRefWarps][kRefPeakSmem], s_py[kRefWarps][kRefPeakSmem],
        s_pa[kRefWarps][kRefPeakSmem];
    __shared__ int s_act[kRefWarps][kRefActCap];
    __shared__ double s_R[kRefWarps][2][9];
    __shared__ float s_Rf[kRefWarps][9];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* px = s_px[warp];
    float* py = s_py[warp];
    float* pa = s_pa[warp];
    int* act = s_act[warp];
    double* Rc = s_R[warp][0];        // the run in progress
    double* Rb = s_R[warp][1];        // the best refined rotation so far
    for (int64_t b = (int64_t)blockIdx.x * kRefWarps + warp; b < a.nb;
         b += (int64_t)gridDim.x * kRefWarps) {
        int64_t p0;
        __syncwarp();
        const int M = load_peaks(a, b, p0, px, py, pa);
        if (M < 0) continue;
        // starts: orient, its twin, orient_alt, its twin (in that order; a
        // later start wins only with a strictly higher score)
        const float* src0 = a.orient + 9 * b;
        const float* src1 = a.orient_alt ? a.orient_alt + 9 * b : nullptr;
        float best = -CUDART_INF_F;
        int best_start = 0;
        for (int st = 0; st < 4; ++st) {
            const float* src = (st & 2) ? src1 : src0;
            if (!src || ((st & 1) && !a.twin)) continue;
            __syncwarp();
            if (lane < 9) {
                const int i = lane / 3, j = lane - 3 * (lane / 3);
                const float v = src[3 * j + i];                    // R = m^T
                const float r = ((st & 1) && i < 2) ? -v : v;      // (m Rz(pi))^T
                Rc[lane] = (double)r;
                s_Rf[warp][lane] = r;
            }
            const float S = refine_run(a, Rc, s_Rf[warp], p0, M, px, py, pa, act);
            __syncwarp();
            if (S > best || st == 0) {
                best = S;
                best_start = st;
                if (lane == 0)
                    for (int i = 0; i < 9; ++i) Rb[i] = Rc[i];
            }
        }
        __syncwarp();
        if (lane == 0) {
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) a.orient[9 * b + 3 * i + j] = (float)Rb[3 * j + i];
            if (a.score) a.score[b] = best;
            if (a.start_out) a.start_out[b] = (uint8_t)best_start;
        }
    }
}

// Score, gradient dS/dr and Gauss-Newton matrix at R = Exp(r) m^T.
__global__ void __launch_bounds__(kRefWarps * 32) k_kin_score(RefArgs a) {
    __shared__ float s_px[kRefWarps][kRefPeakSmem], s_py[kRefWarps][kRefPeakSmem],
        s_pa[kRefWarps][kRefPeakSmem];
    __shared__ int s_act[kRefWarps][kRefActCap];
    __shared__ double s_R[kRefWarps][9];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* px = s_px[warp];
    float* py = s_py[warp];
    float* pa = s_pa[warp];
    int* act = s_act[warp];
    double* Rd = s_R[warp];
    for (int64_t b = (int64_t)blockIdx.x * kRefWarps + warp; b < a.nb;
         b += (int64_t)gridDim.x * kRefWarps) {
        int64_t p0;
        __syncwarp();
        const int M = load_peaks(a, b, p0, px, py, pa);
        if (M < 0) continue;
        double r[3] = {0, 0, 0};
        if (lane == 0) {
            double M0[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) M0[3 * i + j] = (double)a.orient[9 * b + 3 * j + i];
            if (a.r)
                for (int i = 0; i < 3; ++i) r[i] = a.r[3 * b + i];
            double E[9];
            exp_so3(r, E);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Rd[3 * i + j] = E[3 * i] * M0[j] + E[3 * i + 1] * M0[3 + j] +
                                    E[3 * i + 2] * M0[6 + j];
        }
        float R[9], S, g[3], H[6], e[6], de[6];
        __syncwarp();
        for (int i = 0; i < 9; ++i) R[i] = (float)Rd[i];
        for (int i = 0; i < 6; ++i) e[i] = a.strain ? a.strain[6 * b + i] : 0.0f;
        score_at<true>(a, R, e, a.rho, p0, M, px, py, pa, act, S, g, H, de);
        if (lane == 0) {
            if (a.score) a.score[b] = S;
            if (a.grad) {
                // dS/dr = J(r)^T dS/dw, J = I + (1 - cos t)/t^2 K + (t - sin t)/t^3 K^2
                const double t = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                double A, B;
                if (t < 1e-6) {
                    A = 0.5;
                    B = 1.0 / 6.0;
                } else {
                    A = (1.0 - cos(t)) / (t * t);
                    B = (t - sin(t)) / (t * t * t);
                }
                const double K[9] = {0, -r[2], r[1], r[2], 0, -r[0], -r[1], r[0], 0};
                for (int j = 0; j < 3; ++j) {
                    double acc = 0;
                    for (int i = 0; i < 3; ++i) {
                        double k2 = 0;
                        for (int l = 0; l < 3; ++l) k2 += K[3 * i + l] * K[3 * l + j];
                        const double Jij = (i == j ? 1.0 : 0.0) + A * K[3 * i + j] + B * k2;
                        acc += Jij * (double)g[i];
                    }
                    a.grad[3 * b + j] = (float)acc;
                }
            }
            if (a.gn)
                for (int i = 0; i < 6; ++i) a.gn[6 * b + i] = H[i];
            if (a.strain_grad)
                for (int i = 0; i < 6; ++i) a.strain_grad[6 * b + i] = de[i];
        }
    }
}

// FP32 table (g, |g|^gamma |F_g|^omega) from the plan's FP64 reflections
// (refl_amp holds |F_g|^omega).
__global__ void k_refl_table(const double* __restrict__ g, const double* __restrict__ amp, int G,
                             double gamma_pow, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    const double x = g[3 * i], y = g[3 * i + 1], z = g[3 * i + 2];
    const double n = sqrt(x * x + y * y + z * z);
    out[i] = make_float4((float)x, (float)y, (float)z, (float)(pow(n, gamma_pow) * amp[i]));
}

}  // namespace

acom_status refine_table(acom_plan_s* p, cudaStream_t st) {
    if (p->refl_tab) return ACOM_OK;
    if (p->n_phases != 1 || !p->refl_g || !p->refl_amp || p->G <= 0)
        return set_error(ACOM_ERR_UNSUPPORTED,
                         "refinement needs a single-phase plan with its reflections");
    cudaError_t e = pool_alloc(reinterpret_cast<void**>(&p->refl_tab), sizeof(float4) * p->G, st);
    if (e != cudaSuccess) return cuda_error(e, "refinement table allocation");
    p->bytes += sizeof(float4) * p->G;
    e = pool_alloc(reinterpret_cast<void**>(&p->refine_pairs), sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_error(e, "refinement counter allocation");
    prof_begin(kKMisc, st);
    k_refl_table<<<(p->G + 255) / 256, 256, 0, st>>>(p->refl_g, p->refl_amp, p->G, p->gamma_pow,
                                                      p->refl_tab);
    prof_end(kKMisc, st);
    return ACOM_OK;
}

static RefArgs ref_args(const acom_plan_s* p, const acom_peaks_csr* pk) {
    RefArgs a{};
    a.refl = p->refl_tab;
    a.G = p->G;
    a.row_ptr = pk->row_ptr;
    a.qx = pk->qx;
    a.qy = pk->qy;
    a.I = pk->I;
    a.nb = pk->n_patterns;
    a.gamma_pow = (float)p->gamma_pow;
    a.omega = (float)p->omega;
    a.inv_lam = (float)(1.0 / p->lambda);
    a.se2 = p->omega > 0 ? (float)(2.0 * p->sigma_exc * p->sigma_exc / p->omega) : HUGE_VALF;
    a.err = p->err;
    return a;
}

static int ref_grid(int64_t nb) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (nb + kRefWarps - 1) / kRefWarps;
    const int64_t cap = (int64_t)nsm * 8;
    return (int)(need < cap ? need : cap);
}

void launch_refine_orient(const acom_plan_s* p, const acom_peaks_csr* pk, int steps,
                          float rho_start, float rho_end, float damping, float max_step, int twin,
                          float* orient, const float* orient_alt, float* score, uint8_t* start_out,
                          cudaStream_t st) {
    RefArgs a = ref_args(p, pk);
    a.steps = steps;
    a.rho_start = rho_start;
    a.rho_end = rho_end;
    a.damping = damping;
    a.max_step = max_step;
    a.twin = twin;
    a.orient = orient;
    a.orient_alt = orient_alt;
    a.score = score;
    a.start_out = start_out;
    a.pairs = p->refine_pairs;
    const int grid = ref_grid(pk->n_patterns);
    if (grid <= 0) return;
    prof_begin(kKRefineOrient, st);
    k_refine<<<grid, kRefWarps * 32, 0, st>>>(a);
    prof_end(kKRefineOrient, st);
}

void launch_kin_score(const acom_plan_s* p, const acom_peaks_csr* pk, const float* orient,
                      const float* r, const float* strain, float rho, float* score, float* grad,
                      float* gn, float* strain_grad, cudaStream_t st) {
    RefArgs a = ref_args(p, pk);
    a.orient = const_cast<float*>(orient);
    a.r = r;
    a.strain = strain;
    a.strain_grad = strain_grad;
    a.rho = rho;
    a.score = score;
    a.grad = grad;
    a.gn = gn;
    const int grid = ref_grid(pk->n_patterns);
    if (grid <= 0) return;
    prof_begin(kKRefineOrient, st);
    k_kin_score<<<grid, kRefWarps * 32, 0, st>>>(a);
    prof_end(kKRefineOrient, st);
}

}  // namespace acom
