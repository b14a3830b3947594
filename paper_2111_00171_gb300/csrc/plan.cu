// Orientation-plan builder (section "Generation of an Orientation Plan").
//
//   k_reflections   every lattice point 0 < |g| < q_max (Eq. 2) and its
//                   structure factor F_hkl = sum_n f_n(|g|) exp(-2 pi i hkl.p_n)
//                   (Eq. 3), in FP64, compacted in lexicographic (h, k, l)
//                   order; reflections with |F| < 1e-9 max|F| are dropped
//                   (V_g of Eq. 4 is zero there).
//   raster (raster.cu, PlanLoader)  P0 per zone axis and its Fourier
//                   transform along phi3, plus ||P0||^2.
//   k_scale_rows    P = A P0, A = 1/||P0||_2.
//
// The zone-axis grid, the rotations R = Rz(phi1) Rx(theta2) (first two factors
// of Eq. 10) and the grid-neighbour lists are small host computations in FP64.
#include <math_constants.h>

#include <algorithm>
#include <cmath>

#include "acom_internal.cuh"

namespace acom {

struct ReflParams {
    double rb[9];       // reciprocal basis rows a*, b*, c*
    int n0, n1, n2;     // index box |h| <= n0, |k| <= n1, |l| <= n2
    double q_max;
    double omega;
    int n_atoms;
};

constexpr int kReflThreads = 1024;

// Single CTA: the candidate box is at most a few hundred thousand points.
__global__ void __launch_bounds__(kReflThreads)
k_reflections(ReflParams prm, const double* __restrict__ atoms,  // [n][5]: px py pz A B
              double* tmp_g, double* tmp_F, double* out_g, double* out_amp, int* out_count) {
    __shared__ int s_warp[33];
    __shared__ double s_max[32];
    const int64_t n1w = 2 * prm.n1 + 1, n2w = 2 * prm.n2 + 1;
    const int64_t total = (int64_t)(2 * prm.n0 + 1) * n1w * n2w;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int count = 0;
    double fmx = 0.0;
    for (int64_t base = 0; base < total; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        bool keep = false;
        double gx = 0, gy = 0, gz = 0, absF = 0;
        if (idx < total) {
            int h = (int)(idx / (n1w * n2w)) - prm.n0;
            int k = (int)((idx / n2w) % n1w) - prm.n1;
            int l = (int)(idx % n2w) - prm.n2;
            gx = h * prm.rb[0] + k * prm.rb[3] + l * prm.rb[6];
            gy = h * prm.rb[1] + k * prm.rb[4] + l * prm.rb[7];
            gz = h * prm.rb[2] + k * prm.rb[5] + l * prm.rb[8];
            double q = sqrt(gx * gx + gy * gy + gz * gz);
            keep = (q > 0.0) && (q < prm.q_max);
            if (keep) {
                double re = 0.0, im = 0.0;
                for (int n = 0; n < prm.n_atoms; ++n) {
                    const double* a = atoms + 5 * n;
                    double fn = a[3] * exp(-a[4] * q * q);
                    double ph = h * a[0] + k * a[1] + l * a[2];
                    double sn, cs;
                    sincospi(2.0 * ph, &sn, &cs);     // exp(-2 pi i ph)
                    re += fn * cs;
                    im -= fn * sn;
                }
                absF = sqrt(re * re + im * im);
                fmx = fmx > absF ? fmx : absF;
            }
        }
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                int c = s_warp[w];
                s_warp[w] = acc;
                acc += c;
            }
            s_warp[32] = acc;
        }
        __syncthreads();
        if (keep) {
            int pos = count + s_warp[warp] + __popc(m & ((1u << lane) - 1u));
            tmp_g[3 * pos] = gx;
            tmp_g[3 * pos + 1] = gy;
            tmp_g[3 * pos + 2] = gz;
            tmp_F[pos] = absF;
        }
        count += s_warp[32];
        __syncthreads();
    }
    // block max of |F|
    for (int o = 16; o > 0; o >>= 1) fmx = fmax(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
    if (lane == 0) s_max[warp] = fmx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = mm > s_max[w] ? mm : s_max[w];
        s_max[0] = mm;
    }
    __syncthreads();
    const double thr = 1e-9 * s_max[0];
    // second pass: drop extinct reflections, keep order
    int out = 0;
    for (int base = 0; base < count; base += blockDim.x) {
        int i = base + threadIdx.x;
        bool keep = (i < count) && (tmp_F[i] >= thr);
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                int c = s_warp[w];
                s_warp[w] = acc;
                acc += c;
            }
            s_warp[32] = acc;
        }
        __syncthreads();
        if (keep) {
            int pos = out + s_warp[warp] + __popc(m & ((1u << lane) - 1u));
            out_g[3 * pos] = tmp_g[3 * i];
            out_g[3 * pos + 1] = tmp_g[3 * i + 1];
            out_g[3 * pos + 2] = tmp_g[3 * i + 2];
            out_amp[pos] = pow(tmp_F[i], prm.omega);
        }
        out += s_warp[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_count = out;
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

acom_status build_plan_device(acom_plan_s* p, const acom_crystal* cr, cudaStream_t st) {
    // Eq. 1: reciprocal basis without 2 pi
    const double* a = cr->lattice[0];
    const double* b = cr->lattice[1];
    const double* c = cr->lattice[2];
    double bxc[3], cxa[3], axb[3];
    cross3(b, c, bxc);
    cross3(c, a, cxa);
    cross3(a, b, axb);
    const double V = a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2];
    if (!(std::fabs(V) > 1e-12)) return set_error(ACOM_ERR_INVALID_ARG, "degenerate lattice");
    ReflParams prm{};
    for (int i = 0; i < 3; ++i) {
        prm.rb[i] = bxc[i] / V;
        prm.rb[3 + i] = cxa[i] / V;
        prm.rb[6 + i] = axb[i] / V;
    }
    // |h| = |g . a| <= q_max |a|: the box holds every point of the sphere
    auto nrm = [](const double* v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); };
    prm.n0 = (int)std::floor(p->q_max * nrm(a));
    prm.n1 = (int)std::floor(p->q_max * nrm(b));
    prm.n2 = (int)std::floor(p->q_max * nrm(c));
    const int64_t cand = (int64_t)(2 * prm.n0 + 1) * (2 * prm.n1 + 1) * (2 * prm.n2 + 1);
    if (cand > (int64_t)4 << 20)
        return set_error(ACOM_ERR_UNSUPPORTED, "q_max * |a_i| too large (index box > 4M points)");
    prm.q_max = p->q_max;
    prm.omega = p->omega;
    prm.n_atoms = cr->n_atoms;

    std::vector<double> atoms(5 * cr->n_atoms);
    for (int n = 0; n < cr->n_atoms; ++n) {
        for (int d = 0; d < 3; ++d) atoms[5 * n + d] = cr->frac_pos[3 * n + d];
        atoms[5 * n + 3] = cr->ff_A[n];
        atoms[5 * n + 4] = cr->ff_B[n];
    }
    double *d_atoms = nullptr, *d_tmp_g = nullptr, *d_tmp_F = nullptr, *d_g = nullptr,
           *d_amp = nullptr;
    int* d_cnt = nullptr;
    cudaError_t e;
#define ACOM_TRY(x)                                        \
    do {                                                   \
        e = (x);                                           \
        if (e != cudaSuccess) goto fail;                   \
    } while (0)
    {
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_atoms), sizeof(double) * atoms.size(), st));
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_tmp_g), sizeof(double) * 3 * cand, st));
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_tmp_F), sizeof(double) * cand, st));
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_g), sizeof(double) * 3 * cand, st));
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_amp), sizeof(double) * cand, st));
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_cnt), sizeof(int), st));
        ACOM_TRY(cudaMemcpyAsync(d_atoms, atoms.data(), sizeof(double) * atoms.size(),
                                 cudaMemcpyHostToDevice, st));
        prof_begin(kKReflections, st);
        k_reflections<<<1, kReflThreads, 0, st>>>(prm, d_atoms, d_tmp_g, d_tmp_F, d_g, d_amp,
                                                  d_cnt);
        prof_end(kKReflections, st);
        ACOM_TRY(cudaGetLastError());
        int G = 0;
        ACOM_TRY(cudaMemcpyAsync(&G, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        ACOM_TRY(cudaStreamSynchronize(st));
        p->G = G;
        p->refl_g = d_g;
        p->refl_amp = d_amp;
        p->bytes += sizeof(double) * 4 * cand;
        d_g = d_amp = nullptr;
        pool_free(d_atoms, st);
        pool_free(d_tmp_g, st);
        pool_free(d_tmp_F, st);
        pool_free(d_cnt, st);
        d_atoms = d_tmp_g = d_tmp_F = nullptr;
        d_cnt = nullptr;

        // P0 -> FFT along phi3 -> scale by A
        float* d_sumsq = nullptr;
        ACOM_TRY(pool_alloc(reinterpret_cast<void**>(&d_sumsq), sizeof(float) * p->Zp, st));
        ACOM_TRY(cudaMemsetAsync(d_sumsq, 0, sizeof(float) * p->Zp, st));
        RasterGeom geo{p->S, p->Spad, p->N, p->F, (float)p->dq, (float)p->delta,
                       (float)p->gamma_pow, 1};
        PlanSource src{p->refl_g, p->refl_amp, p->frames, p->G, p->lambda};
        RasterOut ro;
        ro.re = p->Pr;
        ro.im = p->Pi;
        ro.sre = p->Psr;
        ro.sim = p->Psi;
        ro.sumsq = d_sumsq;
        launch_raster_plan(geo, src, p->Z, ro, p->err, st);
        ACOM_TRY(cudaGetLastError());
        launch_scale_rows(p->Pr, p->Pi, d_sumsq, p->Z, p->F * p->Spad, st);
        launch_scale_rows(p->Psr, p->Psi, d_sumsq, p->Z, shell_row_stride(p->F) * p->Spad, st);
        ACOM_TRY(cudaGetLastError());
        int herr = 0;
        ACOM_TRY(cudaMemcpyAsync(&herr, p->err, sizeof(int), cudaMemcpyDeviceToHost, st));
        ACOM_TRY(cudaStreamSynchronize(st));
        prof_resolve();
        pool_free(d_sumsq, st);
        if (herr & kErrTooManyPeaks)
            return set_error(ACOM_ERR_UNSUPPORTED,
                             "more than 1024 reflections near the Ewald sphere for one zone axis");
        return ACOM_OK;
    }
fail:
    pool_free(d_atoms, st);
    pool_free(d_tmp_g, st);
    pool_free(d_tmp_F, st);
    pool_free(d_g, st);
    pool_free(d_amp, st);
    pool_free(d_cnt, st);
    if (e == cudaErrorMemoryAllocation) return set_error(ACOM_ERR_OOM, "plan: device allocation");
    return cuda_error(e, "plan build");
#undef ACOM_TRY
}

}  // namespace acom
