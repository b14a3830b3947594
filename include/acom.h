/*
 * acom.h - C ABI of the GB300 sparse correlation match (automated crystal
 * orientation mapping by sparse correlation matching, arXiv 2111.00171).
 *
 * The library builds an orientation plan for a crystal and matches Bragg-peak
 * lists against it on one CUDA device (sm_103a).  Every entry point takes
 * plain pointers and sizes; no C++ or PyTorch type crosses this boundary and
 * no exception escapes it.  All device work is ordered on the caller's CUDA
 * stream (``cuda_stream`` is a cudaStream_t; NULL means the legacy default
 * stream).
 *
 * Error behaviour: every entry point returns an acom_status.  Arguments are
 * validated before any launch; on error nothing is launched and outputs are
 * untouched, except where noted for device-side validation.  A human-readable
 * message for the most recent error of the calling thread is returned by
 * acom_last_error().
 */
#ifndef ACOM_H
#define ACOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ACOM_OK = 0,
    ACOM_ERR_INVALID_ARG = 1,  /* bad pointer, size or option; nothing launched    */
    ACOM_ERR_OOM = 2,          /* device allocation failed                          */
    ACOM_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed              */
    ACOM_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                */
    ACOM_ERR_UNSUPPORTED = 5,  /* size or mode outside the compiled limits          */
    ACOM_ERR_BAD_INPUT = 6     /* device-side check of the peak data failed         */
} acom_status;

/* Arithmetic used by the shell contraction and the inverse transform. */
typedef enum {
    ACOM_PREC_FP32 = 0,   /* FP32 CUDA-core path (reference GPU path)               */
    ACOM_PREC_BF16 = 1,   /* BF16 operands on tcgen05 tensor cores, FP32 accumulate,
                             top candidates re-scored in FP32                       */
    ACOM_PREC_FP16 = 2,   /* FP16 operands on tcgen05 tensor cores, FP32 accumulate;
                             pattern and plan spectra are scaled by powers of two
                             into FP16 range and the bound scaled back; top
                             candidates re-scored in FP32                           */
    ACOM_PREC_FP8 = 3     /* experiment: E4M3 operands (the FP16 operands times
                             2^-6, exact) on the tensor cores, FP32 accumulate.
                             Their 2^-4 rounding makes the certified margin about
                             a quarter of the bound, so certified pruning
                             evaluates most axes; use rescore_top            */
} acom_precision;

typedef struct acom_plan_s* acom_plan;

/*
 * Crystal (section "Structure Factor Calculations"): lattice vectors a, b, c
 * as the rows of ``lattice`` (Angstrom, Cartesian), and the atomic basis:
 * fractional positions p_n in [0, 1) and the form factor of each atom,
 * f_n(q) = ff_A[n] exp(-ff_B[n] q^2) with q = |g| in 1/Angstrom (no 2 pi).
 * All pointers are HOST memory, read during the call only.
 */
typedef struct {
    double lattice[3][3];
    int32_t n_atoms;          /* 1 .. 64                                         */
    const double* frac_pos;   /* [n_atoms][3]                                   */
    const double* ff_A;       /* [n_atoms]                                      */
    const double* ff_B;       /* [n_atoms]                                      */
} acom_crystal;

/*
 * Zone-axis grid (section "Generation of an Orientation Plan"): three
 * boundary directions of the symmetry-reduced region (crystal Cartesian, any
 * length, rows of ``v``) sampled by spherical linear interpolation.  With
 * n = floor(sqrt(2 solid_angle) / step) the points are, for i = 0..n and
 * j = 0..i, slerp(slerp(v0,v1,i/n), slerp(v0,v2,i/n), j/i), in (i, j) order.
 */
typedef struct {
    double v[3][3];
    double step_deg;          /* > 0                                            */
    double solid_angle;       /* steradians of the region (4 pi / 48 for m-3m)  */
} acom_za_grid;

/* Radial shells q_s = (s + 1) * dq, s = 0 .. n_shells - 1 (1/Angstrom). */
typedef struct {
    int32_t n_shells;         /* 1 .. 512                                       */
    double dq;                /* > 0                                            */
} acom_shells;

/*
 * Plan options.  ``delta`` is the correlation kernel size, ``gamma_pow`` and
 * ``omega`` the radial and amplitude power laws of the plan and image
 * expressions, ``lambda`` the electron wavelength (Angstrom), ``q_max`` the
 * reflection cut-off 0 < |g| < q_max, ``precision`` an acom_precision.
 */
typedef struct {
    double delta;
    double gamma_pow;
    double omega;
    double lambda;
    double q_max;
    int32_t precision;
} acom_plan_opts;

/*
 * acom_plan_create - build the orientation plan (section "Generation of an
 * Orientation Plan"): structure factors F_hkl of every reflection with
 * 0 < |g| < q_max (Eqs. 2-3, FP64 phase sums on the device), the zone-axis
 * grid and the rotation of each axis onto +z (the first two factors of
 * Eq. 10), excitation errors (Eq. 6, beam along -z), the plan P0 over
 * (zone axis, phi3, q_s), its normalisation A = 1/||P0||_2, and the Fourier
 * transform of P = A P0 along phi3 (n_phi bins phi_j = 2 pi j / n_phi).
 *
 *   crystal, grid, shells, opts : host structs, read during the call.
 *   n_phi      : in-plane bins, even, 8 .. 720.
 *   sigma_exc  : excitation-error tolerance sigma of the Gaussian shape factor
 *                (Eq. 8); the plan itself does not use it (the tent of size
 *                delta carries the excitation error), it is kept on the plan
 *                for forward models.
 *   cuda_stream: stream on which the build runs; the call returns after the
 *                plan is complete (it synchronises that stream once).
 *   out        : receives the plan handle.  The plan owns its device memory
 *                until acom_plan_destroy; it is bound to the device current at
 *                creation.
 */
acom_status acom_plan_create(const acom_crystal* crystal, const acom_za_grid* grid,
                             const acom_shells* shells, int32_t n_phi, double sigma_exc,
                             const acom_plan_opts* opts, void* cuda_stream,
                             acom_plan* out);

/* Release a plan and all its device memory (after work on it has finished). */
acom_status acom_plan_destroy(acom_plan plan);

typedef struct {
    int32_t n_za;             /* Z zone axes                                    */
    int32_t n_shells;         /* S                                              */
    int32_t n_phi;            /* N                                              */
    int32_t n_freq;           /* F = N/2 + 1                                    */
    int32_t n_reflections;    /* reflections kept (0 < |g| < q_max, F != 0)     */
    int32_t precision;
    int64_t device_bytes;     /* device memory owned by the plan                */
    int64_t last_evaluated;   /* zone axes evaluated in full by the last match  */
    int32_t n_phases;         /* crystal structures (1 unless concatenated)     */
    int64_t last_refine_pairs; /* (reflection, peak) pairs the last acom_refine
                                  summed over all its score evaluations        */
    int32_t k0;               /* first shell of the tensor-core contraction: the
                                 plan's rows below it are zero for every axis,
                                 so those products are skipped (0: none)      */
} acom_plan_info;

acom_status acom_plan_get_info(acom_plan plan, acom_plan_info* info);

/*
 * acom_plan_concat - one plan for a sample of several phases (section "ACOM
 * Integration": with several crystal structures there is one orientation plan
 * and one correlation match per structure).  The zone axes of plans[0] come
 * first, then those of plans[1], and so on; phase p owns the axes
 * [offset_p, offset_{p+1}) (acom_plan_get_phases).  One acom_match on the
 * result rasterises each pattern once, contracts it against every phase's
 * axes in the same launches, and returns the best over all phases (so the
 * phase decision is the phase of the winning axis: the highest raw
 * correlation, ties to the lower phase) and, on request, each phase's best
 * score.
 *
 *   plans     : n_plans (1..8 phases in total; an input may itself be a
 *               concatenation) plans on the current device with equal n_shells,
 *               dq, n_phi, delta, gamma_pow, omega and precision, so that one
 *               polar image serves them all; ACOM_ERR_INVALID_ARG otherwise.
 *               They are read, not taken: the caller still owns and destroys
 *               them.
 *   cuda_stream: stream of the copies; the call synchronises it once.
 *   out       : receives the new plan, which owns copies of the inputs'
 *               spectra, axes, frames and neighbour lists (neighbours stay
 *               within their phase).
 */
acom_status acom_plan_concat(const acom_plan* plans, int32_t n_plans, void* cuda_stream,
                             acom_plan* out);

/* Copy the phase offsets (n_phases + 1 values: 0, Z_0, Z_0 + Z_1, ..., Z) to
 * HOST memory ``dst``.  Synchronous. */
acom_status acom_plan_get_phases(acom_plan plan, int32_t* dst);

/* Copy the zone axes (unit vectors, crystal Cartesian) to HOST memory
 * ``dst`` [Z][3].  Synchronous. */
acom_status acom_plan_get_zone_axes(acom_plan plan, double* dst);

/* Copy the plan spectrum FFT_phi3{P} to DEVICE memory ``dst`` laid out
 * [Z][S][F][2] (real, imaginary), FP32.  Stream-ordered. */
acom_status acom_plan_get_spectra(acom_plan plan, float* dst, void* cuda_stream);

/*
 * Bragg peaks of n_patterns diffraction patterns in CSR form (section
 * "Correlation Pattern Matching"): the peaks of pattern b are the entries
 * row_ptr[b] .. row_ptr[b+1]-1 of qx, qy (1/Angstrom, detector frame) and I
 * (intensity).  All pointers are DEVICE memory owned by the caller.
 * row_ptr[0] must be 0 and row_ptr non-decreasing; each pattern holds at most
 * 1024 peaks; values must be finite.  These properties are checked on the
 * device: a violation makes acom_match return ACOM_ERR_BAD_INPUT (outputs
 * are then undefined).
 */
typedef struct {
    int64_t n_patterns;
    const int64_t* row_ptr;   /* [n_patterns + 1]                               */
    const float* qx;          /* [row_ptr[n_patterns]]                          */
    const float* qy;
    const float* I;
} acom_peaks_csr;

/*
 * Per-pattern results, DEVICE memory owned by the caller, [n_patterns] unless
 * stated.  Pointers marked optional may be NULL.
 *   za_idx    best zone axis (maximum over zone axes of max(C, C_mirror))
 *   phi3_bin  its phi3 bin k (C is maximal at phi_k = 2 pi k / N)
 *   mirror    1 when C_mirror gave the maximum
 *   score     the maximum correlation value (raw C)
 *   score_cos optional: score / ||X||_2, in [0, 1] since ||P_z||_2 = 1
 *   phi3      optional: refined in-plane angle of the orientation (radians)
 *   orient    optional: [n_patterns][9] refined orientation matrix m, row
 *             major, mapping sample to crystal coordinates (Eq. 9)
 *   za_scores optional: [n_patterns][Z] max over phi3 and mirror per axis.
 *             With certified pruning (the default) the value is exact for
 *             every axis that was evaluated (the winner and every axis whose
 *             bound could reach it) and is otherwise an upper bound of the
 *             axis' maximum (the bound of acom_bounds plus a rounding margin).
 *   runner_za, runner_score, runner_orient  optional (certified pruning
 *             only; ACOM_ERR_UNSUPPORTED with exhaustive): the best zone axis
 *             outside the winner's grid neighbourhood, certified like the
 *             winner (every axis there whose bound could beat it is evaluated;
 *             -1 if the neighbourhood is the whole plan), its exact score, and
 *             its grid orientation [n_patterns][9] (no sub-grid refinement;
 *             the winner's when there is none): a second start for acom_refine
 *   phase     optional: the phase of za_idx (0 for a single-phase plan)
 *   phase_score optional: [n_patterns][n_phases] the best score of each
 *             phase (its maximum over its axes, phi3 and mirror).  With
 *             certified pruning, asking for it makes the search certify every
 *             phase's best, not only the overall winner; 0 for an all-zero
 *             image.
 * Ties: the lowest zone-axis index wins, then C before C_mirror, then the
 * lowest phi3 bin.
 */
typedef struct {
    int32_t* za_idx;
    int32_t* phi3_bin;
    uint8_t* mirror;
    float* score;
    float* score_cos;
    float* phi3;
    float* orient;
    float* za_scores;
    int32_t* phase;
    float* phase_score;
    int32_t* runner_za;
    float* runner_score;
    float* runner_orient;
} acom_result;

typedef struct {
    int32_t refine;           /* 1: sub-grid refinement of phi3 / orient        */
    int32_t chunk;            /* patterns per internal chunk, 0 = default       */
    int32_t exhaustive;       /* 1: inverse-transform every zone axis (test and
                                 reference mode); 0: certified pruning         */
    int32_t rescore_top;      /* > 0 (with exhaustive = 0): no certification;
                                 only the rescore_top axes of largest bound are
                                 evaluated exactly in FP32 and the best of them
                                 wins (the grid neighbours of the winner are
                                 evaluated for the refinement as usual)       */
    int32_t tile_order;       /* tensor-core contraction schedule: 0 consecutive
                                 tiles share a pattern tile (default), 1 they
                                 share a zone-axis tile                       */
    int32_t cta_pairs;        /* tensor-core contraction: 0 (default) one CTA
                                 per MMA; 1 pairs of CTAs compute each MMA
                                 together (cta_group::2, M = 256 pattern rows) */
} acom_match_opts;

/*
 * acom_autotune - the contraction's schedule picked by measurement: the
 * match of ``peaks`` (a representative sample, DEVICE) is timed (CUDA events,
 * after a warm-up match) for chunk sizes 8192, 16384 and 32768, both tile
 * orders and both CTA arrangements (one CTA or a CTA pair per MMA), with the
 * other options from ``base`` (may be NULL).  ``best`` receives the fastest
 * (chunk, tile_order, cta_pairs, ms), ``trials`` (optional, 12 entries) every
 * one.  Pass best's chunk, tile_order and cta_pairs in acom_match_opts.
 */
typedef struct {
    int32_t chunk;
    int32_t tile_order;
    int32_t cta_pairs;
    float ms;
} acom_tune_result;

acom_status acom_autotune(acom_plan plan, const acom_peaks_csr* peaks, const acom_match_opts* base,
                          acom_tune_result* best, acom_tune_result* trials, void* cuda_stream);

/*
 * acom_match - sparse correlation match (section "Correlation Pattern
 * Matching"): for every pattern, the sparse polar image X(phi3, q_s) of its
 * peaks, its Fourier transform along phi3, the contraction over shells with
 * the plan's conjugate spectra for every zone axis, the inverse transform to
 * C and C_mirror over phi3, the maximum over (zone axis, phi3, mirror), and
 * the refinement of the winner into an orientation matrix.
 *
 * Certified pruning (default): the contraction reduces each (zone axis,
 * pattern) pair to the bound U = (1/N) sum_f w_f max(|c_f^dir|, |c_f^mir|)
 * >= max_k max(C[k], C_mirror[k]) of its correlation spectra (w_0 = w_{N/2} =
 * 1, else 2) plus a rounding margin;
 * axes are then evaluated in full, in decreasing U, until no remaining bound
 * can reach the best score.  The winner equals that of the exhaustive
 * evaluation.  Zone-axis counts above 16384 require exhaustive mode.
 *
 * Work is queued on ``cuda_stream``; the call synchronises that stream once at
 * the end to read the device error word.  The first call on a plan allocates
 * its scratch workspace (sized for ``chunk`` patterns).  ``opts`` may be NULL.
 */
acom_status acom_match(acom_plan plan, const acom_peaks_csr* peaks,
                       const acom_match_opts* opts, acom_result* out,
                       void* cuda_stream);

/*
 * acom_match_async - acom_match without its final synchronisation: the work
 * is enqueued on ``cuda_stream`` and the call returns.  The error word and the
 * evaluation count go to pinned memory owned by the plan; acom_sync waits for
 * the stream and returns the status acom_match would have returned (and sets
 * last_evaluated).  Once the plan's workspace fits (after one acom_match with
 * the same chunk and mode) the call allocates nothing and makes no host
 * synchronisation, so it can be captured into a CUDA graph and the graph
 * replayed on new contents of the same peak and result buffers; under
 * capture it records no profiling events, and it refuses
 * (ACOM_ERR_INVALID_ARG) a workspace that would need allocating.
 */
acom_status acom_match_async(acom_plan plan, const acom_peaks_csr* peaks,
                             const acom_match_opts* opts, acom_result* out, void* cuda_stream);
acom_status acom_sync(acom_plan plan, void* cuda_stream);

/*
 * acom_match_multi - several orientations per pattern (section "Matching of
 * Overlapping Diffraction Patterns"): match; compute the forward pattern of
 * the match's grid orientation (the reflections of the plan whose Gaussian
 * shape factor D(s_g), Eq. 8 with the plan's sigma_exc, is at least 1e-3);
 * remove every peak within ``r_del`` of a forward spot and keep (d - r_del) /
 * (delta - r_del) of the intensity of those within the plan's delta; match
 * the rest again, n_matches times in all.
 *
 *   results   : n_matches (1..8) result structs as for acom_match (za_idx,
 *               phi3_bin, mirror, score required; the other fields optional).
 *               results[j] holds the j-th match of every pattern.  ``score``
 *               and ``score_cos`` are those of the ORIGINAL full pattern at
 *               the match's (zone axis, phi3 bin, mirror), as the paper
 *               reports them; orient/phi3 refine the match as acom_match does.
 *               za_idx = -1 marks "no further orientation": the best
 *               correlation of what was left was 0 (score 0).
 *   r_del     : deletion radius (1/Angstrom), 0 <= r_del < delta.
 *   opts      : as for acom_match (certified pruning or exhaustive).
 *
 * A single-phase plan (ACOM_ERR_UNSUPPORTED otherwise).  The peaks are read,
 * not changed (a working copy is made).  Synchronises the stream once per
 * match and once at the end.
 */
acom_status acom_match_multi(acom_plan plan, const acom_peaks_csr* peaks,
                             const acom_match_opts* opts, int32_t n_matches, float r_del,
                             acom_result* results, void* cuda_stream);

/*
 * acom_polar_spectra - the first half of acom_match alone: the sparse polar
 * image of every pattern and its Fourier transform along phi3, written to
 * DEVICE memory ``dst`` laid out [n_patterns][S][F][2] FP32, and optionally
 * ||X||_2 per pattern to ``xnorm`` [n_patterns] (may be NULL).  Stream-ordered;
 * synchronises once to read the error word.
 */
acom_status acom_polar_spectra(acom_plan plan, const acom_peaks_csr* peaks,
                               float* dst, float* xnorm, void* cuda_stream);

/*
 * Tracing: per-kernel-class device time.  When enabled, each kernel the
 * library launches is bracketed by CUDA events on its stream; the pairs are
 * resolved at the library's next stream synchronisation (end of acom_match,
 * acom_polar_spectra, acom_plan_create).  acom_profile_read fills up to
 * ``max`` entries (name, launches timed, total milliseconds) and returns the
 * number written (with out == NULL: the number of classes).
 * acom_kernel_launches counts every kernel the library has launched in this
 * process (timed or not).  Process-global state; not thread-safe.
 */
typedef struct {
    const char* name;
    int64_t launches;
    double total_ms;
} acom_profile_entry;

void acom_profile_enable(int32_t on);
void acom_profile_reset(void);
int32_t acom_profile_read(acom_profile_entry* out, int32_t max);
int64_t acom_kernel_launches(void);

/*
 * acom_device_allocations - how many device-memory (stream-ordered pool) and
 * pinned host allocations the library has requested in this process, whether
 * the pool served them from cached blocks or not.  A diagnostic: a caller
 * checks that a call allocated nothing by reading it before and after.
 */
int64_t acom_device_allocations(void);

/*
 * acom_set_device_wait_limit - failure detection of the tensor-core
 * contraction.  Its producer, MMA-issuing and epilogue roles wait on each
 * other through shared-memory barriers, every wait bounded by a budget of
 * clock cycles (default, cycles <= 0: 4e9, about 2 s).  A wait that runs out
 * sets the device error word and stops every role of its CTA; the CTA then
 * waits (always with the full budget) for its copies and MMAs in flight,
 * frees its tensor memory and exits, and the call returns ACOM_ERR_TIMEOUT
 * with the plan still usable.  A short budget makes a wait run out on
 * purpose (tests of that path); it applies to later launches of this
 * process.  Not thread-safe.
 */
void acom_set_device_wait_limit(int64_t cycles);

/*
 * Continuous refinement of orientations (the paper stops at the grid and its
 * sub-grid refinement; this makes the orientation a continuous variable).
 * The kinematical correlation score of a pattern with an orientation m
 * (R = m^T, crystal to lab) is
 *
 *   S(R) = sum_m sum_g a_m b_g exp(-|p_m - (R g)_xy|^2 / (2 rho^2)) / ||b||
 *
 * with p_m the peak positions, a_m = q_m^gamma I_m^(omega/2) the peak weights
 * of the polar image, and b_g = |g|^gamma |F_g|^omega D(s_g)^(omega/2) the
 * weight of the kinematical intensity of reflection g: D the Gaussian shape
 * factor (Eq. 8) with the plan's sigma_exc, s_g the excitation error of R g
 * (Eq. 6, beam along -z, the plan's lambda).  The reflections, gamma and omega
 * are the plan's (a single-phase plan; ACOM_ERR_UNSUPPORTED for a
 * concatenation).  FP32 arithmetic; rotations composed in FP64.
 */
typedef struct {
    int32_t steps;            /* damped Gauss-Newton ascent steps              */
    float rho_start;          /* spot width at the first step (1/Angstrom)     */
    float rho_end;            /* at the last step (geometric in between)       */
    float damping;            /* Levenberg-Marquardt damping of the step       */
    float max_step_deg;       /* cap on the rotation of one step               */
    int32_t twin;             /* 1: also refine m Rz(pi) (the in-plane Friedel
                                 twin a grid match cannot tell apart) and keep
                                 the higher final score                      */
} acom_refine_opts;

/* 20 steps, rho 0.15 -> 0.03, damping 0.3, 1 degree per step, twin on. */
acom_refine_opts acom_refine_defaults(void);

/*
 * acom_refine - for every pattern, `steps` ascent steps of S from the
 * orientation in ``orient`` ([n_patterns][9] FP32 row-major m, DEVICE, e.g.
 * acom_match's output), each w = (H + damping diag H)^-1 dS/dw applied as
 * R <- Exp(w) R (H the Gauss-Newton matrix, |w| capped), rho shrinking
 * geometrically; with ``orient_alt`` (optional, [n_patterns][9], e.g. the
 * match's runner_orient) the same from that second start; with opts->twin
 * also from the Friedel twin of each start.  The start whose refinement ends
 * with the highest S wins (ties: orient before its twin before orient_alt)
 * and its refined m overwrites ``orient``.  ``score`` (optional,
 * [n_patterns]) receives S at rho_end, ``start`` (optional, uint8) the
 * winning start: bit 0 twin, bit 1 orient_alt.  ``opts`` may be NULL
 * (defaults).  Stream-ordered; synchronises once to read the error word (bad
 * peak data: ACOM_ERR_BAD_INPUT).
 */
acom_status acom_refine(acom_plan plan, const acom_peaks_csr* peaks, const acom_refine_opts* opts,
                        float* orient, const float* orient_alt, float* score, uint8_t* start,
                        void* cuda_stream);

/*
 * acom_kinematical_score - S at R = Exp(r) m^T for each pattern, with m from
 * ``orient`` ([n][9], DEVICE) and r from ``r`` ([n][3] axis-angle, DEVICE;
 * NULL means r = 0), at spot width ``rho``.  Writes ``score`` [n], ``grad``
 * [n][3] = dS/dr (through the left Jacobian of SO(3)) and ``gn`` [n][6], the
 * Gauss-Newton matrix for a lab-frame rotation (xx, xy, xz, yy, yz, zz);
 * each output may be NULL.  Stream-ordered; synchronises once.
 */
acom_status acom_kinematical_score(acom_plan plan, const acom_peaks_csr* peaks, const float* orient,
                                   const float* r, float rho, float* score, float* grad,
                                   float* gn, void* cuda_stream);

/*
 * acom_kinematical_score_strain - the same with the reciprocal lattice of
 * each pattern deformed by a small symmetric strain e: every reflection g of
 * the plan moves to R (I + e) g, R = Exp(r) m^T (reading: strain moves the
 * spots and changes their excitation errors; the amplitudes |g|^gamma
 * |F_g|^omega keep their unstrained values).  ``strain`` [n][6] DEVICE
 * (xx, xy, xz, yy, yz, zz; NULL means e = 0); ``strain_grad`` [n][6] DEVICE
 * receives dS/de in the same component order, an off-diagonal component
 * counting both symmetric entries (dS/de_kl = sum_g u_k g_l + u_l g_k with
 * u = R^T dS/d(R (I + e) g)).  Other arguments, outputs and errors as for
 * acom_kinematical_score, which is this call with both strain pointers NULL.
 */
acom_status acom_kinematical_score_strain(acom_plan plan, const acom_peaks_csr* peaks,
                                          const float* orient, const float* r,
                                          const float* strain, float rho, float* score,
                                          float* grad, float* gn, float* strain_grad,
                                          void* cuda_stream);

/*
 * acom_bounds - the shell contraction alone: for every pattern and zone axis
 * the spectral bound U = (1/N) sum_f w_f max(|c_f^dir|, |c_f^mir|) of the
 * direct and mirror correlation spectra, which is >= max over phi3 of both C
 * and C_mirror (section "Correlation Pattern Matching"; w_0 = w_{N/2} = 1,
 * else 2).  Computed at the plan's precision (FP32 CUDA
 * cores, or BF16 / FP16 tensor cores with FP32 accumulation) without any
 * rounding margin.  ``dst``: DEVICE [n_patterns][Z] FP32.  Stream-ordered; synchronises
 * once to read the error word.
 */
acom_status acom_bounds(acom_plan plan, const acom_peaks_csr* peaks, float* dst,
                        void* cuda_stream);

/*
 * acom_bounds_static - the same result as acom_bounds, computed without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate while they run, such as an
 * acquisition loop that reserved its whole device-memory budget up front, or
 * a host process whose device memory is held by another allocator (a
 * cudaMalloc there could fail or stall).  The plan must already exist; the
 * caller passes the peaks and ``dst`` ([n_patterns][Z] FP32, DEVICE), as for
 * acom_bounds.  FP32 and BF16 plans get their own precision's bounds; FP16
 * and FP8 (E4M3) plans get the bounds of the FP32 path (every plan keeps its
 * FP32 spectra), i.e. the values an FP32 plan's acom_bounds returns.  Peak data
 * are checked as for acom_bounds (row_ptr[0] == 0, monotone rows, finite values,
 * at most 1024 peaks per pattern): a violation returns ACOM_ERR_BAD_INPUT.
 *
 * Scratch: the pattern spectra of one chunk live in a file-scope device array
 * of 32 MiB that every device loading the library keeps until the process
 * exits.  Patterns are processed in chunks of as many as that array holds for
 * the plan's geometry (a multiple of 64); plans whose geometry leaves room for
 * fewer than 64 patterns are rejected with ACOM_ERR_UNSUPPORTED.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  With CUDA's lazy module loading (the default) that first call is
 * also when the device commits the 32 MiB array and loads the modules of the
 * kernels it launches, so the first call on each device belongs in set-up;
 * later calls take no device memory.  All calls share the one array and leave the last call's contents
 * in it (every value a call reads it writes first), so calls whose work
 * overlaps on the GPU - on different streams, or from different threads -
 * race on the array and must be ordered by the caller.  The call performs no
 * cudaMalloc, cudaFree or other allocating library call, records no profiling
 * events, and synchronises ``cuda_stream`` once to read the error word.
 */
acom_status acom_bounds_static(acom_plan plan, const acom_peaks_csr* peaks, float* dst,
                               void* cuda_stream);

const char* acom_status_str(acom_status status);
const char* acom_last_error(void);

/* Library version, for the Python binding's compatibility check. */
int32_t acom_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ACOM_H */
