// Tensor-core (tcgen05) contraction over shells with the spectral-bound
// epilogue (section "Correlation Pattern Matching"; see match_prune.cu for the
// bound).
//
// Per frequency f the pattern spectra (shells x patterns, BF16) meet the plan
// spectra (zone axes x shells, BF16) on the 5th-generation tensor cores in one
// MMA per 16 shells:
//   D = X_f [Pr_f ; Pi_f]^T,  M = 128 pattern rows, N = 256 axis rows,
// FP32 accumulation in tensor memory.  Each 16-row group of the pattern tile
// holds the real parts of 8 patterns and then their imaginary parts, so TMEM
// lanes L and L + 8 carry Xr and Xi of one pattern; D columns 0..127 are the
// axes' real parts and 128..255 their imaginary parts.  A 16x256b TMEM load
// hands one thread (Xr.Pr, Xi.Pr) of lanes (L, L + 8), and the same load 128
// columns on gives (Xr.Pi, Xi.Pi): the four products A = Pr.Xr, C = Pr.Xi,
// D = Pi.Xr, B = Pi.Xi of a pair meet in one thread, which accumulates
// w_f max(|(A+B) + i(C-D)|, |(A-B) - i(C+D)|) over f.  The spectra never leave
// the chip; only U is written.
//
// A thread issues one tcgen05.mma per ~120 cycles whatever its size, about the
// time an M = 128, N = 256, K = 16 MMA takes on the tensor core, and every
// barrier round trip and commit between MMAs leaves the tensor core idle.  So
// one N = 256 MMA per 16 shells, and two issuing warps: warp 1 takes the even
// frequencies into TMEM buffer 0, warp 2 the odd ones into buffer 1, and their
// MMAs interleave in the tensor pipe.  Both consume stages of one operand ring
// in the producer's order; each issuer has its own full barrier per ring slot
// (the producer signals the stage's owner), so every full barrier has one
// consumer and its phases are consumed in order.  A slot's empty barrier is
// committed by the owner of each use; the producer issues the next use only
// after that commit, so those phases are ordered too.
//
// CTA: two TMA producer warps (warp 0 loads the pattern operand X, warp 3 the
// plan operand: one box of 256 rows, the axis tile's real rows followed by its
// imaginary rows), two MMA-issuing warps, sixteen epilogue warps; persistent
// over (64-pattern x 128-axis) tiles; with 16-bit operands a ring stage holds
// two K tiles of 64 elements (128-byte rows, 128-byte swizzle), the whole K
// range of a frequency on the 1-degree plan, in two stages of 96 KB, and each
// K tile completes on its own full barrier, so the first K tile's MMAs start
// while the second K tile lands; accumulators are double-buffered over f in
// 512 TMEM columns.  Issuing a TMA copy costs the
// issuing thread a few hundred cycles whatever the box (measured: one thread
// issuing three boxes per stage was busy 80 % of the time, and halving the
// boxes' rows or bytes changed nothing), so the copies of a stage are
// issued by two threads and the plan operand is one box.
// Every mbarrier wait is bounded: a timeout sets the device error word, stops
// all roles, drains copies and MMAs in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>
#include <math_constants.h>

#include "acom_internal.cuh"

namespace acom {
namespace tc {

constexpr int kM = 128;               // zone axes per tile (MMA N = 256 rows: re, im)
constexpr int kNP = 64;               // patterns per tile (MMA M = 128 rows: re, im)
constexpr int kKT = 64;               // 16-bit operands per K tile row (128 bytes)
constexpr int kKT8 = 128;             // 8-bit operands per K tile row (128 bytes)
constexpr int kTileBytes = 128 * kKT * 2;      // 16 KB
constexpr int kEpiWarps = 16;
constexpr int kIssuers = 2;                    // MMA-issuing warps, one per TMEM buffer
constexpr int kProdP = 1 + kIssuers;           // warp of the plan-operand producer
constexpr int kEpi0 = kProdP + 1;               // first epilogue warp
constexpr int kThreads = (kEpi0 + kEpiWarps) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

// instruction descriptors: D f32, A and B both bf16 (format 1) or both f16
// (format 0), both K-major, N = 256, M = 128
constexpr uint32_t kIdescF16 = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescBF16 = kIdescF16 | (1u << 7) | (1u << 10);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait of at most `budget` clock cycles; false on timeout (recorded)
// or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, long long budget) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) {
            atomicOr(err, kErrTimeout);
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_f16kind(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// E4M3 x E4M3 -> FP32 (both operands the same type; K = 32 per instruction,
// the same 32 bytes of each operand row as K = 16 of a 16-bit type)
__device__ __forceinline__ void mma_f8kind(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- CTA pairs (cta_group::2): a cluster of two CTAs shares each MMA ----
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// the shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t caddr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
// a TMA copy into this CTA's shared memory that completes on a barrier of
// either CTA of the pair (`bar` a shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mma_f16kind_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                                 uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_f8kind_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the barrier at this offset in both CTAs once this thread's MMAs complete
__device__ __forceinline__ void mma_commit_pair_both(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(bar), "h"((uint16_t)3)
        : "memory");
}
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 16 TMEM lanes x 32 columns: thread t receives, for n = 0..3, lane t/4 at
// columns 8n + 2(t%4) + {0, 1} in r[4n], r[4n+1] and lane t/4 + 8 at the same
// columns in r[4n+2], r[4n+3]
#define ACOM_TMEM_LD16x256_X4(taddr, r)                                                      \
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,"    \
                 "%10,%11,%12,%13,%14,%15}, [%16];"                                          \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),   \
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), \
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                        \
                 : "r"(taddr))

// wait for this thread's TMEM loads; the registers are tied to the wait so no
// use can be scheduled before it
#define ACOM_TMEM_WAIT32(p, q)                                                             \
    asm volatile("tcgen05.wait::ld.sync.aligned;"                                          \
                 : "+r"(p[0]), "+r"(p[1]), "+r"(p[2]), "+r"(p[3]), "+r"(p[4]), "+r"(p[5]), \
                   "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]),            \
                   "+r"(p[11]), "+r"(p[12]), "+r"(p[13]), "+r"(p[14]), "+r"(p[15]),        \
                   "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), \
                   "+r"(q[6]), "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]),            \
                   "+r"(q[11]), "+r"(q[12]), "+r"(q[13]), "+r"(q[14]), "+r"(q[15])         \
                 :                                                                         \
                 : "memory")

// |c| from |c|^2 (approximate square root, relative error ~2^-23, covered by
// the bound's rounding margin)
__device__ __forceinline__ float mag_from_sq(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// w max(|c_dir|, |c_mir|) added to the bound of two pairs (axes z and z + 1,
// adjacent registers of a 16x256b load): with p = A^2+B^2+C^2+D^2 and
// q = AB - CD, |c_dir|^2 = |(A+B) + i(C-D)|^2 = p + 2q and
// |c_mir|^2 = |(A-B) - i(C+D)|^2 = p - 2q, so the larger is p + 2|q|.  Packed
// FP32x2 arithmetic halves the epilogue's instructions, which share the issue
// slots with the MMA-issuing warps.
__device__ __forceinline__ void accumulate_pair2(uint32_t a0, uint32_t a1, uint32_t c0,
                                                 uint32_t c1, uint32_t d0, uint32_t d1,
                                                 uint32_t b0, uint32_t b1, float w, float& acc0,
                                                 float& acc1) {
    float t0, t1;
    asm("{\n"
        ".reg .b64 A, B, C, D, P, Q, R;\n"
        "mov.b64 A, {%2, %3};\n"
        "mov.b64 C, {%4, %5};\n"
        "mov.b64 D, {%6, %7};\n"
        "mov.b64 B, {%8, %9};\n"
        "mul.rn.f32x2 P, D, D;\n"
        "fma.rn.f32x2 P, C, C, P;\n"
        "fma.rn.f32x2 P, B, B, P;\n"
        "fma.rn.f32x2 P, A, A, P;\n"
        "mul.rn.f32x2 Q, C, D;\n"
        "mul.rn.f32x2 R, A, B;\n"
        "sub.rn.f32x2 Q, R, Q;\n"
        "and.b64 Q, Q, 0x7FFFFFFF7FFFFFFF;\n"
        "add.rn.f32x2 Q, Q, Q;\n"
        "add.rn.f32x2 P, P, Q;\n"
        "mov.b64 {%0, %1}, P;\n"
        "}\n"
        : "=f"(t0), "=f"(t1)
        : "r"(a0), "r"(a1), "r"(c0), "r"(c1), "r"(d0), "r"(d1), "r"(b0), "r"(b1));
    acc0 = fmaf(w, mag_from_sq(t0), acc0);
    acc1 = fmaf(w, mag_from_sq(t1), acc1);
}

struct TcArgs {
    int F, N, Z, nb, ZT, PT, KT;   // frequencies, bins, axes, patterns, axis tiles, pattern tiles, K tiles
    int PTs;                       // pattern tiles per frequency in the pattern map (row stride)
    int Spad;                      // shells (K) in the operand rows
    int k0;                        // first shell of the contraction's K range (the
                                   // plan's rows below it are zero for every axis)
    int Zrows;                     // rows per frequency in the plan map (ZT * 256)
    float* U;                      // [nb][Z]
    int* err;
    uint32_t idesc;                // MMA instruction descriptor (operand format)
    const float* xscale;           // [nb] 2^e of FP16 pattern spectra, or nullptr
    float xs_mul;                  // the operands hold xscale * xs_mul times X^
    float inv_pscale;              // 2^-k of the plan operand's scale (1 for BF16)
    int zmajor;                    // tile order: 0 consecutive tiles share a pattern
                                   // tile, 1 they share an axis tile
    long long wait_cycles;         // budget of each pipeline wait (the drain waits
                                   // that precede the exit always take kWaitCycles)
};

// F8: E4M3 operands (kind::f8f6f4, 128 elements per K tile), else 16-bit
// (kind::f16, 64 elements per K tile); a template parameter, so the MMA issue
// loop carries no branch on it
// Ring geometry.  A stage holds kSub K tiles of X (16 KB each) and of the B
// operand: for a single CTA with 16-bit operands two K tiles (128 shells: the
// whole K range of a frequency on the 1-degree plan, so one barrier round trip
// per frequency instead of two), X 32 KB + B 64 KB, two stages; with E4M3
// operands (128 shells per K tile already) one K tile, four stages; a CTA of a
// pair stages X and its half of B (16 KB each), so a pair's ring is deeper.
// A single CTA with two K tiles per stage gives each K tile its own full
// barrier (kFull = 2): the issuer starts the first K tile's MMAs while the
// second K tile's copies are still landing (measured: 9.32 -> 8.98 ms per step
// on the 256 x 256 scan, the same bounds bit for bit); the stage is still
// released by one commit.
template <bool F8, bool PAIR>
struct Ring {
    static constexpr int kSub = (PAIR || F8) ? 1 : 2;
    static constexpr int kStageBytes = kSub * (PAIR ? 2 : 3) * kTileBytes;
    static constexpr int kStages = PAIR ? 6 : (kSub == 2 ? 2 : 4);
    static constexpr int kFull = kSub;      // full barriers per stage and issuer
};

// F8: E4M3 operands (kind::f8f6f4, 128 elements per K tile), else 16-bit
// (kind::f16, 64 elements per K tile); a template parameter, so the MMA issue
// loop carries no branch on it.
// PAIR: a cluster of two CTAs computes each MMA together (cta_group::2,
// M = 256): CTA rank r of the pair holds pattern tile 2 p + r of the pair's
// pattern tiles (its A rows) and half of the axis tile's B operand (rank 0 the
// real rows, rank 1 the imaginary rows); rank 0's two threads issue every MMA,
// whose accumulators land in both CTAs' tensor memory, lanes = the CTA's own
// patterns, columns = all 256 B rows, exactly as for a single CTA.  Both CTAs'
// copies complete on rank 0's full barriers; commits arrive on both CTAs'
// barriers; both epilogues release rank 0's accumulator barrier.
template <bool F8, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
k_contract_bound_tc(const __grid_constant__ CUtensorMap map_p,
                    const __grid_constant__ CUtensorMap map_x, TcArgs a) {
    constexpr int kSt = Ring<F8, PAIR>::kStages;
    constexpr int kSB = Ring<F8, PAIR>::kStageBytes;
    constexpr int kSub = Ring<F8, PAIR>::kSub;
    constexpr int kFS = Ring<F8, PAIR>::kFull;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the operand ring
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* ring = base;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + kSt * kSB);
    uint64_t* full = bars;                          // [kIssuers][kSt][kFS]
    uint64_t* empty = bars + kIssuers * kSt * kFS;  // [kSt]
    uint64_t* tfull = empty + kSt;              // [kIssuers]
    uint64_t* tempty = tfull + kIssuers;        // [kIssuers]
    uint64_t* drain = tempty + kIssuers;        // [kIssuers]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + kIssuers);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const bool leader = rank == 0;
    // the pair's abort flag of the other CTA: a timeout stops both CTAs
    const uint32_t peer_abort =
        PAIR ? mapa_rank(smem_u32(const_cast<int*>(abort_flag)), rank ^ 1u) : 0u;
    if (threadIdx.x == 0) {
        // a full barrier completes on the arrivals of the (leading CTA's) two
        // producers and the bytes of every copy of its K tile (of the stage)
        for (int s = 0; s < kIssuers * kSt * kFS; ++s) mbar_init(smem_u32(full + s), 2);
        for (int s = 0; s < kSt; ++s) mbar_init(smem_u32(empty + s), 1);
        for (int b = 0; b < kIssuers; ++b) {
            mbar_init(smem_u32(tfull + b), 1);
            mbar_init(smem_u32(tempty + b), (PAIR ? 2 : 1) * kEpiWarps);
            mbar_init(smem_u32(drain + b), 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_p)));
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_x)));
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    fence_before();
    if constexpr (PAIR)
        cluster_sync_all();      // both CTAs' barriers exist before any copy or arrival
    else
        __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    // tiles: single CTA (axis tile, pattern tile); pair (axis tile, pair of
    // pattern tiles), the pair's CTAs taking the two pattern tiles
    const int PTu = PAIR ? (a.PT + 1) / 2 : a.PT;
    const int n_tiles = a.ZT * PTu;
    const int t0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int tstep = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    auto set_abort = [&]() {
        if constexpr (PAIR) st_cluster_u32(peer_abort, 1u);
    };
    bool aborted = false;

    if (warp == 0 || warp == kProdP) {
        // ------------------------------------------------ TMA producers: warp 0
        // the pattern operand, warp kProdP the plan operand of every stage
        const bool xprod = warp == 0;
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            // per issuer and slot: the parity of the owner's next full phase;
            // the last stage issued into each slot and its owner, for the drain
            uint32_t fpar[kIssuers] = {0u, 0u};
            uint32_t issued_mask = 0, last_par = 0, last_own = 0;
            int fcount = 0;
            bool ok = true;
            for (int t = t0; t < n_tiles && ok; t += tstep) {
                const int zt = a.zmajor ? t / PTu : t % a.ZT;
                const int pu = a.zmajor ? t % PTu : t / a.ZT;
                const int pt = PAIR ? 2 * pu + (int)rank : pu;
                for (int f = 0; f < a.F && ok; ++f, ++fcount) {
                    // a pair's CTA loads the real (rank 0) or imaginary rows of the tile
                    const int prow = f * a.Zrows + zt * 256 + (PAIR ? 128 * (int)rank : 0);
                    const int xrow = (f * a.PTs + pt) * 128;
                    const int own = fcount & 1;
                    for (int kt = 0; kt < a.KT; ++kt) {
                        if (!mbar_wait(smem_u32(empty + stage), phase ^ 1u, abort_flag, a.err,
                                       a.wait_cycles)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = smem_u32(full + (own * kSt + stage) * kFS);
                        unsigned char* sbuf = ring + stage * kSB;
                        constexpr int ktel = F8 ? kKT8 : kKT;
                        // the stage's first shell; K tiles past the padded shells are
                        // not loaded (nor expected, nor multiplied)
                        const int kbase = a.k0 + kt * ktel * kSub;
                        const int nsub = (kSub == 1 || a.Spad - kbase > ktel) ? kSub : 1;
                        if constexpr (PAIR) {
                            // every copy completes on the leading CTA's barrier, which
                            // expects both CTAs' bytes of its operand
                            const uint32_t fbl = mapa_rank(fb, 0);
                            if (leader) mbar_expect_tx(fb, 2 * kTileBytes);
                            if (xprod)
                                tma_load_2d_pair(smem_u32(sbuf), &map_x, kbase, xrow, fbl);
                            else
                                tma_load_2d_pair(smem_u32(sbuf + kTileBytes), &map_p, kbase,
                                                 prow, fbl);
                        } else if (kFS > 1) {
                            // K tile u completes on full barrier u (X: 16 KB, the
                            // plan's 256-row box: 32 KB); a K tile past the padded
                            // shells is only arrived on, so every barrier of the
                            // stage completes once per use
                            for (int u = 0; u < kFS; ++u) {
                                const uint32_t fbu = fb + 8u * (uint32_t)u;
                                if (u < nsub) {
                                    mbar_expect_tx(fbu, (xprod ? 1 : 2) * kTileBytes);
                                    if (xprod)
                                        tma_load_2d(smem_u32(sbuf + u * kTileBytes), &map_x,
                                                    kbase + u * ktel, xrow, fbu);
                                    else
                                        tma_load_2d(smem_u32(sbuf + (kSub + 2 * u) * kTileBytes),
                                                    &map_p, kbase + u * ktel, prow, fbu);
                                } else {
                                    mbar_arrive(fbu);
                                }
                            }
                        } else if (xprod) {
                            mbar_expect_tx(fb, nsub * kTileBytes);
                            for (int u = 0; u < nsub; ++u)
                                tma_load_2d(smem_u32(sbuf + u * kTileBytes), &map_x,
                                            kbase + u * ktel, xrow, fb);
                        } else {
                            // B operand: 256 rows, the tile's re rows then its im rows
                            mbar_expect_tx(fb, nsub * 2 * kTileBytes);
                            for (int u = 0; u < nsub; ++u)
                                tma_load_2d(smem_u32(sbuf + (kSub + 2 * u) * kTileBytes), &map_p,
                                            kbase + u * ktel, prow, fb);
                        }
                        issued_mask |= 1u << stage;
                        const uint32_t par = (fpar[own] >> stage) & 1u;
                        last_par = (last_par & ~(1u << stage)) | (par << stage);
                        last_own = (last_own & ~(1u << stage)) | ((uint32_t)own << stage);
                        fpar[own] ^= 1u << stage;
                        if (++stage == kSt) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                aborted = true;
                set_abort();
                if (!PAIR || leader) {
                    // let copies in flight land before the CTA's shared memory goes away
                    for (int s = 0; s < kSt; ++s)
                        if (issued_mask & (1u << s)) {
                            const uint32_t par = (last_par >> s) & 1u;
                            const int own = (last_own >> s) & 1u;
                            for (int u = 0; u < kFS; ++u) {
                                const long long w0 = clock64();
                                while (!mbar_try(smem_u32(full + (own * kSt + s) * kFS + u), par) &&
                                       clock64() - w0 < kWaitCycles) {
                                }
                            }
                        }
                } else {
                    // this CTA's copies complete on the other CTA's barriers: give
                    // them time to land (a copy takes microseconds)
                    const long long w0 = clock64();
                    while (clock64() - w0 < (1LL << 22)) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp <= kIssuers) {
        // ------------------------------------------------ MMA issuers
        // issuer mi takes the frequencies with fcount % 2 == mi into TMEM
        // buffer mi; it walks the ring in the producer's order and waits only
        // on its own full barriers (a pair: the leading CTA's issuers only)
        const int mi = warp - 1;
        if (lane == 0 && (!PAIR || leader)) {
            int stage = 0;
            uint32_t fpar = 0;           // bit s: parity of this issuer's next phase of slot s
            uint32_t tph = 0;
            int fcount = 0;
            bool ok = true;
            uint64_t* myfull = full + mi * kSt * kFS;
            for (int t = t0; t < n_tiles && ok; t += tstep) {
                for (int f = 0; f < a.F && ok; ++f, ++fcount) {
                    if ((fcount & 1) != mi) {
                        stage = (stage + a.KT) % kSt;
                        continue;
                    }
                    if (!mbar_wait(smem_u32(tempty + mi), tph ^ 1u, abort_flag, a.err,
                                   a.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    tph ^= 1u;
                    fence_after();
                    const uint32_t dacc = tmem + mi * 256;
                    for (int kt = 0; kt < a.KT; ++kt) {
                        const uint32_t spar = (fpar >> stage) & 1u;
                        fpar ^= 1u << stage;
                        const uint32_t sb = smem_u32(ring + stage * kSB);
                        // K steps of 32 bytes inside the shells (16 16-bit or 32
                        // 8-bit elements; the tail of the last tile is TMA zero
                        // fill); a step moves the descriptors' start address by
                        // 32 bytes (2 units of 16)
                        constexpr int ktel = F8 ? kKT8 : kKT;
                        const int kbase = a.k0 + kt * ktel * kSub;
                        const int nk = (min(ktel * kSub, a.Spad - kbase) * (F8 ? 1 : 2)) >> 5;
#pragma unroll
                        for (int j = 0; j < 4 * kSub; ++j) {
                            // before the stage's first MMA (one full barrier) or
                            // each K tile's first (one per K tile)
                            if ((kFS > 1 && (j & 3) == 0) || j == 0) {
                                if (!mbar_wait(smem_u32(myfull + stage * kFS + (kFS > 1 ? (j >> 2) : 0)),
                                               spar, abort_flag, a.err, a.wait_cycles)) {
                                    ok = false;
                                    break;
                                }
                                fence_after();
                            }
                            if (j < nk) {
                                // K tile j / 4 of the stage, step j % 4 inside it
                                const int k4 = j & 3, u = j >> 2;
                                const uint64_t xa = sdesc(sb + u * kTileBytes);
                                const uint64_t pb = sdesc(sb + (kSub + 2 * u) * kTileBytes);
                                const uint32_t acc = (kt | j) ? 1u : 0u;
                                if constexpr (PAIR) {
                                    if constexpr (F8)
                                        mma_f8kind_pair(dacc, xa + 2 * k4, pb + 2 * k4, a.idesc, acc);
                                    else
                                        mma_f16kind_pair(dacc, xa + 2 * k4, pb + 2 * k4, a.idesc, acc);
                                } else {
                                    if constexpr (F8)
                                        mma_f8kind(dacc, xa + 2 * k4, pb + 2 * k4, a.idesc, acc);
                                    else
                                        mma_f16kind(dacc, xa + 2 * k4, pb + 2 * k4, a.idesc, acc);
                                }
                            }
                        }
                        if (!ok) break;
                        // frees the stage (in both CTAs of a pair)
                        if constexpr (PAIR)
                            mma_commit_pair_both(smem_u32(empty + stage));
                        else
                            mma_commit(smem_u32(empty + stage));
                        if (++stage == kSt) stage = 0;
                    }
                    if (ok) {                                    // accumulators ready
                        if constexpr (PAIR)
                            mma_commit_pair_both(smem_u32(tfull + mi));
                        else
                            mma_commit(smem_u32(tfull + mi));
                    }
                }
            }
            if (!ok) {
                aborted = true;
                set_abort();
            }
            // all MMAs issued by this thread complete before TMEM is released
            if constexpr (PAIR)
                mma_commit_pair(smem_u32(drain + mi));
            else
                mma_commit(smem_u32(drain + mi));
            const long long w0 = clock64();
            while (!mbar_try(smem_u32(drain + mi), 0) && clock64() - w0 < kWaitCycles) {
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;                  // TMEM lane quarter: patterns 16q .. 16q + 15
        const int zq = (warp - kEpi0) >> 2;      // axis columns 32 zq .. 32 zq + 31
        const float invN = 1.0f / (float)a.N;
        float ud[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) ud[j] = 0.f;
        uint32_t tph[2] = {0, 0};
        int fcount = 0;
        bool ok = true;
        // the accumulator barriers live in the leading CTA
        const uint32_t tempty_l[2] = {PAIR ? mapa_rank(smem_u32(tempty), 0) : smem_u32(tempty),
                                      PAIR ? mapa_rank(smem_u32(tempty + 1), 0)
                                           : smem_u32(tempty + 1)};
        for (int t = t0; t < n_tiles && ok; t += tstep) {
            const int zt = a.zmajor ? t / PTu : t % a.ZT;
            const int pu = a.zmajor ? t % PTu : t / a.ZT;
            const int pt = PAIR ? 2 * pu + (int)rank : pu;
            for (int f = 0; f < a.F; ++f, ++fcount) {
                const int buf = fcount & 1;
                if (!mbar_wait(smem_u32(tfull + buf), tph[buf], abort_flag, a.err, a.wait_cycles)) {
                    ok = false;
                    break;
                }
                tph[buf] ^= 1u;
                fence_after();
                const float w = (f == 0 || 2 * f == a.N) ? 1.f : 2.f;
                const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + buf * 256 + zq * 32;
                // two halves of 8 patterns (16 lanes each); the second half's
                // loads are in flight while the first is reduced
                uint32_t R0[16], I0[16], R1[16], I1[16];
                ACOM_TMEM_LD16x256_X4(tb, R0);                          // (Xr, Xi) . Pr
                ACOM_TMEM_LD16x256_X4(tb + 128, I0);                    // (Xr, Xi) . Pi
                ACOM_TMEM_WAIT32(R0, I0);
                ACOM_TMEM_LD16x256_X4(tb + (16u << 16), R1);
                ACOM_TMEM_LD16x256_X4(tb + (16u << 16) + 128, I1);
#pragma unroll
                for (int n = 0; n < 4; ++n)
                    accumulate_pair2(R0[4 * n], R0[4 * n + 1], R0[4 * n + 2], R0[4 * n + 3],
                                     I0[4 * n], I0[4 * n + 1], I0[4 * n + 2], I0[4 * n + 3], w,
                                     ud[2 * n], ud[2 * n + 1]);
                ACOM_TMEM_WAIT32(R1, I1);
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR)
                        mbar_arrive_cluster(tempty_l[buf]);
                    else
                        mbar_arrive(tempty_l[buf]);
                }
#pragma unroll
                for (int n = 0; n < 4; ++n)
                    accumulate_pair2(R1[4 * n], R1[4 * n + 1], R1[4 * n + 2], R1[4 * n + 3],
                                     I1[4 * n], I1[4 * n + 1], I1[4 * n + 2], I1[4 * n + 3], w,
                                     ud[8 + 2 * n], ud[8 + 2 * n + 1]);
            }
            if (!ok) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = pt * kNP + 8 * (2 * q + h) + (lane >> 2);
                // FP16 spectra carry power-of-two scales: divide them out
                const float sc = (a.xscale && b < a.nb)
                                     ? invN * a.inv_pscale / (a.xscale[b] * a.xs_mul)
                                     : invN * a.inv_pscale;
#pragma unroll
                for (int n = 0; n < 4; ++n)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int z = zt * kM + zq * 32 + 8 * n + 2 * (lane & 3) + e;
                        if (b < a.nb && z < a.Z) a.U[(int64_t)b * a.Z + z] = ud[h * 8 + 2 * n + e] * sc;
                        ud[h * 8 + 2 * n + e] = 0.f;
                    }
            }
        }
        if (!ok && lane == 0) set_abort();
    }
    (void)aborted;
    fence_before();
    if constexpr (PAIR)
        cluster_sync_all();      // the leading CTA's MMAs and every copy are done in both CTAs
    else
        __syncthreads();
    if (warp == 1) {
        fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(kTmemCols)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(kTmemCols)
                         : "memory");
    }
}

template <bool F8, bool PAIR>
size_t tc_smem_bytes() {
    return 1024 + (size_t)Ring<F8, PAIR>::kStages * Ring<F8, PAIR>::kStageBytes +
           8 * ((kIssuers * Ring<F8, PAIR>::kFull + 1) * Ring<F8, PAIR>::kStages + 3 * kIssuers) + 16;
}

}  // namespace tc

// ---------------------------------------------------------------------------
// host side: tensor maps and launch
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool get_encoder() {
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return true;
}

// 2-D operand map: rows x cols (cols contiguous), boxes of 128 bytes x box_rows
// rows (64 16-bit or 128 8-bit columns), 128-byte swizzle; boxes reaching
// past the last column are zero-filled.  kind: 0 BF16, 1 FP16, 2 E4M3 (as
// bytes).
acom_status make_bf16_map(void* map_storage, const void* base, uint64_t rows, uint64_t cols,
                          int kind, int box_rows) {
    if (!get_encoder()) return set_error(ACOM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    const uint64_t eb = kind == 2 ? 1 : 2;
    if ((cols * eb) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
        return set_error(ACOM_ERR_INVALID_ARG, "tensor map: stride or base not 16-byte aligned");
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(map_storage);
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * eb};
    if (box_rows < 8 || box_rows > 256 || box_rows % 8 != 0)
        return set_error(ACOM_ERR_INVALID_ARG, "tensor map: unsupported box");
    const cuuint32_t box[2] = {(cuuint32_t)(kind == 2 ? tc::kKT8 : tc::kKT), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = kind == 2   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = g_encode(m, dt, 2, const_cast<void*>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(ACOM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return ACOM_OK;
}

size_t tensor_map_bytes() { return sizeof(CUtensorMap); }

// Budget of the contraction's pipeline waits (acom_set_device_wait_limit);
// 0: the default of about 2 s.  Process-global.
static long long g_wait_cycles = 0;
void set_wait_cycles(long long cycles) { g_wait_cycles = cycles > 0 ? cycles : 0; }

void launch_contract_bound_tc(const acom_plan_s* p, const void* map_x, int pt_stride, int nb,
                              float* U, cudaStream_t st, const float* xscale, int tile_order,
                              int cta_pairs) {
    tc::TcArgs a;
    a.zmajor = tile_order == 1 ? 1 : 0;
    a.F = p->F;
    a.N = p->N;
    a.Z = p->Z;
    a.nb = nb;
    a.ZT = p->Zp / tc::kM;
    a.PT = (nb + tc::kNP - 1) / tc::kNP;
    a.PTs = pt_stride;
    const bool f8 = p->precision == ACOM_PREC_FP8;
    const int ktel = f8 ? tc::kKT8 : tc::kKT;
    // the K range starts at the plan's first non-zero shell (a multiple of 16);
    // KT stages of kSub K tiles each per frequency
    a.k0 = p->k0;
    auto stages = [&](int sub) { return (p->Spad - p->k0 + ktel * sub - 1) / (ktel * sub); };
    a.Spad = p->Spad;
    a.Zrows = 2 * p->Zp;
    a.U = U;
    a.err = p->err;
    // E4M3 is format 0 for A and B, the same bits as F16
    a.idesc = p->precision == ACOM_PREC_BF16 ? tc::kIdescBF16 : tc::kIdescF16;
    a.xscale = xscale;
    a.xs_mul = f8 ? kFp8Shift : 1.0f;
    a.inv_pscale = 1.0f / p->pscale;
    a.wait_cycles = g_wait_cycles > 0 ? g_wait_cycles : tc::kWaitCycles;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(map_x);
    if (cta_pairs && nsm >= 2) {
        // CTA pairs: M = 256 (the pair's two pattern tiles), each CTA loading
        // half of the 256 B rows (128-row boxes)
        a.idesc = (a.idesc & ~(0x1Fu << 24)) | ((256u >> 4) << 24);
        a.KT = stages(1);
        const size_t smem = f8 ? tc::tc_smem_bytes<true, true>() : tc::tc_smem_bytes<false, true>();
        auto kern = f8 ? tc::k_contract_bound_tc<true, true> : tc::k_contract_bound_tc<false, true>;
        set_max_dynamic_smem((const void*)kern, smem);
        const int n_tiles = a.ZT * ((a.PT + 1) / 2);
        const int clusters = n_tiles < nsm / 2 ? n_tiles : nsm / 2;
        if (clusters <= 0) return;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * clusters, 1, 1);
        cfg.blockDim = dim3(tc::kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        prof_begin(kKContractBf16, st);
        cudaLaunchKernelEx(&cfg, kern, *reinterpret_cast<const CUtensorMap*>(p->map_p128), mx, a);
        prof_end(kKContractBf16, st);
        return;
    }
    a.KT = f8 ? stages(tc::Ring<true, false>::kSub) : stages(tc::Ring<false, false>::kSub);
    const size_t smem = f8 ? tc::tc_smem_bytes<true, false>() : tc::tc_smem_bytes<false, false>();
    auto kern = f8 ? tc::k_contract_bound_tc<true, false> : tc::k_contract_bound_tc<false, false>;
    set_max_dynamic_smem((const void*)kern, smem);
    const int n_tiles = a.ZT * a.PT;
    const int grid = n_tiles < nsm ? n_tiles : nsm;
    if (grid <= 0) return;
    prof_begin(kKContractBf16, st);
    kern<<<grid, tc::kThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap*>(p->map_p), mx, a);
    prof_end(kKContractBf16, st);
}

// FP32 spectra [Zp][F][Spad] (real and imaginary arrays) -> the merged
// tensor-core operand [F][Zp / 128][256][Spad]: per frequency and 128-axis
// tile, the 128 real rows then the 128 imaginary rows, BF16 / FP16 / E4M3 of
// scale x (a power of two, exact in FP32).
template <class T>
__device__ __forceinline__ T to_half_type(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_half_type<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half to_half_type<__half>(float x) {
    return __float2half_rn(x);
}
template <>
__device__ __forceinline__ __nv_fp8_e4m3 to_half_type<__nv_fp8_e4m3>(float x) {
    return __nv_fp8_e4m3(x);           // round to nearest, saturating to +-448
}

template <class T>
__global__ void k_plan_to_operand(const float* __restrict__ Pr, const float* __restrict__ Pi,
                                  int Zp, int F, int Spad, T* __restrict__ dst, float scale) {
    // one warp per operand row (f, zt, row): row < 128 takes the real part of
    // axis zt 128 + row, row >= 128 the imaginary part of axis zt 128 + row - 128;
    // lanes over the shells, four at a time (Spad is a multiple of 32)
    const int lane = threadIdx.x & 31;
    const int64_t orow = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int ZT = Zp / 128;
    if (orow >= (int64_t)F * ZT * 256) return;
    const int row = (int)(orow % 256);
    const int64_t t = orow / 256;
    const int zt = (int)(t % ZT), f = (int)(t / ZT);
    const int z = zt * 128 + (row & 127);
    const float4* src = reinterpret_cast<const float4*>((row < 128 ? Pr : Pi) +
                                                        ((int64_t)z * F + f) * Spad);
    T* d = dst + orow * Spad;
    for (int q = lane; q < Spad / 4; q += 32) {
        const float4 v = src[q];
        d[4 * q] = to_half_type<T>(scale * v.x);
        d[4 * q + 1] = to_half_type<T>(scale * v.y);
        d[4 * q + 2] = to_half_type<T>(scale * v.z);
        d[4 * q + 3] = to_half_type<T>(scale * v.w);
    }
}

void launch_plan_to_operand(const float* Pr, const float* Pi, int Zp, int F, int Spad, void* dst,
                            cudaStream_t st, int kind, float scale) {
    const int64_t rows = (int64_t)F * (Zp / 128) * 256;        // one warp per row
    const unsigned blocks = (unsigned)((rows + 7) / 8);
    prof_begin(kKMisc, st);
    if (kind == 2)
        k_plan_to_operand<__nv_fp8_e4m3><<<blocks, 256, 0, st>>>(
            Pr, Pi, Zp, F, Spad, reinterpret_cast<__nv_fp8_e4m3*>(dst), scale);
    else if (kind == 1)
        k_plan_to_operand<__half><<<blocks, 256, 0, st>>>(Pr, Pi, Zp, F, Spad,
                                                           reinterpret_cast<__half*>(dst), scale);
    else
        k_plan_to_operand<__nv_bfloat16><<<blocks, 256, 0, st>>>(
            Pr, Pi, Zp, F, Spad, reinterpret_cast<__nv_bfloat16*>(dst), 1.0f);
    prof_end(kKMisc, st);
}

// FP16 operand rows -> E4M3 rows times mul (a power of two, exact), 8 per thread.
__global__ void k_half_to_e4m3(const __half* __restrict__ src, uint8_t* __restrict__ dst,
                               int64_t n8, float mul) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n8;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4*>(src)[i];
        const __half2* h = reinterpret_cast<const __half2*>(&v);
        uint16_t o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 f = __half22float2(h[j]);
            f.x *= mul;
            f.y *= mul;
            o[j] = (uint16_t)__nv_cvt_float2_to_fp8x2(f, __NV_SATFINITE, __NV_E4M3);
        }
        reinterpret_cast<uint2*>(dst)[i] = *reinterpret_cast<const uint2*>(o);
    }
}

void launch_half_to_e4m3(const void* src, void* dst, int64_t n, float mul, cudaStream_t st) {
    const int64_t n8 = n / 8;
    if (n8 <= 0) return;
    const int blocks = (int)std::min<int64_t>((n8 + 255) / 256, 152 * 32);
    prof_begin(kKMisc, st);
    k_half_to_e4m3<<<blocks, 256, 0, st>>>(reinterpret_cast<const __half*>(src),
                                            reinterpret_cast<uint8_t*>(dst), n8, mul);
    prof_end(kKMisc, st);
}

}  // namespace acom
