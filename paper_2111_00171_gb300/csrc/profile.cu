// Per-kernel-class timing with CUDA events and a launch counter.
//
// When enabled, every library launch is bracketed by two events recorded on
// the launching stream; after the library's own stream synchronisation the
// pending pairs are resolved into per-class totals.  The launch counter runs
// always.  Process-global, not thread-safe.
#include <vector>

#include "acom_internal.cuh"

namespace acom {

namespace {
struct Pending {
    int cls;
    cudaEvent_t a, b;
};
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[kKCount] = {};
int64_t g_cnt[kKCount] = {};
int64_t g_launches = 0;
cudaEvent_t g_open[kKCount];
bool g_has_open[kKCount] = {};
const char* kNames[kKCount] = {"reflections", "raster_plan", "scale_plan", "raster_patterns",
                               "contract_fp32", "idft_argmax_fp32", "refine", "misc",
                               "contract_tc", "idft_argmax_tc", "rescore_fp32", "select_exact",
                               "refine_orient"};

cudaEvent_t take() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

thread_local bool t_suppress = false;

void prof_suppress(bool on) { t_suppress = on; }

void prof_begin(int cls, cudaStream_t st) {
    ++g_launches;
    if (!g_on || t_suppress) return;
    cudaEvent_t a = take();
    cudaEventRecord(a, st);
    g_open[cls] = a;
    g_has_open[cls] = true;
}

void prof_end(int cls, cudaStream_t st) {
    if (!g_on || t_suppress || !g_has_open[cls]) return;
    cudaEvent_t b = take();
    cudaEventRecord(b, st);
    g_pending.push_back({cls, g_open[cls], b});
    g_has_open[cls] = false;
}

void prof_resolve() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.cls] += ms;
            g_cnt[p.cls] += 1;
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace acom

extern "C" {

void acom_profile_enable(int32_t on) { acom::g_on = on != 0; }

void acom_profile_reset(void) {
    acom::prof_resolve();
    for (int i = 0; i < acom::kKCount; ++i) {
        acom::g_ms[i] = 0;
        acom::g_cnt[i] = 0;
    }
}

int32_t acom_profile_read(acom_profile_entry* out, int32_t max) {
    int n = 0;
    for (int i = 0; i < acom::kKCount && n < max; ++i) {
        if (!out) break;
        out[n].name = acom::kNames[i];
        out[n].launches = acom::g_cnt[i];
        out[n].total_ms = acom::g_ms[i];
        ++n;
    }
    return out ? n : acom::kKCount;
}

int64_t acom_kernel_launches(void) { return acom::g_launches; }

}  // extern "C"
