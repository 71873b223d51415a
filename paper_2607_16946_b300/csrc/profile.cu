// Kernel timing by CUDA events (sdf_profile_*): a tracing aid used to measure
// each kernel family's device time inside a longer timed region.  Every range
// is also an NVTX range named "ptsdf:<family>" on the launching host thread,
// which a profiler attached to the process shows around the launches (the
// header-only NVTX API does nothing when no tool is attached).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <mutex>
#include <vector>

#include "internal.h"

namespace ptsdf {

namespace {
struct Rec {
    int kernel;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
const char* kNames[SDF_K_COUNT_] = {"prepass", "fwd", "merge", "build", "fwd_grad", "bwd_params", "fwd_tc", "radius", "knn", "plane"};
const char* kNvtxNames[SDF_K_COUNT_] = {"ptsdf:prepass", "ptsdf:fwd", "ptsdf:merge", "ptsdf:build", "ptsdf:fwd_grad",
                                        "ptsdf:bwd_params", "ptsdf:fwd_tc", "ptsdf:radius", "ptsdf:knn", "ptsdf:plane"};

void clear_locked() {
    for (auto& r : g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
}
}  // namespace

ProfRange::ProfRange(int kernel, cudaStream_t st) : st_(st), idx_(-1) {
    nvtxRangePushA(kernel >= 0 && kernel < SDF_K_COUNT_ ? kNvtxNames[kernel] : "ptsdf");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    Rec r{kernel, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
        cudaEventDestroy(r.a);
        return;
    }
    cudaEventRecord(r.a, st);
    idx_ = (int)g_recs.size();
    g_recs.push_back(r);
}

ProfRange::~ProfRange() {
    nvtxRangePop();
    if (idx_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx_ < (int)g_recs.size()) cudaEventRecord(g_recs[idx_].b, st_);
}

}  // namespace ptsdf

using namespace ptsdf;

extern "C" sdf_status sdf_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (on) clear_locked();
    g_on = on != 0;
    return SDF_OK;
}

extern "C" sdf_status sdf_profile_read(int32_t kernel, int64_t* launches, double* total_ms) {
    if (kernel < 0 || kernel >= SDF_K_COUNT_ || !launches || !total_ms)
        return set_error(SDF_EINVAL, "sdf_profile_read: bad kernel id or NULL output");
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t n = 0;
    double ms = 0.0;
    for (const auto& r : g_recs) {
        if (r.kernel != kernel) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_error(e, "sdf_profile_read");
        ++n;
        ms += t;
    }
    *launches = n;
    *total_ms = ms;
    return SDF_OK;
}

extern "C" const char* sdf_kernel_name(int32_t kernel) {
    return (kernel >= 0 && kernel < SDF_K_COUNT_) ? kNames[kernel] : nullptr;
}
