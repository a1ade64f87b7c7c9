// Launch accounting and optional per-kernel CUDA-event timing.
#include <mutex>
#include <set>
#include <utility>

#include "mb_internal.h"

namespace mb {

// Raise a kernel's dynamic shared-memory limit to `bytes` (the device's
// opt-in maximum) minus its static shared memory, once per (kernel, device)
// instead of on every launch.
cudaError_t smem_limit_once(const void *func, int device, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(func, device);
    if (done.count(key)) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

const char *const kKernelNames[KN_COUNT] = {
    "plane", "epilogue", "proj", "coef", "backproj", "banded", "gram", "combine",
    "jacobi", "small", "vec", "gram32", "combine32"};

// whether a launch of `kernel` is bracketed by events in the current mode
static bool prof_on(const mb_handle *h, int kernel) {
    return h->profiling == 1 || (h->profiling == 2 && kernel == KN_PLANE);
}

void prof_begin(mb_handle *h, cudaStream_t s, int kernel, cudaEvent_t *a) {
    h->launches++;
    *a = nullptr;
    if (!prof_on(h, kernel)) return;
    if (h->prof_pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        h->prof_pool.push_back(e);
    }
    *a = h->prof_pool.back();
    h->prof_pool.pop_back();
    cudaEventRecord(*a, s);
}

void prof_end(mb_handle *h, cudaStream_t s, int kernel, cudaEvent_t a) {
    if (!prof_on(h, kernel) || !a) return;
    cudaEvent_t b;
    if (h->prof_pool.empty()) {
        if (cudaEventCreate(&b) != cudaSuccess) return;
    } else {
        b = h->prof_pool.back();
        h->prof_pool.pop_back();
    }
    cudaEventRecord(b, s);
    h->prof_pending.push_back({kernel, a, b});
}

int prof_collect(mb_handle *h) {
    for (auto &p : h->prof_pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return cuda_fail(h, e);
        cudaEventElapsedTime(&ms, p.a, p.b);
        h->prof_ms[p.kernel] += ms;
        h->prof_count[p.kernel] += 1;
        h->prof_pool.push_back(p.a);
        h->prof_pool.push_back(p.b);
    }
    h->prof_pending.clear();
    return MB_OK;
}

}  // namespace mb

using namespace mb;

extern "C" {

int mb_set_profiling(mb_handle *h, int on) {
    if (!h) return MB_EINVAL;
    int rc = prof_collect(h);
    if (on < 0 || on > 2) return rc ? rc : MB_EINVAL;
    h->profiling = on;
    return rc;
}

int mb_profile_read(mb_handle *h, int kernel, double *ms_total, long long *count) {
    if (!h || kernel < 0 || kernel >= KN_COUNT) return MB_EINVAL;
    int rc = prof_collect(h);
    if (ms_total) *ms_total = h->prof_ms[kernel];
    if (count) *count = h->prof_count[kernel];
    return rc;
}

int mb_profile_reset(mb_handle *h) {
    if (!h) return MB_EINVAL;
    int rc = prof_collect(h);
    for (int i = 0; i < KN_COUNT; ++i) {
        h->prof_ms[i] = 0;
        h->prof_count[i] = 0;
    }
    return rc;
}

long long mb_launch_count(const mb_handle *h) { return h ? h->launches : -1; }

const char *mb_kernel_name(int kernel) {
    return (kernel >= 0 && kernel < KN_COUNT) ? kKernelNames[kernel] : "";
}

}  // extern "C"
