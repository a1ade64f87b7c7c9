// mb_apply_H_noalloc: the H apply of mb_apply_H for one k-point, with its
// scratch in a fixed array compiled into this file instead of device memory
// that the handle allocates on demand.
//
// The scratch holds the rows that two neighbouring runs of knot intervals
// both contribute to, the projector overlaps W and the back-projection
// coefficients C.  Every kernel of the apply writes each scratch element it
// later reads, so nothing has to start at zero and no clearing pass runs.
#include <mutex>

#include "mb_internal.h"

namespace mb {

// Device-side scratch.  In host code the name below is only a handle for
// cudaGetSymbolAddress: passing it to a kernel directly would hand the kernel
// a host address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MB_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};
}  // namespace

// Device address of g_noalloc_scratch on the handle's device, with that device
// current.  Outside stream capture it is looked up on every call (so a
// re-created context never leaves a stale address behind); inside a capture
// the address of the last uncaptured call on that device is used, and a
// first call inside a capture is refused (MB_EINVAL).
static int noalloc_scratch(mb_handle *h, cudaStream_t s, void **out) {
    if (h->device < 0 || h->device >= kMaxDevices) return MB_EINVAL;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(h, e);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(h, e);
        g_scratch_ptr[h->device] = p;
    } else if (!g_scratch_ptr[h->device]) {
        return MB_EINVAL;
    }
    *out = g_scratch_ptr[h->device];
    return MB_OK;
}

}  // namespace mb

using namespace mb;

extern "C" int mb_apply_H_noalloc(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec,
                                  void *stream) {
    if (!h || ik < 0 || ik >= (int)h->kp.size() || !X || !Y || X == Y) return MB_EINVAL;
    if (nbands <= 0 || nbands > h->max_bands) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    if (apply_H_scratch_need(h, ik, nbands, prec) > (size_t)MB_NOALLOC_SCRATCH_BYTES) return MB_EINVAL;
    void *scratch = nullptr;
    int rc = noalloc_scratch(h, (cudaStream_t)stream, &scratch);
    if (rc) return rc;
    return apply_H_on_scratch(h, ik, X, Y, nbands, prec, (cudaStream_t)stream, scratch);
}
