// C ABI entry points declared in include/mb.h.
#include <cstring>
#include <new>

#include "mb_internal.h"

using namespace mb;

namespace mb {
int eigsolve(mb_handle *h, int nbands, double tol, int prec, double *evals, void *evecs,
             const mb_solve_opts *sopts, mb_solve_info *info, cudaStream_t s);
}

namespace mb {
int setup_device(mb_handle *h) {
    if (cudaSetDevice(h->device) != cudaSuccess) return MB_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) {
        h->smem_optin = (int)prop.sharedMemPerBlockOptin;
        h->num_sms = prop.multiProcessorCount;
    }
    return upload_tables(h);
}
}  // namespace mb

extern "C" {

int mb_setup(const mb_cell *cell, const double *kpts, int nk, double ecut, const double *breaks,
             int nbreaks, int order, const mb_atom *atoms, int natoms, const mb_opts *opts,
             mb_handle **out) {
    if (!out) return MB_EINVAL;
    *out = nullptr;
    if (!opts) return MB_EINVAL;
    mb_handle *h = new (std::nothrow) mb_handle();
    if (!h) return MB_ENOMEM;
    h->device = opts->device;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts->device < 0 || opts->device >= ndev) {
        delete h;
        return MB_ECUDA;
    }
    int rc = build_host_tables(h, cell, kpts, nk, ecut, breaks, nbreaks, order, atoms, natoms, opts);
    if (rc == MB_OK) rc = setup_device(h);
    if (rc != MB_OK) {
        free_tables(h);
        delete h;
        return rc;
    }
    *out = h;
    return MB_OK;
}

void mb_destroy(mb_handle *h) {
    if (!h) return;
    free_tables(h);
    delete h;
}

int mb_sizes(const mb_handle *h, int ik, int *ng, int *nb, int *ldg) {
    if (!h || ik < 0 || ik >= (int)h->kp.size()) return MB_EINVAL;
    if (ng) *ng = h->kp[ik].ng;
    if (nb) *nb = h->nb;
    if (ldg) *ldg = h->kp[ik].ldg;
    return MB_OK;
}

int mb_gvectors(const mb_handle *h, int ik, int *idx) {
    if (!h || !idx || ik < 0 || ik >= (int)h->kp.size()) return MB_EINVAL;
    const KPoint &kp = h->kp[ik];
    for (int g = 0; g < kp.ng; ++g) {
        idx[2 * g] = kp.n1[g];
        idx[2 * g + 1] = kp.n2[g];
    }
    return MB_OK;
}

int mb_zplanes(const mb_handle *h, int *nq, double *zq, double *wq) {
    if (!h) return MB_EINVAL;
    if (nq) *nq = h->nq;
    if (zq) std::memcpy(zq, h->zq.data(), sizeof(double) * h->nq);
    if (wq) std::memcpy(wq, h->wq.data(), sizeof(double) * h->nq);
    return MB_OK;
}

int mb_set_local_potential(mb_handle *h, const double *V) {
    if (!h || !V || !h->d_vloc) return MB_EINVAL;
    size_t n = (size_t)h->nq * h->n1 * h->n2;
    for (size_t i = 0; i < n; ++i)
        if (!(V[i] == V[i]) || V[i] > 1e300 || V[i] < -1e300) return MB_EINVAL;   // NaN / inf
    // the old tables may still be read by queued work on any stream
    if (cudaSetDevice(h->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MB_ECUDA;
    MB_CUDA(cudaMemcpyAsync(h->d_vloc, V, n * sizeof(double), cudaMemcpyHostToDevice, h->hs));
    return vloc_derive_tables(h);
}

int mb_local_potential(mb_handle *h, double *V) {
    if (!h || !V || !h->d_vloc) return MB_EINVAL;
    MB_CUDA(cudaSetDevice(h->device));
    MB_CUDA(cudaMemcpyAsync(V, h->d_vloc, (size_t)h->nq * h->n1 * h->n2 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->hs));
    MB_CUDA(cudaStreamSynchronize(h->hs));
    return MB_OK;
}

int mb_apply_H(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, void *stream) {
    if (!h) return MB_EINVAL;
    const void *xs[1] = {X};
    void *ys[1] = {Y};
    return apply_H_batch(h, 1, &ik, xs, ys, nbands, prec, (cudaStream_t)stream);
}

int mb_apply_H_batch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                     int nbands, int prec, void *stream) {
    if (!h) return MB_EINVAL;
    return apply_H_batch(h, nsel, iks, X, Y, nbands, prec, (cudaStream_t)stream);
}

int mb_apply_S(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, void *stream) {
    if (!h) return MB_EINVAL;
    const void *xs[1] = {X};
    void *ys[1] = {Y};
    return apply_banded_batch(h, BAND_S, 1, &ik, xs, ys, nbands, prec, (cudaStream_t)stream);
}

int mb_apply_Sinv(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, void *stream) {
    if (!h) return MB_EINVAL;
    const void *xs[1] = {X};
    void *ys[1] = {Y};
    return apply_banded_batch(h, BAND_SINV, 1, &ik, xs, ys, nbands, prec, (cudaStream_t)stream);
}

int mb_apply_S_batch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands,
                     int prec, void *stream) {
    if (!h) return MB_EINVAL;
    return apply_banded_batch(h, BAND_S, nsel, iks, X, Y, nbands, prec, (cudaStream_t)stream);
}

int mb_apply_Sinv_batch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands,
                        int prec, void *stream) {
    if (!h) return MB_EINVAL;
    return apply_banded_batch(h, BAND_SINV, nsel, iks, X, Y, nbands, prec, (cudaStream_t)stream);
}

int mb_status(mb_handle *h) {
    if (!h) return MB_EINVAL;
    if (!h->d_tcerr) return MB_OK;
    if (cudaSetDevice(h->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return MB_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, h->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MB_ECUDA;
    if (v && cudaMemset(h->d_tcerr, 0, sizeof(int)) != cudaSuccess) return MB_ECUDA;
    return v ? MB_ETIMEOUT : MB_OK;
}

int mb_eigsolve(mb_handle *h, int nbands, double tol, int prec, double *evals, void *evecs,
                const mb_solve_opts *sopts, mb_solve_info *info, void *stream) {
    if (!h) return MB_EINVAL;
    return eigsolve(h, nbands, tol, prec, evals, evecs, sopts, info, (cudaStream_t)stream);
}

const char *mb_strerror(int code) {
    switch (code) {
        case MB_OK: return "ok";
        case MB_EINVAL: return "invalid argument";
        case MB_ENOMEM: return "out of memory";
        case MB_ENOTCONV: return "eigensolver did not converge";
        case MB_ETIMEOUT: return "device wait timed out";
        case MB_ECUDA: return "CUDA runtime error";
        case MB_EUNSUPPORTED: return "unsupported request";
        default: return "unknown error";
    }
}

const char *mb_last_cuda_error(const mb_handle *h) {
    return h ? h->last_cuda_error.c_str() : "";
}

}  // extern "C"
