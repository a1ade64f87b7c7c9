// Generalized Lanczos-Krylov eigensolver (§II.C) -- placeholder until the
// device solver lands.
#include "mb_internal.h"

namespace mb {
int eigsolve(mb_handle *h, int nbands, double tol, int prec, double *evals, void *evecs,
             const mb_solve_opts *sopts, mb_solve_info *info, cudaStream_t s) {
    (void)h; (void)nbands; (void)tol; (void)prec; (void)evals; (void)evecs; (void)sopts; (void)info; (void)s;
    return MB_EUNSUPPORTED;
}
}  // namespace mb
