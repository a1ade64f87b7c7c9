/* Cyclic Jacobi diagonalization of a complex Hermitian matrix (§II.C: the
 * paper diagonalizes every subspace matrix by the Jacobi method).
 *
 * Oracle code: plain, sequential, FP64.  Test infrastructure only.
 *
 * For each pair p < q in row order, the 2x2 Hermitian block
 * [[a_pp, a_pq], [conj(a_pq), a_qq]] is brought to real form by the phase
 * exp(-i arg a_pq) on column q and then annihilated by a real plane rotation
 * (tangent t of the smaller angle).  Sweeps repeat until the off-diagonal
 * Frobenius norm falls below rel_tol times the Frobenius norm of the input.
 *
 * a:      n*n complex (interleaved re, im), row-major, overwritten.
 * evals:  n reals (ascending on return).
 * evecs:  n*n complex row-major, column c is the eigenvector of evals[c];
 *         may be NULL.
 * returns the number of sweeps used, or -1 if max_sweeps was reached.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static double offnorm2(const cplx *a, int n) {
    double s = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            if (i != j) s += creal(a[i * n + j] * conj(a[i * n + j]));
    return s;
}

int oracle_jacobi_herm(int n, double *a_in, double *evals, double *evecs_out,
                       double rel_tol, int max_sweeps) {
    cplx *a = (cplx *)a_in;
    cplx *v = (cplx *)malloc(sizeof(cplx) * (size_t)n * (size_t)n);
    if (!v) return -2;
    memset(v, 0, sizeof(cplx) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; i++) v[i * n + i] = 1.0;

    double fro2 = 0.0;
    for (int i = 0; i < n * n; i++) fro2 += creal(a[i] * conj(a[i]));
    /* force an exactly Hermitian start */
    for (int i = 0; i < n; i++) {
        a[i * n + i] = creal(a[i * n + i]);
        for (int j = i + 1; j < n; j++) {
            cplx m = 0.5 * (a[i * n + j] + conj(a[j * n + i]));
            a[i * n + j] = m;
            a[j * n + i] = conj(m);
        }
    }
    double stop2 = rel_tol * rel_tol * fro2;
    int sweep = 0, converged = 0;
    for (; sweep < max_sweeps; sweep++) {
        if (offnorm2(a, n) <= stop2) { converged = 1; break; }
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                cplx apq = a[p * n + q];
                double mag = cabs(apq);
                if (mag == 0.0) continue;
                double app = creal(a[p * n + p]), aqq = creal(a[q * n + q]);
                cplx e = apq / mag;               /* exp(i phi) */
                double theta = (aqq - app) / (2.0 * mag);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                cplx ec = conj(e);                /* exp(-i phi) */
                /* columns: A <- A J, J = diag(1, exp(-i phi)) * [[c, s], [-s, c]] */
                for (int r = 0; r < n; r++) {
                    cplx xp = a[r * n + p], xq = a[r * n + q];
                    a[r * n + p] = c * xp - s * ec * xq;
                    a[r * n + q] = s * xp + c * ec * xq;
                    cplx vp = v[r * n + p], vq = v[r * n + q];
                    v[r * n + p] = c * vp - s * ec * vq;
                    v[r * n + q] = s * vp + c * ec * vq;
                }
                /* rows: A <- J^H A */
                for (int r = 0; r < n; r++) {
                    cplx yp = a[p * n + r], yq = a[q * n + r];
                    a[p * n + r] = c * yp - s * e * yq;
                    a[q * n + r] = s * yp + c * e * yq;
                }
                a[p * n + q] = 0.0;
                a[q * n + p] = 0.0;
                a[p * n + p] = app - t * mag;
                a[q * n + q] = aqq + t * mag;
            }
        }
    }
    /* selection sort ascending, permuting eigenvector columns */
    int *perm = (int *)malloc(sizeof(int) * (size_t)n);
    double *ev = (double *)malloc(sizeof(double) * (size_t)n);
    if (!perm || !ev) {
        free(perm); free(ev); free(v);
        return -2;
    }
    for (int i = 0; i < n; i++) { perm[i] = i; ev[i] = creal(a[i * n + i]); }
    for (int i = 0; i < n; i++) {
        int m = i;
        for (int j = i + 1; j < n; j++) if (ev[perm[j]] < ev[perm[m]]) m = j;
        int tmp = perm[i]; perm[i] = perm[m]; perm[m] = tmp;
    }
    for (int i = 0; i < n; i++) evals[i] = ev[perm[i]];
    if (evecs_out) {
        cplx *vo = (cplx *)evecs_out;
        for (int r = 0; r < n; r++)
            for (int i = 0; i < n; i++) vo[r * n + i] = v[r * n + perm[i]];
    }
    free(perm); free(ev); free(v);
    return converged ? sweep : -1;
}
