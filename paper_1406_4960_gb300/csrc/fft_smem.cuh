// Radix-2 FFTs of planes held in shared memory (used by the radix-2 plane
// kernel of the H apply and by the density and Coulomb kernels of the
// self-consistent loop).
#pragma once

#include "cplx.cuh"

namespace mb {

// radix-2 FFTs on ns planes of N1 x N2 in shared memory (row-major, i2 fastest)
// Inverse: decimation in frequency, natural in -> bit-reversed out, sign +.
// Forward: decimation in time, bit-reversed in -> natural out, sign -.
template <typename R2, bool INV>
__device__ void fft_axis(R2 *buf, int ns, int N1, int N2, int axis, const R2 *tw, int nmax) {
    const int NN = N1 * N2;
    const int N = axis == 2 ? N2 : N1;
    const int estride = axis == 2 ? 1 : N2;
    const int ntr_plane = axis == 2 ? N1 : N2;
    const int ntr = ns * ntr_plane;
    const int nbf = ntr * (N / 2);
    for (int stage = 0, half = INV ? N / 2 : 1; INV ? half >= 1 : half < N;
         ++stage, half = INV ? half / 2 : half * 2) {
        const int twstep = nmax / (2 * half);
        for (int bi = threadIdx.x; bi < nbf; bi += blockDim.x) {
            int tr = bi / (N / 2);
            int r = bi - tr * (N / 2);
            int plane = tr / ntr_plane;
            int line = tr - plane * ntr_plane;
            int base = plane * NN + (axis == 2 ? line * N2 : line);
            int grp = r / half;
            int j = r - grp * half;
            int i0 = grp * 2 * half + j;
            int i1 = i0 + half;
            R2 w = tw[j * twstep];
            R2 *p0 = buf + base + i0 * estride;
            R2 *p1 = buf + base + i1 * estride;
            R2 a = *p0, b = *p1;
            if (INV) {
                *p0 = a + b;
                *p1 = cmul(a - b, w);
            } else {
                R2 t = cmul_c(b, w);
                *p0 = a + t;
                *p1 = a - t;
            }
        }
        __syncthreads();
    }
}

}  // namespace mb
