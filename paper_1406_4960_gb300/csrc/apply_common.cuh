// Launch descriptors shared by the apply kernels.
#pragma once

#include "cplx.cuh"

namespace mb {

constexpr int kMaxK = 64;   // k-points per launch (descriptors travel as kernel parameters)
constexpr int kMaxChunks = 64;   // runs of knot intervals per (k, band) in the plane kernel

// First knot interval of run c when nint intervals are split into nchunks
// runs of balanced length (lengths differ by at most one).
__host__ __device__ inline int chunk_begin(int c, int nint, int nchunks) {
    return (int)(((long long)c * nint) / nchunks);
}

struct KDesc {
    const void *X;
    void *Y;
    void *part;      // boundary partial rows
    void *W;         // projector overlaps: Zx[b][f][G] (CUDA-core path) or W[(b, j)][p] (tensor cores)
    void *C;         // projector coefficients: c[b][p] (CUDA-core path) or C[(b, j)][p] (tensor cores)
    int ng, ldg;
    int kofs;        // offset of per-k G arrays
    int qofs;        // offset of q_p(G) table
    int rows_ofs;    // offset of this k-point's list of grid rows that hold disc points
    int nrows;
    unsigned long long rowmask;   // bit i1 set when grid row i1 holds disc points
    unsigned rows_magic;          // floor(2^32 / nrows) + 1: e / nrows = umulhi(e, rows_magic)
    // compact planes (FP32 plane kernel): the disc's rows n1 = n1min ..
    // n1min + nocc - 1 stored as rows 0 .. nocc-1; zofs/nz: the positions of
    // those rows that hold no disc point (zeroed after every interval)
    int nocc, zofs, nz;
};

template <typename R> struct PlaneArgs {
    const R *Bq;
    const R *V;       // bit-reversed layout (radix-2 kernel)
    const R *Vn;      // natural layout (register-FFT kernel)
    const int *rows;  // active grid rows of every k-point
    const typename V2<R>::T *tw;
    const int *goff;
    const R *Vt;      // compact-plane kernel: [q][i2][i1], w_q V / (N1 N2), i1 fastest
    const int *cpos;  // compact-plane offset (n1 - n1min) (N2 + 1) + i2 of every G (offset kofs)
    const int *zpos;  // non-disc positions of the compact planes (offset zofs of each k-point)
    int n1, n2, l1, l2, nmax;
    int order, nquad, nint, nb;
    int nbands, nchunks, chunk, np, ldg_max;
    int nsel;
    int bt;           // bands per CTA (register-FFT kernel)
    int *queue;       // compact-plane kernel, persistent mode: {next item, finished CTAs}, zero between launches
    KDesc d[kMaxK];
};


// register-FFT plane kernel (plane_reg.cu): available grids and launch
template <typename R> bool plane_reg_supported(int n1, int n2, int order);
template <typename R>
cudaError_t plane_reg_launch(const PlaneArgs<R> &a, unsigned grid, size_t smem, cudaStream_t s);
void upload_fft_twiddles();

// FP32 compact-plane kernel (plane_reg.cu): one instance per grid shape, with
// compile-time bounds on the occupied rows (nocc) and the disc row width
// (ldg); the host checks a batch against them before choosing it.
struct Plane32Shape {
    bool ok = false;
    int id = -1;           // instance id
    char name[96] = {0};   // kernel instance
    int nocc_max = 0;      // largest nocc the instance stores
    int ldg_max = 0;       // threads x columns per thread
    int bt = 1;            // bands per CTA
    int threads = 0;
    int ctas_per_sm = 1;
    size_t smem_fixed = 0; // planes + accumulator ring (bytes); + 144 B per interval of a run
};
// the instances that can run a batch of this grid, occupied-row count and
// row width (default first); returns how many were written to out (<= max)
int plane32_shapes(int n1, int n2, int order, int nquad, int nocc, int ldg, Plane32Shape *out, int max);
constexpr int kMaxPlane32Shapes = 8;
cudaError_t plane32_launch(const PlaneArgs<float> &a, const Plane32Shape &sh, unsigned grid, size_t smem,
                           cudaStream_t s);

}  // namespace mb
