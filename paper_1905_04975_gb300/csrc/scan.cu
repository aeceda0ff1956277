// Block-structure kernels of a real Schur form (Eq. 4): input validation,
// the subdiagonal pattern that marks the 2x2 blocks, and the eigenvalues read
// from the diagonal blocks.
#include "common.cuh"

#include <limits.h>

namespace gbr {

namespace {

// One warp per column: entries two or more below the diagonal must be zero;
// a 2x2 block [[a, b], [c, d]] (c != 0) must not overlap the next block and
// must be standardized (a == d, bc < 0).
__global__ void validate_kernel(int n, const double* __restrict__ S, int ldS,
                                DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nwarps) {
        bool bad = false;
        const double* col = S + cm(0, j, ldS);
        for (int i = j + 2 + lane; i < n; i += 32) bad |= (col[i] != 0.0);
        if (lane == 0 && j + 1 < n && col[j + 1] != 0.0) {
            double a = col[j], c = col[j + 1];
            double b = S[cm(j, j + 1, ldS)], d = S[cm(j + 1, j + 1, ldS)];
            if (j + 2 < n && S[cm(j + 2, j + 1, ldS)] != 0.0) bad = true;
            if (a != d) bad = true;
            if (!(b * c < 0.0)) bad = true;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMin(&ctr->bad_column, j);
    }
}

__global__ void subdiag_kernel(int n, const double* __restrict__ S, int ldS,
                               uint8_t* __restrict__ sub) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        sub[i] = (i + 1 < n && S[cm(i + 1, i, ldS)] != 0.0) ? 1 : 0;
}

// 1x1 block s -> (s, 0); standardized 2x2 [[a, b], [c, a]] -> a +- i sqrt(-bc),
// positive imaginary part on the first row.
__global__ void eigs_kernel(int n, const double* __restrict__ S, int ldS, double* __restrict__ wr,
                            double* __restrict__ wi) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double re = S[cm(i, i, ldS)], im = 0.0;
        if (i + 1 < n && S[cm(i + 1, i, ldS)] != 0.0) {
            im = sqrt(fabs(S[cm(i, i + 1, ldS)])) * sqrt(fabs(S[cm(i + 1, i, ldS)]));
        } else if (i > 0 && S[cm(i, i - 1, ldS)] != 0.0) {
            im = -(sqrt(fabs(S[cm(i - 1, i, ldS)])) * sqrt(fabs(S[cm(i, i - 1, ldS)])));
        }
        wr[i] = re;
        wi[i] = im;
    }
}

int grid_for(int n, int threads) {
    int g = (n + threads - 1) / threads;
    return g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
}

}  // namespace

cudaError_t launch_validate(int n, const double* S, int ldS, DevCounters* ctr, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int warps = n < 152 * 64 ? n : 152 * 64;
    int blocks = (warps * 32 + 255) / 256;
    validate_kernel<<<blocks, 256, 0, st>>>(n, S, ldS, ctr);
    return cudaGetLastError();
}

cudaError_t launch_subdiag(int n, const double* S, int ldS, uint8_t* sub, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    subdiag_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, S, ldS, sub);
    return cudaGetLastError();
}

cudaError_t launch_eigs(int n, const double* S, int ldS, double* wr, double* wi, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    eigs_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, S, ldS, wr, wi);
    return cudaGetLastError();
}

}  // namespace gbr
