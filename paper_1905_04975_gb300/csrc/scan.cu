// Block-structure kernels of a real Schur form (Eq. 4): input validation,
// the subdiagonal pattern that marks the 2x2 blocks, and the eigenvalues read
// from the diagonal blocks.
#include "scan_body.cuh"

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

// Eigenvalues read off the diagonal blocks (eig_at).
__global__ void eigs_kernel(int n, const double* __restrict__ S, int ldS, double* __restrict__ wr,
                            double* __restrict__ wi) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        eig_at(n, S, ldS, i, &wr[i], &wi[i]);
}

// Batched forms: blockIdx.y (strided) picks the instance, the x dimension
// covers its positions.
__global__ void validate_batched_kernel(int count, const Inst* __restrict__ inst) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = blockIdx.y; b < count; b += gridDim.y) {
        const Inst I = inst[b];
        for (int j = warp; j < I.n; j += nwarps) {
            bool bad = false;
            const double* col = I.S + cm(0, j, I.ldS);
            for (int i = j + 2 + lane; i < I.n; i += 32) bad |= (col[i] != 0.0);
            if (lane == 0 && j + 1 < I.n && col[j + 1] != 0.0) {
                double a = col[j], c = col[j + 1];
                double bb = I.S[cm(j, j + 1, I.ldS)], d = I.S[cm(j + 1, j + 1, I.ldS)];
                if (j + 2 < I.n && I.S[cm(j + 2, j + 1, I.ldS)] != 0.0) bad = true;
                if (a != d) bad = true;
                if (!(bb * c < 0.0)) bad = true;
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMin(&I.ctr->bad_column, j);
        }
    }
}

__global__ void subdiag_batched_kernel(int count, const Inst* __restrict__ inst,
                                       const long long* __restrict__ off, uint8_t* __restrict__ sub,
                                       int* mismatch) {
    for (int b = blockIdx.y; b < count; b += gridDim.y) {
        const Inst I = inst[b];
        uint8_t* sb = sub + off[b];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.n; i += gridDim.x * blockDim.x) {
            const uint8_t f = (i + 1 < I.n && I.S[cm(i + 1, i, I.ldS)] != 0.0) ? 1 : 0;
            if (!mismatch) sb[i] = f;
            else if (f != sb[i]) atomicExch(mismatch, 2);
        }
    }
}

__global__ void eigs_batched_kernel(int count, const Inst* __restrict__ inst,
                                    const long long* __restrict__ off, double* __restrict__ wr,
                                    double* __restrict__ wi) {
    for (int b = blockIdx.y; b < count; b += gridDim.y) {
        const Inst I = inst[b];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.n; i += gridDim.x * blockDim.x)
            eig_at(I.n, I.S, I.ldS, i, &wr[off[b] + i], &wi[off[b] + i]);
    }
}

dim3 batched_grid(int count, int xblocks) {
    return dim3(xblocks < 1 ? 1 : xblocks, count < 65535 ? (count < 1 ? 1 : count) : 65535);
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

// The x dimension is sized for a few hundred positions per instance; larger
// instances are covered by the grid-stride loops.
cudaError_t launch_validate_batched(int count, const Inst* inst, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    validate_batched_kernel<<<batched_grid(count, 4), 256, 0, st>>>(count, inst);
    return cudaGetLastError();
}

cudaError_t launch_subdiag_batched(int count, const Inst* inst, const long long* off, uint8_t* sub,
                                   int* mismatch, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    subdiag_batched_kernel<<<batched_grid(count, 2), 256, 0, st>>>(count, inst, off, sub, mismatch);
    return cudaGetLastError();
}

cudaError_t launch_eigs_batched(int count, const Inst* inst, const long long* off, double* wr,
                                double* wi, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    eigs_batched_kernel<<<batched_grid(count, 2), 256, 0, st>>>(count, inst, off, wr, wi);
    return cudaGetLastError();
}

}  // namespace gbr
