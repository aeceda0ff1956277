// Per-window launch of the window task (one CTA).
#include "window_body.cuh"

namespace gbr {

namespace {

__global__ void __launch_bounds__(win::WIN_THREADS, 1)
window_kernel(int n, double* __restrict__ S, int ldS, int s0, int w, uint8_t* __restrict__ gsel,
              double* __restrict__ Ug, int strong, DevCounters* __restrict__ ctr, int abort) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    win::window_body(n, S, ldS, s0, w, gsel, Ug, strong, ctr, smem_raw, nullptr,
                     abort ? &ctr->aborted : nullptr);
}

}  // namespace

size_t window_smem_bytes(int /*w*/) { return win::kWindowSmem; }

cudaError_t launch_window(int n, const Window& wd, double* S, int ldS, uint8_t* sel, double* U,
                          int strong, DevCounters* ctr, cudaStream_t st, bool abort) {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    size_t smem = window_smem_bytes(WMAX);
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    int w = wd.e - wd.s;
    window_kernel<<<1, win::WIN_THREADS, smem, st>>>(n, S, ldS, wd.s, w, sel, U, strong, ctr,
                                                     abort ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace gbr
