// Per-window launch of the off-diagonal updates: one CTA per BM-row tile of
// the left, right and Q panels (update_body.cuh).
#include "update_body.cuh"

namespace gbr {

namespace {

__global__ void __launch_bounds__(upd::UPD_THREADS, 1)
update_kernel(int n, int s, int e, double* __restrict__ S, int ldS, double* __restrict__ Q,
              int ldQ, const double* __restrict__ Ug, int tL, int tR, DevCounters* ctr, int fma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = blockIdx.x;
    int panel = upd::PANEL_L;
    if (b >= tL + tR) { panel = upd::PANEL_Q; b -= tL + tR; }
    else if (b >= tL) { panel = upd::PANEL_R; b -= tL; }
    double* base;
    long long rs, ks;
    int R;
    upd::panel_geom(panel, n, s, e, S, ldS, Q, ldQ, &base, &rs, &ks, &R);
    const int r0 = b * upd::BM;
    if (fma)
        upd::update_tile_fma(base, rs, ks, r0, min(upd::BM, R - r0), e - s, Ug, true, smem_raw,
                             ctr ? &ctr->upd_issued : nullptr);
    else
        upd::update_tile(base, rs, ks, r0, min(upd::BM, R - r0), e - s, Ug, true, smem_raw,
                         ctr ? &ctr->upd_issued : nullptr);
}

}  // namespace

size_t update_smem_bytes(int /*w*/) { return upd::kUpdateSmem; }

cudaError_t launch_update(int n, const Window& wd, double* S, int ldS, double* Q, int ldQ,
                          const double* U, DevCounters* ctr, cudaStream_t st, bool fma) {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    size_t smem = update_smem_bytes(WMAX);
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    const int BM = upd::BM;
    int tL = (n - wd.e + BM - 1) / BM;
    int tR = (wd.s + BM - 1) / BM;
    int tQ = Q ? (n + BM - 1) / BM : 0;
    int grid = tL + tR + tQ;
    if (grid == 0) return cudaSuccess;
    update_kernel<<<grid, upd::UPD_THREADS, smem, st>>>(n, wd.s, wd.e, S, ldS, Q, ldQ, U, tL, tR, ctr,
                                                        fma ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace gbr
