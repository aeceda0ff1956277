// One off-diagonal update Y <- Y U on a single panel (Section 3.2: the
// accumulated transformation of a window applied to a section of the matrix
// by a left, right or Q update task), as its own launch: FP64 DMMA tiles, or
// split-precision tiles on the tensor cores.  Used by gbr_update_panel.
#include "ozaki.cuh"
#include "update_body.cuh"
#include "window_body.cuh"

namespace gbr {

namespace {

// One BM-row tile per CTA (FP64 DMMA).
__global__ void __launch_bounds__(upd::UPD_THREADS, 1)
panel_dmma_kernel(double* __restrict__ Y, long long rs, long long ks, int rows, int w,
                  const double* __restrict__ Ug) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int r0 = blockIdx.x * upd::BM;
    upd::update_tile(Y, rs, ks, r0, min(upd::BM, rows - r0), w, Ug, true, smem_raw, nullptr);
}

// One BM-row tile per CTA (FP64 FMA register tiles), the scheduler's CTA size.
constexpr int PANEL_FMA_THREADS = 512;
__global__ void __launch_bounds__(PANEL_FMA_THREADS, 1)
panel_fma_kernel(double* __restrict__ Y, long long rs, long long ks, int rows, int w,
                 const double* __restrict__ Ug) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int r0 = blockIdx.x * upd::BM;
    upd::update_tile_fma(Y, rs, ks, r0, min(upd::BM, rows - r0), w, Ug, true, smem_raw, nullptr);
}

// U's digit slices and column exponents (the window task's writer).
__global__ void __launch_bounds__(512, 1) uslices_kernel(const double* __restrict__ Ug, int w,
                                                         unsigned char* __restrict__ us) {
    win::write_u_slices(Ug, w, us);
}

// Rows [blockIdx.x * per, ...) of the panel per CTA, split precision.
__global__ void __launch_bounds__(oz::TILE_THREADS, 1)
panel_ozaki_kernel(double* __restrict__ Y, long long rs, long long ks, int rows, int w, int per,
                   const unsigned char* __restrict__ us, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t slot;
    if ((threadIdx.x >> 5) == 0) oz::tmem_alloc(&slot, oz::TMEM_COLS);
    oz::tc_fence_before();
    __syncthreads();
    oz::tc_fence_after();
    const uint32_t tmem = slot;
    const int r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    if (r0 < r1 && !oz::update_tile_tc(Y, rs, ks, r0, r1 - r0, w, us, smem_raw, tmem) &&
        threadIdx.x == 0)
        atomicExch(err, 1);
    oz::tc_fence_before();
    __syncthreads();
    oz::tc_fence_after();
    if ((threadIdx.x >> 5) == 0) oz::tmem_dealloc(tmem, oz::TMEM_COLS);
}

template <typename K>
cudaError_t set_smem_once(K kernel, size_t bytes, bool* done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

}  // namespace

cudaError_t launch_panel_dmma(int rows, int w, double* Y, long long rs, long long ks,
                              const double* Ug, cudaStream_t st, bool fma) {
    if (fma) {
        static bool done_f[64] = {};
        cudaError_t e = set_smem_once(panel_fma_kernel, upd::kUpdateSmem, done_f);
        if (e != cudaSuccess || rows == 0) return e;
        panel_fma_kernel<<<(rows + upd::BM - 1) / upd::BM, PANEL_FMA_THREADS, upd::kUpdateSmem,
                           st>>>(Y, rs, ks, rows, w, Ug);
        return cudaGetLastError();
    }
    static bool done[64] = {};
    cudaError_t e = set_smem_once(panel_dmma_kernel, upd::kUpdateSmem, done);
    if (e != cudaSuccess || rows == 0) return e;
    panel_dmma_kernel<<<(rows + upd::BM - 1) / upd::BM, upd::UPD_THREADS, upd::kUpdateSmem, st>>>(
        Y, rs, ks, rows, w, Ug);
    return cudaGetLastError();
}

cudaError_t launch_panel_ozaki(int rows, int w, double* Y, long long rs, long long ks,
                               const double* Ug, unsigned char* us, int* err, int grid,
                               cudaStream_t st) {
    static bool done[64] = {};
    cudaError_t e = set_smem_once(panel_ozaki_kernel, oz::kSmem, done);
    if (e != cudaSuccess || rows == 0) return e;
    uslices_kernel<<<1, 512, 0, st>>>(Ug, w, us);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int per = (rows + grid - 1) / grid;
    grid = (rows + per - 1) / per;
    panel_ozaki_kernel<<<grid, oz::TILE_THREADS, oz::kSmem, st>>>(Y, rs, ks, rows, w, per, us, err);
    return cudaGetLastError();
}

}  // namespace gbr
