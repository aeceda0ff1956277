// Off-diagonal updates of one window (Section 3.2: the accumulated
// transformation U applied to "the relevant sections of the matrix" as
// level-3 operations -- the left and right update tasks):
//
//   left   S[s:e, e:n] <- U^T S[s:e, e:n]
//   right  S[0:s, s:e] <- S[0:s, s:e] U
//   Q      Q[:,  s:e]  <- Q[:,  s:e]  U
//
// All three are the same product Y <- Y U on a tall panel Y (R x w): for the
// right and Q updates Y is the column-major panel itself; for the left update
// Y is its transpose, i.e. the panel read row-major (row c of Y = column c of
// S[s:e, e:n], contiguous in memory).  One launch covers the three panels;
// each CTA owns BM whole rows of one panel, so the product is done in place.
// The contraction runs on the FP64 tensor path (DMMA, mma.sync m8n8k4 f64).
#include "common.cuh"

namespace gbr {

namespace {

constexpr int BM = 64;            // panel rows per CTA
constexpr int UPD_THREADS = 256;  // 8 warps, each owning 16 output columns
constexpr int LDY = WMAX + 4;     // padded row pitch of the Y tile in shared memory
constexpr int LDU = WMAX + 8;     // padded row pitch of U (row k holds U[k, :])

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(UPD_THREADS, 1)
update_kernel(int n, int s, int e, double* __restrict__ S, int ldS, double* __restrict__ Q,
              int ldQ, const double* __restrict__ Ug, int tL, int tR) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Us = reinterpret_cast<double*>(smem_raw);  // WMAX x LDU
    double* Ys = Us + WMAX * LDU;                        // BM x LDY

    const int w = e - s;
    const int wp = (w + 15) & ~15;  // padded to the warp column width
    const int tid = threadIdx.x;

    // which panel and which row tile
    int b = blockIdx.x;
    double* base;
    long long rs, ks;  // element (r, k) of Y at base + r*rs + k*ks
    int R;
    if (b < tL) {
        base = S + cm(s, e, ldS);  // Y(r, k) = S[s + k, e + r]
        rs = ldS; ks = 1; R = n - e;
    } else if (b < tL + tR) {
        b -= tL;
        base = S + cm(0, s, ldS);  // Y(r, k) = S[r, s + k]
        rs = 1; ks = ldS; R = s;
    } else {
        b -= tL + tR;
        base = Q + cm(0, s, ldQ);  // Y(r, k) = Q[r, s + k]
        rs = 1; ks = ldQ; R = n;
    }
    const int r0 = b * BM;
    const int rows = min(BM, R - r0);

    // U into shared memory, row-major, zero-padded to wp x wp
    for (int i = tid; i < wp * wp; i += UPD_THREADS) {
        int k = i / wp, c = i % wp;  // consecutive threads: consecutive c (strided global)
        Us[k * LDU + c] = (k < w && c < w) ? Ug[(size_t)c * w + k] : 0.0;
    }
    // Y tile, zero-padded
    if (rs == 1) {
        for (int i = tid; i < BM * wp; i += UPD_THREADS) {
            int r = i % BM, k = i / BM;
            Ys[r * LDY + k] = (r < rows && k < w) ? base[(r0 + r) + (long long)k * ks] : 0.0;
        }
    } else {
        for (int i = tid; i < BM * wp; i += UPD_THREADS) {
            int k = i % wp, r = i / wp;
            Ys[r * LDY + k] = (r < rows && k < w) ? base[(long long)(r0 + r) * rs + k] : 0.0;
        }
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int c0 = warp * 16;
    if (c0 < wp) {
        double acc[8][2][2];
#pragma unroll
        for (int rt = 0; rt < 8; ++rt)
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) acc[rt][ct][0] = acc[rt][ct][1] = 0.0;
        for (int kk = 0; kk < wp; kk += 4) {
            double a[8], bb[2];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt) a[rt] = Ys[(rt * 8 + gid) * LDY + kk + tig];
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) bb[ct] = Us[(kk + tig) * LDU + c0 + ct * 8 + gid];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt)
#pragma unroll
                for (int ct = 0; ct < 2; ++ct) dmma(acc[rt][ct][0], acc[rt][ct][1], a[rt], bb[ct]);
        }
        // write back (in place: this CTA read all of its rows before any write)
#pragma unroll
        for (int rt = 0; rt < 8; ++rt) {
            int r = rt * 8 + gid;
            if (r >= rows) continue;
#pragma unroll
            for (int ct = 0; ct < 2; ++ct)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    int k = c0 + ct * 8 + tig * 2 + v;
                    if (k < w) base[(long long)(r0 + r) * rs + (long long)k * ks] = acc[rt][ct][v];
                }
        }
    }
}

}  // namespace

size_t update_smem_bytes(int /*w*/) {
    return sizeof(double) * ((size_t)WMAX * LDU + (size_t)BM * LDY);
}

cudaError_t launch_update(int n, const Window& win, double* S, int ldS, double* Q, int ldQ,
                          const double* U, cudaStream_t st) {
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
    int tL = (n - win.e + BM - 1) / BM;
    int tR = (win.s + BM - 1) / BM;
    int tQ = Q ? (n + BM - 1) / BM : 0;
    int grid = tL + tR + tQ;
    if (grid == 0) return cudaSuccess;
    update_kernel<<<grid, UPD_THREADS, smem, st>>>(n, win.s, win.e, S, ldS, Q, ldQ, U, tL, tR);
    return cudaGetLastError();
}

}  // namespace gbr
