// Window kernel: reorders the selected blocks inside one diagonal window of
// S and accumulates the window's orthogonal transformation U (Section 3.2,
// Fig. 1b; the "window task" that outputs updated tiles and an accumulator).
//
// One CTA owns one window [s, e) of width w <= WMAX.  The window of S lives
// in shared memory in packed upper-Hessenberg column order (column c keeps
// rows 0..c+1), U (w x w, starting at the identity) in dense column order.
//
// The swaps are organised in parallel steps instead of one at a time: in a
// step, every selected block whose upper neighbour is an unselected block
// swaps with it.  Such swaps touch disjoint index ranges, so their left
// transformations (rows) and right transformations (columns) commute and are
// applied concurrently; the result is the same stable partition as moving
// blocks one by one, reached in about w steps instead of m (w - m) swaps on
// the critical path.  Each swap is computed by one thread in FP64 registers:
//   * 1x1 | 1x1: a Givens rotation from (t12, t22 - t11);
//   * otherwise: the Sylvester equation T11 X - X T22 = gamma T12 (Kronecker
//     form, complete pivoting), Householder QR of [-X; gamma I], the weak and
//     strong stability tests against 10 eps max|D|, and a rotation per new
//     2x2 block that restores the standard form -- all folded into one
//     orthogonal k x k matrix Z (k = p + q <= 4).
// A rejected swap leaves the window unchanged and marks the block stuck: it
// never moves again and later selected blocks stop below it.
#include "common.cuh"
#include "swap_math.cuh"

#include <float.h>

namespace gbr {

namespace {

constexpr int WIN_THREADS = 512;
constexpr int MAXSW = WMAX / 2;  // at most one swap per two positions

__device__ __forceinline__ int poff(int c) { return (c * (c + 3)) >> 1; }

// Edge rows of a window that belong to a 2x2 block cut by the window
// boundary (possible only after a rejected swap made the plan stale) are
// walls: nothing swaps with them and they do not move.
constexpr uint8_t SEL_WALL = 3;

__global__ void __launch_bounds__(WIN_THREADS, 1)
window_kernel(int n, double* __restrict__ S, int ldS, int s0, int w, uint8_t* __restrict__ gsel,
              double* __restrict__ Ug, int strong, DevCounters* __restrict__ ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* U = reinterpret_cast<double*>(smem_raw);           // w*w
    double* Sp = U + WMAX * WMAX;                               // packed window
    double* Zs = Sp + poff(WMAX);                               // MAXSW * 16
    int* swj = reinterpret_cast<int*>(Zs + MAXSW * 16);
    int* swk = swj + MAXSW;
    int* swp = swk + MAXSW;
    uint8_t* bst = reinterpret_cast<uint8_t*>(swp + MAXSW);
    uint8_t* sel = bst + WMAX;
    __shared__ int nsw, nrej, nacc;

    const int tid = threadIdx.x;
    const int nth = blockDim.x;

    // load: packed window of S, selection, U = I
    for (int c = 0; c < w; ++c) {
        int rows = min(c + 2, w);
        for (int r = tid; r < rows; r += nth)
            Sp[poff(c) + r] = S[cm(s0 + r, s0 + c, ldS)];
    }
    for (int i = tid; i < w * w; i += nth) U[i] = ((i % w) == (i / w)) ? 1.0 : 0.0;
    for (int i = tid; i < w; i += nth) sel[i] = gsel[s0 + i];
    __shared__ int wall_top, wall_bot;
    if (tid == 0) {
        nrej = 0;
        nacc = 0;
        wall_top = s0 > 0 && S[cm(s0, s0 - 1, ldS)] != 0.0;
        wall_bot = s0 + w < n && S[cm(s0 + w, s0 + w - 1, ldS)] != 0.0;
    }
    __syncthreads();
    if (tid == 0 && wall_top) sel[0] = SEL_WALL;
    if (tid == 0 && wall_bot) sel[w - 1] = SEL_WALL;

    // Every accepted swap moves a selected block up and every rejected one
    // retires a block, so the loop ends within w * w steps; the cap only
    // guards against a logic error (reported through the counters).
    for (int iter = 0;; ++iter) {
        __syncthreads();
        if (iter > 4 * WMAX * WMAX) {
            if (tid == 0) atomicAdd(&ctr->step_overflow, 1);
            break;
        }
        for (int i = tid; i < w; i += nth)
            bst[i] = (i == 0) || (Sp[poff(i - 1) + i] == 0.0);
        if (tid == 0) nsw = 0;
        __syncthreads();
        // --- phase A: find and compute the swaps of this step
        for (int t = tid; t < w; t += nth) {
            if (t == 0 || !bst[t] || sel[t] != SEL_YES) continue;
            int ja = bst[t - 1] ? t - 1 : t - 2;
            if (sel[ja] != SEL_NO) continue;
            int p = t - ja;
            int q = (t + 1 < w && !bst[t + 1]) ? 2 : 1;
            int k = p + q;
            double D[16], Z[16], Dn[16];
            for (int c = 0; c < k; ++c)
                for (int r = 0; r < k; ++r)
                    D[c * 4 + r] = (r <= c + 1) ? Sp[poff(ja + c) + ja + r] : 0.0;
            int idx = atomicAdd(&nsw, 1);
            bool ok = swap_transform(D, p, q, strong != 0, Z, Dn);
            if (ok) {
                for (int c = 0; c < k; ++c)
                    for (int r = 0; r <= min(c + 1, k - 1); ++r)
                        Sp[poff(ja + c) + ja + r] = Dn[c * 4 + r];
                for (int i = 0; i < 16; ++i) Zs[idx * 16 + i] = Z[i];
                swj[idx] = ja; swk[idx] = k; swp[idx] = p;
                atomicAdd(&nacc, 1);
            } else {
                swj[idx] = ja; swk[idx] = 0; swp[idx] = t;   // swp carries the stuck block
                atomicAdd(&nrej, 1);
            }
        }
        __syncthreads();
        const int ns = nsw;
        if (ns == 0) break;
        // --- phase B: left transformations, rows [j, j+k), columns [j+k, w)
        for (int it = tid; it < ns * WMAX; it += nth) {
            int sw = it / WMAX, c = it % WMAX;
            int j = swj[sw], k = swk[sw];
            if (k == 0 || c < j + k || c >= w) continue;
            const double* Z = &Zs[sw * 16];
            double x[4], y[4];
            for (int r = 0; r < k; ++r) x[r] = Sp[poff(c) + j + r];
            for (int r = 0; r < k; ++r) {
                double acc = 0.0;
                for (int i = 0; i < k; ++i) acc = fma(Z[r * 4 + i], x[i], acc);
                y[r] = acc;
            }
            for (int r = 0; r < k; ++r) Sp[poff(c) + j + r] = y[r];
        }
        __syncthreads();
        // --- phase C: right transformations, columns [j, j+k) of S rows [0, j) and of U
        for (int it = tid; it < 2 * ns * WMAX; it += nth) {
            int half = it / (ns * WMAX);
            int rem = it - half * ns * WMAX;
            int sw = rem / WMAX, r = rem % WMAX;
            int j = swj[sw], k = swk[sw];
            if (k == 0) continue;
            const double* Z = &Zs[sw * 16];
            double x[4], y[4];
            if (half == 0) {
                if (r >= j) continue;
                for (int i = 0; i < k; ++i) x[i] = Sp[poff(j + i) + r];
            } else {
                if (r >= w) continue;
                for (int i = 0; i < k; ++i) x[i] = U[(j + i) * w + r];
            }
            for (int c = 0; c < k; ++c) {
                double acc = 0.0;
                for (int i = 0; i < k; ++i) acc = fma(x[i], Z[c * 4 + i], acc);
                y[c] = acc;
            }
            if (half == 0)
                for (int c = 0; c < k; ++c) Sp[poff(j + c) + r] = y[c];
            else
                for (int c = 0; c < k; ++c) U[(j + c) * w + r] = y[c];
        }
        __syncthreads();
        // --- phase D: move the selection flags with the blocks
        for (int sw = tid; sw < ns; sw += nth) {
            int j = swj[sw], k = swk[sw];
            if (k == 0) {
                sel[swp[sw]] = SEL_STUCK;
                continue;
            }
            int p = swp[sw], q = k - p;
            for (int i = 0; i < q; ++i) sel[j + i] = SEL_YES;
            for (int i = q; i < k; ++i) sel[j + i] = SEL_NO;
        }
        // a stuck 2x2 block is flagged on both of its rows
        __syncthreads();
        for (int t = tid; t + 1 < w; t += nth)
            if (sel[t] == SEL_STUCK && Sp[poff(t) + t + 1] != 0.0) sel[t + 1] = SEL_STUCK;
    }
    __syncthreads();
    // store: window of S, selection, U
    for (int c = 0; c < w; ++c) {
        int rows = min(c + 2, w);
        for (int r = tid; r < rows; r += nth)
            S[cm(s0 + r, s0 + c, ldS)] = Sp[poff(c) + r];
    }
    for (int i = tid; i < w; i += nth)
        if (sel[i] != SEL_WALL) gsel[s0 + i] = sel[i];
    for (int i = tid; i < w * w; i += nth) Ug[i] = U[i];
    if (tid == 0) {
        atomicAdd(&ctr->swaps, (unsigned long long)nacc);
        atomicAdd(&ctr->rejected, (unsigned long long)nrej);
    }
}

}  // namespace

size_t window_smem_bytes(int /*w*/) {
    return sizeof(double) * ((size_t)WMAX * WMAX + (size_t)((WMAX * (WMAX + 3)) / 2) +
                             (size_t)MAXSW * 16) +
           sizeof(int) * 3 * MAXSW + 2 * WMAX;
}

cudaError_t launch_window(int n, const Window& win, double* S, int ldS, uint8_t* sel, double* U,
                          int strong, DevCounters* ctr, cudaStream_t st) {
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
    int w = win.e - win.s;
    window_kernel<<<1, WIN_THREADS, smem, st>>>(n, S, ldS, win.s, w, sel, U, strong, ctr);
    return cudaGetLastError();
}

}  // namespace gbr
