// Bulge-chasing sweep of the Schur reduction (Section 3.2, "Bulge Chasing
// and Eigenvalue Reordering"): one pipelined QR iteration on an upper
// Hessenberg matrix H, bulges chased down the diagonal by overlapping 3x3
// Householder reflectors, organised as the same window tasks and
// left / right / Q update tiles as the reordering (Fig. 1b, Fig. 2).
//
// Bulges come in chains of nb (one per pair of shifts).  At chain step tau,
// bulge j of a chain (j = 0 introduced first) sits at k_j = tau - 3 j - 1:
//   k = -1       introduction: the reflector maps the three nonzeros of the
//                first column of (H - sigma1 I)(H - sigma2 I),
//                x = (h00^2 + h01 h10 - s h00 + p, h10 (h00 + h11 - s),
//                h10 h21), onto beta e_0 (s = sigma1 + sigma2,
//                p = sigma1 sigma2), on rows / columns 0..2;
//   0..n-3       chase: the reflector maps H[k+1..k+3, k] (two entries at
//                k = n-3) onto beta e_0, on rows / columns k+1..k+3; the
//                annihilated entries become exact zeros.
// Within a step the reflectors of different bulges read columns no other
// reflector of the step writes, and touch disjoint rows (left) and disjoint
// columns (right), so a step is: all reflectors, then all left products,
// then all right products -- the same result as applying them one by one
// from the lowest bulge up.
//
// A window task owns rows / columns [s, s + w) and runs the chain steps
// [t0, t1) that keep every active bulge's rows k+1..k+4 inside the window
// (the planner's guarantee), accumulating U (w x w): the rows of H to the
// right of the window and above it, and Q, get U through the update tiles.
#pragma once

#include "common.cuh"

#include <float.h>

namespace gbr {
namespace swp {

constexpr int SW = 96;                 // largest sweep window
constexpr int SWEEP_THREADS = 512;
constexpr int MAXB = SW / 3;           // bulges a window can hold

// Shared memory of sweep_body: the dense window of H and U (SW x SW each),
// per bulge its reflector (v1, v2, tau, beta, first row, length).
constexpr size_t kSweepSmem = sizeof(double) * (2 * (size_t)SW * SW + (size_t)MAXB * 4) +
                              sizeof(int) * 2 * MAXB;

// Reflector I - tau v v^T, v = (1, v1, v2), mapping x (length len = 2 or 3)
// onto beta e_0; tau = 0 when x is a multiple of e_0.
__device__ __forceinline__ void refl3(int len, double x0, double x1, double x2, double* v1,
                                      double* v2, double* tau, double* beta) {
    if (len < 3) x2 = 0.0;
    const double sigma = fma(x1, x1, x2 * x2);
    if (sigma == 0.0) {
        *v1 = 0.0;
        *v2 = 0.0;
        *tau = 0.0;
        *beta = x0;
        return;
    }
    const double nrm = sqrt(fma(x0, x0, sigma));
    const double b = x0 >= 0.0 ? -nrm : nrm;
    const double inv = 1.0 / (x0 - b);
    *v1 = x1 * inv;
    *v2 = x2 * inv;
    *tau = (b - x0) / b;
    *beta = b;
}

// One window task of a sweep.  H: the whole matrix (n x n, ldH); the
// window is [s0, s0 + w); chain steps [t0, t1); nb bulges whose shift
// parameters (s, p) are sp[2 b], sp[2 b + 1]; U (w x w, column-major, ld w)
// is written to Ug.
__device__ __forceinline__ void sweep_body(int n, double* __restrict__ H, int ldH, int s0, int w,
                                           int t0, int t1, int nb, const double* __restrict__ sp,
                                           double* __restrict__ Ug, DevCounters* __restrict__ ctr,
                                           unsigned char* smem_raw) {
    double* Hs = reinterpret_cast<double*>(smem_raw);   // w x w, ld w
    double* Us = Hs + SW * SW;                          // w x w, ld w
    double* R = Us + SW * SW;                           // per bulge: v1, v2, tau, beta
    int* rk = reinterpret_cast<int*>(R + MAXB * 4);     // per bulge: local k (or -1: intro)
    int* rl = rk + MAXB;                                // per bulge: length (0: inactive)
    __shared__ int lo_b;                                // active bulges of the step
    __shared__ int pre_l[MAXB + 1], pre_r[MAXB + 1];
    __shared__ short urlo[SW], urhi[SW];                // nonzero rows of each column of U
    const int tid = threadIdx.x, nth = blockDim.x;
    unsigned long long wflops = 0;

    for (int i = tid; i < w * w; i += nth) {
        const int r = i % w, c = i / w;
        Hs[i] = (r <= c + 4) ? __ldcg(&H[cm(s0 + r, s0 + c, ldH)]) : 0.0;
        Us[i] = (r == c) ? 1.0 : 0.0;
    }
    for (int i = tid; i < w; i += nth) {
        urlo[i] = (short)i;
        urhi[i] = (short)i;
    }
    __syncthreads();
    // Per chase step three barriers: warp 0 (which owns every bulge: at most
    // 32) first records the previous step's U row ranges, finds the active
    // bulges, computes their reflectors and the prefix sums of the work
    // items; then all threads apply the left products, then the right ones.
    // Lane i of warp 0 keeps bulge i's columns and U rows across the step.
    const int lane = tid & 31, warp = tid >> 5;
    int my_c1 = 0, my_len = 0, my_lo = 0, my_cnt = 0;   // warp 0: last step's bulge
    for (int tau = t0; tau < t1; ++tau) {
        if (warp == 0) {
            if (my_len) {
                for (int c = 0; c < my_len; ++c) {
                    urlo[my_c1 + c] = (short)my_lo;
                    urhi[my_c1 + c] = (short)(my_lo + my_cnt - 1);
                }
                my_len = 0;
            }
            __syncwarp();
            // active bulges: -1 <= k_j <= n - 3, k_j = tau - 3 j - 1 (global)
            int jlo = 0, jhi = nb - 1;
            while (jlo <= jhi && tau - 3 * jlo - 1 > n - 3) ++jlo;
            while (jhi >= jlo && tau - 3 * jhi - 1 < -1) --jhi;
            const int na = jhi - jlo + 1;
            int il = 0, ir = 0;
            if (lane < na) {
                const int j = jlo + lane;
                const int kg = tau - 3 * j - 1;
                double x0, x1, x2;
                int len = 3, kl;
                if (kg < 0) {
                    // introduction (the window starts at row 0)
                    const double h00 = Hs[0], h10 = Hs[1], h01 = Hs[w], h11 = Hs[w + 1];
                    const double h21 = Hs[w + 2];
                    const double ss = sp[2 * j], pp = sp[2 * j + 1];
                    x0 = fma(h00, h00, fma(h01, h10, fma(-ss, h00, pp)));
                    x1 = h10 * (h00 + h11 - ss);
                    x2 = h10 * h21;
                    kl = -1;
                } else {
                    kl = kg - s0;
                    len = (kg + 3 <= n - 1) ? 3 : 2;
                    x0 = Hs[kl * w + kl + 1];
                    x1 = Hs[kl * w + kl + 2];
                    x2 = (len == 3) ? Hs[kl * w + kl + 3] : 0.0;
                }
                double v1, v2, tu, be;
                refl3(len, x0, x1, x2, &v1, &v2, &tu, &be);
                R[lane * 4 + 0] = v1;
                R[lane * 4 + 1] = v2;
                R[lane * 4 + 2] = tu;
                R[lane * 4 + 3] = be;
                rk[lane] = kl;
                // item counts: left = columns [max(k, 0), w); right = rows
                // [0, min(k + 5, w)) of H plus the rows [lo, hi] of U holding
                // the nonzeros of the reflector's columns
                const int c1 = kl + 1;
                int lo = urlo[c1], hi = urhi[c1];
                for (int c = 1; c < len; ++c) {
                    lo = min(lo, (int)urlo[c1 + c]);
                    hi = max(hi, (int)urhi[c1 + c]);
                }
                il = w - (kl < 0 ? 0 : kl);
                ir = min(kl + 5, w) + (hi - lo + 1);
                // length, first U row and U row count packed into one word
                rl[lane] = len | (lo << 8) | ((hi - lo + 1) << 20);
                my_c1 = c1;
                my_len = len;
                my_lo = lo;
                my_cnt = hi - lo + 1;
                // 4 len flops per updated vector (dot + axpy): the left
                // columns but the input one, the right rows of H and of U
                const int nl = w - (kl < 0 ? 0 : kl) - (kl < 0 ? 0 : 1);
                wflops += 4ull * len * (unsigned long long)(nl + min(kl + 5, w) + my_cnt);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int a2 = __shfl_up_sync(0xffffffffu, il, o);
                const int b2 = __shfl_up_sync(0xffffffffu, ir, o);
                if (lane >= o) { il += a2; ir += b2; }
            }
            if (lane < na) { pre_l[lane + 1] = il; pre_r[lane + 1] = ir; }
            if (lane == 0) {
                pre_l[0] = 0;
                pre_r[0] = 0;
                lo_b = na;
            }
        }
        __syncthreads();
        const int na = lo_b;
        // left: rows k+1 .. k+len of the window, columns [max(k,0), w); the
        // input column gets beta and exact zeros
        {
            const int total = na > 0 ? pre_l[na] : 0;
            for (int it = tid; it < total; it += nth) {
                int lo = 0, hi = na - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre_l[mid] <= it) lo = mid; else hi = mid - 1;
                }
                const int kl = rk[lo], len = rl[lo] & 0xff, r0 = kl + 1;
                const int c = (kl < 0 ? 0 : kl) + (it - pre_l[lo]);
                const double v1 = R[lo * 4 + 0], v2 = R[lo * 4 + 1], tu = R[lo * 4 + 2];
                double* col = Hs + c * w + r0;
                if (c == kl) {
                    col[0] = R[lo * 4 + 3];
                    col[1] = 0.0;
                    if (len == 3) col[2] = 0.0;
                    continue;
                }
                const double y0 = col[0], y1 = col[1], y2 = (len == 3) ? col[2] : 0.0;
                const double d = tu * fma(v2, y2, fma(v1, y1, y0));
                col[0] = y0 - d;
                col[1] = fma(-d, v1, y1);
                if (len == 3) col[2] = fma(-d, v2, y2);
            }
        }
        __syncthreads();
        // right: columns k+1 .. k+len of rows [0, min(k+5, w)) of the window
        // and of rows [lo, hi] of U
        {
            const int total = na > 0 ? pre_r[na] : 0;
            for (int it = tid; it < total; it += nth) {
                int lo = 0, hi = na - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre_r[mid] <= it) lo = mid; else hi = mid - 1;
                }
                const int kl = rk[lo], pk = rl[lo], len = pk & 0xff, c1 = kl + 1;
                const int nh = min(kl + 5, w), rr = it - pre_r[lo];
                const double v1 = R[lo * 4 + 0], v2 = R[lo * 4 + 1], tu = R[lo * 4 + 2];
                double* base;
                int r;
                if (rr < nh) {
                    base = Hs;
                    r = rr;
                } else {
                    base = Us;
                    r = ((pk >> 8) & 0xfff) + (rr - nh);
                }
                double* p0 = base + c1 * w + r;
                const double y0 = p0[0], y1 = p0[w], y2 = (len == 3) ? p0[2 * w] : 0.0;
                const double d = tu * fma(v2, y2, fma(v1, y1, y0));
                p0[0] = y0 - d;
                p0[w] = fma(-d, v1, y1);
                if (len == 3) p0[2 * w] = fma(-d, v2, y2);
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < w * w; i += nth) {
        const int r = i % w, c = i / w;
        if (r <= c + 4) H[cm(s0 + r, s0 + c, ldH)] = Hs[i];
        Ug[i] = Us[i];
    }
    if (wflops) atomicAdd(&ctr->win_flops, wflops);
}

}  // namespace swp
}  // namespace gbr
