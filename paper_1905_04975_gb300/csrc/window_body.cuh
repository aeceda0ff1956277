// Window task: reorders the selected blocks inside one diagonal window of
// S and accumulates the window's orthogonal transformation U (Section 3.2,
// Fig. 1b; the "window task" that outputs updated tiles and an accumulator).
//
// One CTA owns one window [s, e) of width w.  For w <= WMAX the window of S
// lives in shared memory in packed upper-Hessenberg column order (column c
// keeps rows 0..c+1), U (w x w, starting at the identity) in dense column
// order.  Wider windows (up to WMAX_WIDE) do not fit there: the same packed
// window sits in a global scratch area of the CTA and U is formed in place
// in global memory, both served by the SM's L1 and L2.
//
// The swaps are organised in parallel steps instead of one at a time: in a
// step, every selected block whose upper neighbour is an unselected block
// swaps with it.  Such swaps touch disjoint index ranges, so their left
// transformations (rows) and right transformations (columns) commute and are
// applied concurrently; the result is the same stable partition as moving
// blocks one by one, reached in about w steps instead of m (w - m) swaps on
// the critical path.  A rejected swap leaves the window unchanged and marks
// the block stuck: it never moves again and later selected blocks stop below
// it.
//
// Included by the per-window launch (window.cu) and by the persistent
// scheduler (sched.cu).  Global loads go through L2 (ld.global.cg): in a
// persistent launch other CTAs write S between this CTA's tasks.
#pragma once

#include "common.cuh"
#include "ozaki.cuh"
#include "swap_math.cuh"

#include <cuda_bf16.h>
#include <float.h>

namespace gbr {
namespace win {

constexpr int WIN_THREADS = 512;
// Warps of a window task that compute the swap transforms while the others
// apply the previous step's products (a multiple of 4: the same number on
// each SM sub-partition).
constexpr int WIN_TWARPS = 4;
constexpr int MAXSW = WMAX / 2;  // at most one swap per two positions

__device__ __forceinline__ int poff(int c) { return (c * (c + 3)) >> 1; }



// Edge rows of a window that belong to a 2x2 block cut by the window
// boundary (possible only after a rejected swap made the plan stale) are
// walls: nothing swaps with them and they do not move.
constexpr uint8_t SEL_WALL = 3;

// ---------------------------------------------------------------------------
// 2|2 swap by 16 lanes.  The sequential part (Sylvester elimination with
// complete pivoting, the two reflectors) is computed redundantly by every
// lane -- an FP64 instruction costs the same for 1 or 16 lanes -- and the
// 4x4 products (Qs, Qs^T D Qs, the strong test) are lane-parallel: lane l of
// the half-warp owns entry (r, c) = (l & 3, l >> 2).  No re-standardization
// (done at the end of the window).  Returns false if the fast path cannot
// decide; the caller then runs the full transform.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sel4(int i, double a0, double a1, double a2, double a3) {
    return i == 0 ? a0 : (i == 1 ? a1 : (i == 2 ? a2 : a3));
}

// T11 X - X T22 = T12 for 2x2 blocks of D (ld 4), elimination on the 4x4
// Kronecker system with complete pivoting; registers only.
__device__ __forceinline__ bool sylv22_regs(const double* D, double* X) {
    double K[4][4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = r & 1, kk = r >> 1;
        b[r] = D[(2 + kk) * 4 + i];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int l = c & 1, mm = c >> 1;
            double v = (kk == mm) ? D[l * 4 + i] : 0.0;
            if (i == l) v -= D[(2 + kk) * 4 + 2 + mm];
            K[r][c] = v;
        }
    }
    unsigned long long kmx = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            unsigned long long a = abs_bits(K[r][c]);
            kmx = a > kmx ? a : kmx;
        }
    const double smin = fmax(DBL_EPSILON * bits_double(kmx), DBL_MIN);
    int perm = 0x3210;  // perm nibble c = original unknown now in column c
    double rp[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        unsigned long long best = 0;
        int pr = s, pc = s;
#pragma unroll
        for (int r = s; r < 4; ++r)
#pragma unroll
            for (int c = s; c < 4; ++c) {
                unsigned long long a = abs_bits(K[r][c]);
                if (a > best) { best = a; pr = r; pc = c; }
            }
#pragma unroll
        for (int r = s + 1; r < 4; ++r)
            if (pr == r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) { double t = K[s][c]; K[s][c] = K[r][c]; K[r][c] = t; }
                double t = b[s]; b[s] = b[r]; b[r] = t;
            }
#pragma unroll
        for (int c = s + 1; c < 4; ++c)
            if (pc == c) {
#pragma unroll
                for (int r = 0; r < 4; ++r) { double t = K[r][s]; K[r][s] = K[r][c]; K[r][c] = t; }
                int ns = (perm >> (4 * s)) & 15, nc = (perm >> (4 * c)) & 15;
                perm &= ~((15 << (4 * s)) | (15 << (4 * c)));
                perm |= (nc << (4 * s)) | (ns << (4 * c));
            }
        double piv = K[s][s];
        if (abs_bits(piv) < abs_bits(smin)) piv = smin;
        rp[s] = 1.0 / piv;
#pragma unroll
        for (int r = s + 1; r < 4; ++r) {
            const double f = K[r][s] * rp[s];
#pragma unroll
            for (int c = s + 1; c < 4; ++c) K[r][c] = fma(-f, K[s][c], K[r][c]);
            b[r] = fma(-f, b[s], b[r]);
        }
    }
    double y[4];
#pragma unroll
    for (int s = 3; s >= 0; --s) {
        double acc = b[s];
#pragma unroll
        for (int c = s + 1; c < 4; ++c) acc = fma(-K[s][c], y[c], acc);
        y[s] = acc * rp[s];
    }
    unsigned long long ym = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) ym = abs_bits(y[c]) > ym ? abs_bits(y[c]) : ym;
    if (!(ym < 0x7ff0000000000000ULL)) return false;  // inf or nan
    // un-permute: X[perm(c)] = y[c]   (X column-major 2x2, index i + 2k)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        double v = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (((perm >> (4 * c)) & 15) == t) v = y[c];
        X[t] = v;
    }
    return true;
}

// Returns true (and this lane's Z and Dn entries) if the fast path decided
// the swap and accepted it; *fallback is set when the full transform must run.
__device__ __forceinline__ bool swap22_halfwarp(const double* __restrict__ Sp, int ja, int l,
                                                unsigned hmask, int hbase, bool strong,
                                                double* zrc, double* dnrc, bool* fallback) {
    const int r = l & 3, c = l >> 2;
    double D[16];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
            D[cc * 4 + rr] = (rr <= cc + 1) ? Sp[poff(ja + cc) + ja + rr] : 0.0;
    *fallback = false;
    unsigned long long mx = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) mx = abs_bits(D[i]) > mx ? abs_bits(D[i]) : mx;
    const double thresh = fmax(10.0 * DBL_EPSILON * bits_double(mx), DBL_MIN);
    const unsigned long long tb = abs_bits(thresh);
    double X[4];
    if (!sylv22_regs(D, X)) { *fallback = true; return false; }
    // reflector 1 on column 0 of [-X; I]: (-x00, -x10, 1, 0)
    const double a0 = -X[0], x1 = -X[1];
    const double sig1 = fma(x1, x1, 1.0);
    const double n1 = sqrt(fma(a0, a0, sig1));
    const double be1 = a0 >= 0.0 ? -n1 : n1;
    const double d1 = a0 - be1, rd1 = 1.0 / d1;
    const double v10 = 1.0, v11 = x1 * rd1, v12 = rd1;  // v13 = 0
    const double t1 = -d1 / be1;
    // H1 applied to column 1 of [-X; I]: (-x01, -x11, 0, 1)
    const double m0 = -X[2], m1 = -X[3], m2 = 0.0, m3 = 1.0;
    const double w1 = fma(v12, m2, fma(v11, m1, v10 * m0)) * t1;
    const double q1 = fma(-w1, v11, m1), q2 = fma(-w1, v12, m2), q3 = m3;
    (void)m0;
    // reflector 2 on (q1, q2, q3)
    const double sig2 = fma(q3, q3, q2 * q2);
    double u1 = 1.0, u2 = 0.0, u3 = 0.0, t2 = 0.0;
    if (sig2 != 0.0) {
        const double n2 = sqrt(fma(q1, q1, sig2));
        const double be2 = q1 >= 0.0 ? -n2 : n2;
        const double d2 = q1 - be2, rd2 = 1.0 / d2;
        u2 = q2 * rd2;
        u3 = q3 * rd2;
        t2 = -d2 / be2;
    }
    // Qs = (I - t1 v v^T)(I - t2 u u^T), v = (1, v11, v12, 0), u = (0, 1, u2, u3)
    const double vu = fma(v12, u2, v11 * u1);
    const double vr = sel4(r, v10, v11, v12, 0.0), vc = sel4(c, v10, v11, v12, 0.0);
    const double ur = sel4(r, 0.0, u1, u2, u3), uc = sel4(c, 0.0, u1, u2, u3);
    double qs = (r == c) ? 1.0 : 0.0;
    qs = fma(-t1 * vr, vc, qs);
    qs = fma(-t2 * ur, uc, qs);
    qs = fma(t1 * t2 * vu * vr, uc, qs);
    // T = Qs^T D: T[r][c] = sum_a Qs[a][r] D[a][c]
    double dcol0 = sel4(c, D[0], D[4], D[8], D[12]), dcol1 = sel4(c, D[1], D[5], D[9], D[13]);
    double dcol2 = sel4(c, D[2], D[6], D[10], D[14]), dcol3 = sel4(c, D[3], D[7], D[11], D[15]);
    double T = 0.0;
    T = fma(__shfl_sync(hmask, qs, hbase + 0 + 4 * r), dcol0, T);
    T = fma(__shfl_sync(hmask, qs, hbase + 1 + 4 * r), dcol1, T);
    T = fma(__shfl_sync(hmask, qs, hbase + 2 + 4 * r), dcol2, T);
    T = fma(__shfl_sync(hmask, qs, hbase + 3 + 4 * r), dcol3, T);
    // Dt = T Qs: Dt[r][c] = sum_b T[r][b] Qs[b][c]
    double Dt = 0.0;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb)
        Dt = fma(__shfl_sync(hmask, T, hbase + r + 4 * bb), __shfl_sync(hmask, qs, hbase + bb + 4 * c),
                 Dt);
    // weak test on the lower-left 2x2 block
    const bool low = (r >= 2 && c < 2);
    const bool weak_bad = low && abs_bits(Dt) > tb;
    if (__any_sync(hmask, weak_bad)) { *fallback = true; return false; }
    const double Dt0 = low ? 0.0 : Dt;
    if (strong) {
        // P = Qs Dt0: P[r][b] = sum_a Qs[r][a] Dt0[a][b]
        double P = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
            P = fma(__shfl_sync(hmask, qs, hbase + r + 4 * a), __shfl_sync(hmask, Dt0, hbase + a + 4 * c),
                    P);
        // E = P Qs^T - D: E[r][c] = sum_b P[r][b] Qs[c][b] - D[r][c]
        double E = 0.0;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb)
            E = fma(__shfl_sync(hmask, P, hbase + r + 4 * bb), __shfl_sync(hmask, qs, hbase + c + 4 * bb),
                    E);
        const double drc = sel4(r, dcol0, dcol1, dcol2, dcol3);
        E -= drc;
        if (__any_sync(hmask, abs_bits(E) > tb)) { *fallback = true; return false; }
    }
    *zrc = qs;
    *dnrc = Dt0;
    return true;
}

// Swap types of a step, each handled by its own warps (FP64 issue costs the
// same for 1 or 32 active lanes, so lanes of a warp must share one code path):
//   T_11: 1x1|1x1 (Givens), T_3: 1x2 or 2x1 (k = 3), T_22: 2x2|2x2 (k = 4).
constexpr int T_11 = 0, T_3 = 1, T_22 = 2;

// Writes U's digit slices for the split-precision updates (ozaki.cuh): the
// balanced base-256 digits of every entry relative to the largest exponent of
// its column, as bf16, in the tensor cores' 128-byte-swizzled K-major layout
// [output half][K half][slice][column n mod 64][128 B] (U(k, n) is entry k of
// column n), then one int exponent per column.  Columns/rows beyond w are
// zero.
__device__ __forceinline__ void write_u_slices(const double* U, int w, unsigned char* out) {
    int* cexp = reinterpret_cast<int*>(out + OZ_UDIG_ELEMS * 2);
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    __shared__ int ce[WMAX];
    for (int n = warp; n < WMAX; n += nth / 32) {
        int em = 0;
        if (n < w)
            for (int k = lane; k < w; k += 32) {
                int e = (int)((((unsigned long long)__double_as_longlong(U[n * w + k])) >> 52) & 0x7ff);
                em = e > em ? e : em;
            }
        for (int o = 16; o; o >>= 1) {
            int v = __shfl_xor_sync(0xffffffffu, em, o);
            em = v > em ? v : em;
        }
        if (lane == 0) { ce[n] = em; cexp[n] = em; }
    }
    __syncthreads();
    // unit (column n, 16-byte chunk c of K half kh): consecutive threads fill
    // the 8 chunks of one 128-byte row, then the next column, so the global
    // writes of a warp are 512 contiguous bytes
    for (int u = tid; u < WMAX * (WMAX / 8); u += nth) {
        const int c = u & 7, n = (u >> 3) & (WMAX - 1), kh = u >> 10;
        long long G[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = 64 * kh + 8 * c + j;
            G[j] = (n < w && k < w) ? oz::oz_balanced(U[n * w + k], ce[n]) : oz::OZ_BIAS;
        }
        unsigned char* dst = out + ((size_t)((n >> 6) * 2 + kh) * OZ_SLICES * 64 + (n & 63)) * 128 +
                             (size_t)((c ^ (n & 7)) << 4);
        unsigned wv[4];
#define GBR_PUT_SLICE(P)                                                                   \
        _Pragma("unroll") for (int t = 0; t < 4; ++t) wv[t] = oz::pack_bf16x2(             \
            oz::oz_digit<P>((unsigned)G[2 * t], (unsigned)(G[2 * t] >> 32)),                 \
            oz::oz_digit<P>((unsigned)G[2 * t + 1], (unsigned)(G[2 * t + 1] >> 32)));       \
        *reinterpret_cast<uint4*>(dst + (size_t)((P) - 1) * 64 * 128) =                    \
            make_uint4(wv[0], wv[1], wv[2], wv[3]);
        GBR_PUT_SLICE(1) GBR_PUT_SLICE(2) GBR_PUT_SLICE(3) GBR_PUT_SLICE(4) GBR_PUT_SLICE(5)
        GBR_PUT_SLICE(6) GBR_PUT_SLICE(7)
#undef GBR_PUT_SLICE
    }
}

// Dynamic shared memory needed by window_body: U, the packed window, the
// transforms and swap lists of two steps, block-start and selection flags.
constexpr size_t kWindowSmem = sizeof(double) * ((size_t)WMAX * WMAX +
                                                 (size_t)((WMAX * (WMAX + 3)) / 2) +
                                                 (size_t)2 * MAXSW * 16) +
                               sizeof(int) * 2 * 3 * MAXSW + 2 * WMAX;
// A wide window task keeps only the transforms, swap lists and flags here.
constexpr size_t kWindowSmemWide = sizeof(double) * (size_t)2 * (WMAX_WIDE / 2) * 16 +
                                   sizeof(int) * 2 * 3 * (WMAX_WIDE / 2) + 2 * WMAX_WIDE;

// Row r of U, columns [j, j + K) <- (those columns) Z (the right
// transformation of one swap, applied to U).
template <int K>
__device__ __forceinline__ void right_u_row(double* __restrict__ U, int w, int j, int r,
                                            const double* __restrict__ Z) {
    double x[K], y[K];
#pragma unroll
    for (int i = 0; i < K; ++i) x[i] = U[(j + i) * w + r];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) acc = fma(x[i], Z[c * 4 + i], acc);
        y[c] = acc;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) U[(j + c) * w + r] = y[c];
}

// Left transformation of one swap on one column c of the packed window:
// rows [j, j + K) of column c <- Z^T (those rows).
template <int K>
__device__ __forceinline__ void left_col(double* __restrict__ Sp, int j, int c,
                                         const double* __restrict__ Z) {
    double x[K], y[K];
#pragma unroll
    for (int r = 0; r < K; ++r) x[r] = Sp[poff(c) + j + r];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) acc = fma(Z[r * 4 + i], x[i], acc);
        y[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < K; ++r) Sp[poff(c) + j + r] = y[r];
}

// Right transformation of one swap on one row r (< j) of the packed window:
// columns [j, j + K) of row r <- (those columns) Z.
template <int K>
__device__ __forceinline__ void right_row(double* __restrict__ Sp, int j, int r,
                                          const double* __restrict__ Z) {
    double x[K], y[K];
#pragma unroll
    for (int i = 0; i < K; ++i) x[i] = Sp[poff(j + i) + r];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) acc = fma(x[i], Z[c * 4 + i], acc);
        y[c] = acc;
    }
#pragma unroll
    for (int c = 0; c < K; ++c) Sp[poff(j + c) + r] = y[c];
}

// Last i in [0, cnt) with pre[i] <= it (pre is nondecreasing, pre[0] = 0).
__device__ __forceinline__ int prefix_slot(const int* pre, int cnt, int it) {
    int lo = 0, hi = cnt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Named barriers of the window task's two warp groups (barrier 0 is
// __syncthreads): PRODUCTS among the product warps, CRIT from the product
// warps (arrive) to the transform warps (wait).
__device__ __forceinline__ void bar_products() {
    asm volatile("bar.sync 1, %0;" ::"n"(WIN_THREADS - 32 * WIN_TWARPS) : "memory");
}
__device__ __forceinline__ void bar_crit_arrive() {
    asm volatile("bar.arrive 2, %0;" ::"n"(WIN_THREADS) : "memory");
}
__device__ __forceinline__ void bar_crit_wait() {
    asm volatile("bar.sync 2, %0;" ::"n"(WIN_THREADS) : "memory");
}

// Near-diagonal part of a step's products.  The next step's transforms read
// only diagonal blocks (entries with c - r <= 3).  A left item (swap at j,
// column c) is critical if c < j + CRIT_L, a right item of S (swap at j of
// size k, row r) if r >= j + k - CRIT_R.  Every product reaching an entry
// with c - r <= 3 is critical; no other product reaches one; and a left
// item that shares an entry with a critical right item is critical itself
// (c <= j2 + k2 - 1 <= r + 7 <= j1 + 10), so that applying all critical left
// items, then all critical right items, then the other left items and the
// other right items applies every entry's left transformation before its
// right one, as the unsplit phases do.
constexpr int CRIT_L = 11, CRIT_R = 8;

// abort_word (ABORT on rejection, else null): a window task that starts
// after it was set does nothing (U = I, *skip_out = 1); a window task that
// rejects a swap sets it, finishes the step it is in, restores the standard
// form of its 2x2 blocks and stops.  skip_out (nullable) receives 0 or 1.
//
// WM is the largest window of the instance: WMAX keeps S and U in shared
// memory; WMAX_WIDE keeps the packed S window in gsp (this CTA's global
// scratch, WIDE_SP_STRIDE doubles) and forms U in place in Ug (no split-
// precision slices).  The steps are the same; only where the two arrays live
// differs.
//
// The steps run as a two-stage pipeline over two groups of warps (blockDim
// must be WIN_THREADS): while the product warps apply step q's left and
// right transformations (to S and to U), the WIN_TWARPS transform warps,
// the same number on each SM sub-partition, compute the transforms of
// step q + 1.  Those read only the
// diagonal blocks of step q + 1, so the product warps first apply the part
// of step q that reaches near the diagonal (CRIT_L, CRIT_R), signal the
// transform warps, and then the rest; the two groups touch disjoint entries
// from there on.  Every entry receives the same operations in the same order
// as in a step-by-step execution, so the result does not change.  The state
// of a step (swap lists, transforms, prefix sums of the product work) is kept
// for two steps, by the step's parity.
template <int WM>
__device__ __forceinline__ void window_body_t(int n, double* __restrict__ S, int ldS, int s0, int w,
                                              uint8_t* __restrict__ gsel, double* __restrict__ Ug,
                                              int strong, DevCounters* __restrict__ ctr,
                                              unsigned char* smem_raw,
                                              unsigned char* __restrict__ uslices,
                                              int* abort_word, int* skip_out,
                                              double* __restrict__ gsp) {
    static_assert(WM == WMAX || WM == WMAX_WIDE, "window kernel instances");
    constexpr bool WIDE = WM > WMAX;
    constexpr int MSW = WM / 2;  // at most one swap per two positions
    constexpr int NTW = WIN_TWARPS;
    static_assert(NTW % 4 == 0 && NTW < WIN_THREADS / 32, "transform warps per sub-partition");
    constexpr int PTHREADS = WIN_THREADS - 32 * NTW;
    double* U = WIDE ? Ug : reinterpret_cast<double*>(smem_raw);        // w*w
    double* Sp = WIDE ? gsp : U + WM * WM;                               // packed window
    double* Zbuf = WIDE ? reinterpret_cast<double*>(smem_raw) : Sp + poff(WM);  // [2][MSW * 16]
    int* swbuf = reinterpret_cast<int*>(Zbuf + 2 * MSW * 16);  // [2][3][MSW]: j, k, p
    uint8_t* bst = reinterpret_cast<uint8_t*>(swbuf + 2 * 3 * MSW);
    uint8_t* sel = bst + WM;
    __shared__ int nsw, nrej, nacc;
    unsigned long long wflops = 0;   // per thread (phase D), summed at the end
    __shared__ int tcnt2[2][3];
    __shared__ int tlist2[2][3][MSW];     // slots per type (T_11, T_3, T_22: k = 2, 3, 4)
    __shared__ int kpre_l2[2][3][MSW + 1];  // prefix sums of the far left-apply columns
    __shared__ int kpre_s2[2][3][MSW + 1];  // prefix sums of the far right-apply rows of S
    __shared__ int kpre_u2[2][3][MSW + 1];  // prefix sums of the right-apply rows of U
    // Rows [urlo[c], urhi[c]] hold every nonzero of column c of U: U starts as
    // I and a swap on columns [j, j+k) mixes only those columns, so the rows
    // outside the union of their ranges stay exactly zero and are skipped.
    __shared__ short urlo[WM], urhi[WM];
    __shared__ short slo2[2][MSW], shi2[2][MSW];  // per slot: U rows its right transform touches

    const int tid = threadIdx.x;
    const int nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (abort_word) {
        __shared__ int skip;
        __syncthreads();
        if (tid == 0) skip = *reinterpret_cast<volatile int*>(abort_word) != 0;
        __syncthreads();
        if (skip) {
            // the reordering stopped before this window started: U = I
            for (int i = tid; i < w * w; i += nth) Ug[i] = ((i % w) == (i / w)) ? 1.0 : 0.0;
            if (tid == 0 && skip_out) *skip_out = 1;
            return;
        }
    }
    if (tid == 0 && skip_out) *skip_out = 0;

    // load: packed window of S, selection, U = I
    for (int c = 0; c < w; ++c) {
        int rows = min(c + 2, w);
        for (int r = tid; r < rows; r += nth)
            Sp[poff(c) + r] = __ldcg(&S[cm(s0 + r, s0 + c, ldS)]);
    }
    for (int i = tid; i < w * w; i += nth) U[i] = ((i % w) == (i / w)) ? 1.0 : 0.0;
    for (int i = tid; i < w; i += nth) {
        sel[i] = __ldcg(&gsel[s0 + i]);
        urlo[i] = (short)i;
        urhi[i] = (short)i;
    }
    __shared__ int wall_top, wall_bot;
    if (tid == 0) {
        nrej = 0;
        nacc = 0;
        wall_top = s0 > 0 && __ldcg(&S[cm(s0, s0 - 1, ldS)]) != 0.0;
        wall_bot = s0 + w < n && __ldcg(&S[cm(s0 + w, s0 + w - 1, ldS)]) != 0.0;
    }
    __syncthreads();
    if (tid == 0 && wall_top) sel[0] = SEL_WALL;
    if (tid == 0 && wall_bot) sel[w - 1] = SEL_WALL;

    // --- phase A1 of the step of parity pi (integer work only): every
    // selected block whose upper neighbour is an unselected block swaps with
    // it.  In the final pass, the 2x2 blocks whose standard form has to be
    // restored are listed instead (the fast swap paths leave it to this pass).
    auto list_swaps = [&](int pi, bool fin) {
        int* swj = swbuf + pi * 3 * MSW;
        int* swk = swj + MSW;
        int* swp = swk + MSW;
        int (*tlist)[MSW] = tlist2[pi];
        int* tcnt = tcnt2[pi];
        if (!fin) {
            for (int t = tid; t < w; t += nth) {
                if (t == 0 || !bst[t] || sel[t] != SEL_YES) continue;
                int ja = bst[t - 1] ? t - 1 : t - 2;
                if (sel[ja] != SEL_NO) continue;
                int p = t - ja;
                int q = (t + 1 < w && !bst[t + 1]) ? 2 : 1;
                int slot = atomicAdd(&nsw, 1);
                swj[slot] = ja;
                swk[slot] = p + q;
                swp[slot] = p;
                int ty = (p + q == 2) ? T_11 : (p + q == 3 ? T_3 : T_22);
                tlist[ty][atomicAdd(&tcnt[ty], 1)] = slot;
            }
        } else {
            for (int t = tid; t + 1 < w; t += nth) {
                if (!bst[t] || bst[t + 1]) continue;  // 2x2 block at t
                double m00 = Sp[poff(t) + t], m10 = Sp[poff(t) + t + 1];
                double m01 = Sp[poff(t + 1) + t], m11 = Sp[poff(t + 1) + t + 1];
                if (m00 == m11 && m01 * m10 < 0.0) continue;  // already standard
                int slot = atomicAdd(&nsw, 1);
                swj[slot] = t;
                swk[slot] = 2;
                swp[slot] = -1;   // marks a standardization rotation
                tlist[T_11][atomicAdd(&tcnt[T_11], 1)] = slot;
            }
        }
    };

    // Prefix sums of the product work of the step of parity pi, per k group,
    // by one warp: far left columns, far right rows of S, right rows of U
    // (whose range per swap, from urlo/urhi, it also records).  All listed
    // swaps are counted; a rejected one is skipped when applied.
    auto prefix_sums = [&](int pi) {
        const int* swj = swbuf + pi * 3 * MSW;
#pragma unroll 1
        for (int g = 0; g < 3; ++g) {
            const int k = g + 2, cnt = tcnt2[pi][g];
            int runl = 0, runr = 0, runu = 0;
            for (int base = 0; base < cnt; base += 32) {
                const int i = base + lane;
                int nl = 0, nr = 0, nu = 0;
                if (i < cnt) {
                    const int slot = tlist2[pi][g][i], j = swj[slot];
                    int lo = urlo[j], hi = urhi[j];
                    for (int c = 1; c < k; ++c) {
                        lo = min(lo, (int)urlo[j + c]);
                        hi = max(hi, (int)urhi[j + c]);
                    }
                    slo2[pi][slot] = (short)lo;
                    shi2[pi][slot] = (short)hi;
                    nl = max(0, w - j - CRIT_L);
                    nr = max(0, j + k - CRIT_R);
                    nu = hi - lo + 1;
                }
                int il = nl, ir = nr, iu = nu;
                for (int o = 1; o < 32; o <<= 1) {
                    int a = __shfl_up_sync(0xffffffffu, il, o);
                    int b2 = __shfl_up_sync(0xffffffffu, ir, o);
                    int c2 = __shfl_up_sync(0xffffffffu, iu, o);
                    if (lane >= o) { il += a; ir += b2; iu += c2; }
                }
                if (i < cnt) {
                    kpre_l2[pi][g][i + 1] = runl + il;
                    kpre_s2[pi][g][i + 1] = runr + ir;
                    kpre_u2[pi][g][i + 1] = runu + iu;
                }
                runl += __shfl_sync(0xffffffffu, il, 31);
                runr += __shfl_sync(0xffffffffu, ir, 31);
                runu += __shfl_sync(0xffffffffu, iu, 31);
            }
            if (lane == 0) {
                kpre_l2[pi][g][0] = 0;
                kpre_s2[pi][g][0] = 0;
                kpre_u2[pi][g][0] = 0;
            }
        }
    };

    // --- phase D of the step of parity pp with nsq swaps: move the
    // selection flags with the blocks; widen the U row ranges of the columns
    // each accepted transform mixed; a stuck 2x2 block is flagged on both of
    // its rows.  Needs the step's transforms only (not its products).
    auto phase_d = [&](int pp, int nsq) {
        const int* swj = swbuf + pp * 3 * MSW;
        const int* swk = swj + MSW;
        const int* swp = swk + MSW;
        for (int sw = tid; sw < nsq; sw += nth) {
            int j = swj[sw], k = swk[sw];
            if (k == 0) {
                sel[swp[sw]] = SEL_STUCK;
                continue;
            }
            // in-window flops of this accepted transform: k x k applied to
            // w - j - k columns (left) and j rows of S + its U rows (right)
            wflops += 2ull * k * k *
                      (unsigned long long)((w - j - k) + j + (shi2[pp][sw] - slo2[pp][sw] + 1));
            for (int c = 0; c < k; ++c) {
                urlo[j + c] = slo2[pp][sw];
                urhi[j + c] = shi2[pp][sw];
            }
            int p = swp[sw], q = k - p;
            if (p < 0) continue;   // standardization: blocks do not move
            for (int i = 0; i < q; ++i) sel[j + i] = SEL_YES;
            for (int i = q; i < k; ++i) sel[j + i] = SEL_NO;
        }
        __syncthreads();
        for (int t = tid; t + 1 < w; t += nth)
            if (sel[t] == SEL_STUCK && Sp[poff(t) + t + 1] != 0.0) sel[t + 1] = SEL_STUCK;
    };

    // --- phase A2 of the step of parity pi, by the transform warps (warps
    // 0 .. NTW - 1, NTW / 4 per sub-partition; type-uniform, since an FP64
    // issue costs the same for 1 or 32 active lanes): 2|2 swaps on
    // sub-partitions 0 and 1 (one per half-warp), k = 3 on 2, 1|1 rotations
    // on 3.
    auto transforms = [&](int pi) {
        double* Zs = Zbuf + pi * MSW * 16;
        int* swj = swbuf + pi * 3 * MSW;
        int* swk = swj + MSW;
        int* swp = swk + MSW;
        const int (*tlist)[MSW] = tlist2[pi];
        const int* tcnt = tcnt2[pi];
        const int part = warp & 3, rank = warp >> 2;
        constexpr int NRANK = NTW / 4;
        const int ty = part <= 1 ? T_22 : (part == 2 ? T_3 : T_11);
        if (ty == T_22) {
            // two 2|2 swaps per warp, one per half-warp
            const int h = lane >> 4, l = lane & 15;
            const unsigned hmask = h ? 0xffff0000u : 0x0000ffffu;
            for (int i = (rank * 2 + part) * 2 + h; i < tcnt[T_22]; i += 4 * NRANK) {
                const int slot = tlist[T_22][i];
                const int ja = swj[slot];
                double zrc = 0.0, dnrc = 0.0;
                bool fb = false;
                bool ok = swap22_halfwarp(Sp, ja, l, hmask, h * 16, strong != 0, &zrc, &dnrc, &fb);
                const int r = l & 3, c = l >> 2;
                if (ok) {
                    Zs[slot * 16 + c * 4 + r] = zrc;
                    if (r <= c + 1) Sp[poff(ja + c) + ja + r] = dnrc;
                    if (l == 0) atomicAdd(&nacc, 1);
                } else if (l == 0) {
                    double D[16], Zl[16], Dn[16];
                    for (int cc = 0; cc < 4; ++cc)
                        for (int rr = 0; rr < 4; ++rr)
                            D[cc * 4 + rr] = (rr <= cc + 1) ? Sp[poff(ja + cc) + ja + rr] : 0.0;
                    if (swap_transform(D, 2, 2, strong != 0, Zl, Dn)) {
                        for (int cc = 0; cc < 4; ++cc)
                            for (int rr = 0; rr <= min(cc + 1, 3); ++rr)
                                Sp[poff(ja + cc) + ja + rr] = Dn[cc * 4 + rr];
                        for (int e = 0; e < 16; ++e) Zs[slot * 16 + e] = Zl[e];
                        atomicAdd(&nacc, 1);
                    } else {
                        swk[slot] = 0;
                        swp[slot] = ja + 2;
                        atomicAdd(&nrej, 1);
                    }
                }
                __syncwarp(hmask);
            }
            return;
        }
        for (int i = rank * 32 + lane; i < tcnt[ty]; i += 32 * NRANK) {
            const int slot = tlist[ty][i];
            const int ja = swj[slot], p = swp[slot], k = swk[slot], q = k - p;
            double* Z = &Zs[slot * 16];
            bool ok;
            if (ty == T_11 && p < 0) {
                // restore the standard form of the 2x2 block at ja
                double m[16];
                m[0] = Sp[poff(ja) + ja];
                m[1] = Sp[poff(ja) + ja + 1];
                m[4] = Sp[poff(ja + 1) + ja];
                m[5] = Sp[poff(ja + 1) + ja + 1];
                double cs, sn;
                standardize2(m, &cs, &sn);
                Sp[poff(ja) + ja] = m[0];
                Sp[poff(ja) + ja + 1] = m[1];
                Sp[poff(ja + 1) + ja] = m[4];
                Sp[poff(ja + 1) + ja + 1] = m[5];
                Z[0] = cs; Z[1] = sn; Z[4] = -sn; Z[5] = cs;
                ok = true;
            } else if (ty == T_11) {
                // Givens rotation from (t12, t22 - t11); always accepted
                double t11 = Sp[poff(ja) + ja], t12 = Sp[poff(ja + 1) + ja];
                double t22 = Sp[poff(ja + 1) + ja + 1];
                double c = 1.0, sn = 0.0, n12 = t12;
                if (t11 != t22) {
                    double d = t22 - t11;
                    double rh = 1.0 / sqrt(fma(t12, t12, d * d));
                    c = t12 * rh;
                    sn = d * rh;
                    double r12 = fma(c, t12, sn * t22);
                    n12 = fma(r12, c, -(c * t11) * sn);
                }
                Z[0] = c; Z[1] = sn; Z[4] = -sn; Z[5] = c;
                Sp[poff(ja) + ja] = t22;
                Sp[poff(ja) + ja + 1] = 0.0;
                Sp[poff(ja + 1) + ja] = n12;
                Sp[poff(ja + 1) + ja + 1] = t11;
                ok = true;
            } else {
                double D[16], Zl[16], Dn[16];
                for (int cc = 0; cc < 3; ++cc)
                    for (int rr = 0; rr < 3; ++rr)
                        D[cc * 4 + rr] = (rr <= cc + 1) ? Sp[poff(ja + cc) + ja + rr] : 0.0;
                ok = swap3_fast(D, p, strong != 0, Zl, Dn) ||
                     swap_transform(D, p, q, strong != 0, Zl, Dn);
                if (ok) {
                    for (int cc = 0; cc < 3; ++cc)
                        for (int rr = 0; rr <= min(cc + 1, 2); ++rr)
                            Sp[poff(ja + cc) + ja + rr] = Dn[cc * 4 + rr];
                    for (int e = 0; e < 16; ++e) Z[e] = Zl[e];
                }
            }
            if (ok) {
                if (p >= 0) atomicAdd(&nacc, 1);
            } else {
                swk[slot] = 0;
                swp[slot] = ja + p;   // the stuck (selected) block
                atomicAdd(&nrej, 1);
            }
        }
    };

    // --- phases B and C of the step of parity pp, by the product warps:
    // critical left items, critical right items of S (then the transform
    // warps may start), far left items, far right items of S and the right
    // items of U.  Within each part the items are grouped by k so that the
    // lanes of a warp run the same k, and whole warps claim 32 items at a
    // time (claim counters pclaim): an FP64 instruction holds its
    // sub-partition's pipe for the same time with 1 or 32 lanes, and the
    // transform warps load some sub-partitions' pipes more than others, so
    // the warps of the less loaded sub-partitions take more items.
    // has = the step had swaps; the barriers run either way.
    __shared__ int pclaim[5][3];
    auto products = [&](int pp, bool has) {
        const double* Zs = Zbuf + pp * MSW * 16;
        const int* swj = swbuf + pp * 3 * MSW;
        const int* swk = swj + MSW;
        const int (*tlist)[MSW] = tlist2[pp];
        const int* tcnt = tcnt2[pp];
        constexpr int NCL = CRIT_L - 2, NCR = CRIT_R - 2;  // item slots per swap
        // next item of part `ph`, group g for this lane (or >= total: done)
        auto claim = [&](int ph, int g) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&pclaim[ph][g], 32);
            return __shfl_sync(0xffffffffu, base, 0) + lane;
        };
        if (has) {
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const int k = g + 2, total = tcnt[g] * NCL;
                for (int it = claim(0, g); it - lane < total; it = claim(0, g)) {
                    if (it >= total) continue;
                    const int slot = tlist[g][it / NCL];
                    if (swk[slot] == 0) continue;  // rejected
                    const int j = swj[slot], c = j + k + it % NCL;
                    if (c >= min(w, j + CRIT_L)) continue;
                    const double* Z = Zs + slot * 16;
                    if (g == 0) left_col<2>(Sp, j, c, Z);
                    else if (g == 1) left_col<3>(Sp, j, c, Z);
                    else left_col<4>(Sp, j, c, Z);
                }
            }
        }
        bar_products();
        if (has) {
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const int k = g + 2, total = tcnt[g] * NCR;
                for (int it = claim(1, g); it - lane < total; it = claim(1, g)) {
                    if (it >= total) continue;
                    const int slot = tlist[g][it / NCR];
                    if (swk[slot] == 0) continue;
                    const int j = swj[slot], r = j - 1 - it % NCR;
                    if (r < max(0, j + k - CRIT_R)) continue;
                    const double* Z = Zs + slot * 16;
                    if (g == 0) right_row<2>(Sp, j, r, Z);
                    else if (g == 1) right_row<3>(Sp, j, r, Z);
                    else right_row<4>(Sp, j, r, Z);
                }
            }
        }
        __threadfence_block();
        bar_crit_arrive();
        if (has) {
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const int cnt = tcnt[g];
                const int* pre = kpre_l2[pp][g];
                const int total = pre[cnt];
                for (int it = claim(2, g); it - lane < total; it = claim(2, g)) {
                    if (it >= total) continue;
                    const int lo = prefix_slot(pre, cnt, it);
                    const int slot = tlist[g][lo];
                    if (swk[slot] == 0) continue;
                    const int j = swj[slot], c = j + CRIT_L + (it - pre[lo]);
                    const double* Z = Zs + slot * 16;
                    if (g == 0) left_col<2>(Sp, j, c, Z);
                    else if (g == 1) left_col<3>(Sp, j, c, Z);
                    else left_col<4>(Sp, j, c, Z);
                }
            }
        }
        bar_products();
        if (has) {
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const int cnt = tcnt[g];
                const int* pre = kpre_s2[pp][g];
                const int total = pre[cnt];
                for (int it = claim(3, g); it - lane < total; it = claim(3, g)) {
                    if (it >= total) continue;
                    const int lo = prefix_slot(pre, cnt, it);
                    const int slot = tlist[g][lo];
                    if (swk[slot] == 0) continue;
                    const int j = swj[slot], r = it - pre[lo];
                    const double* Z = Zs + slot * 16;
                    if (g == 0) right_row<2>(Sp, j, r, Z);
                    else if (g == 1) right_row<3>(Sp, j, r, Z);
                    else right_row<4>(Sp, j, r, Z);
                }
            }
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                const int cnt = tcnt[g];
                const int* pre = kpre_u2[pp][g];
                const int total = pre[cnt];
                for (int it = claim(4, g); it - lane < total; it = claim(4, g)) {
                    if (it >= total) continue;
                    const int lo = prefix_slot(pre, cnt, it);
                    const int slot = tlist[g][lo];
                    if (swk[slot] == 0) continue;
                    const int j = swj[slot], r = slo2[pp][slot] + (it - pre[lo]);
                    const double* Z = Zs + slot * 16;
                    if (g == 0) right_u_row<2>(U, w, j, r, Z);
                    else if (g == 1) right_u_row<3>(U, w, j, r, Z);
                    else right_u_row<4>(U, w, j, r, Z);
                }
            }
        }
    };

    // Step pipeline.  Iteration i: the selection flags of step i - 1 move
    // (phase D), step i's swaps are listed (phase A1), then the product warps
    // apply step i - 1 while the transform warps compute step i.  Every
    // accepted swap moves a selected block up and every rejected one retires
    // a block, so the steps end within w * w; the cap only guards against a
    // logic error (reported through the counters).
    bool final_pass = false, overflow = false;
    int ns_prev = 0;
    for (int iter = 0;; ++iter) {
        const int pi = iter & 1, pp = pi ^ 1;
        if (ns_prev > 0) phase_d(pp, ns_prev);
        __syncthreads();
        if (abort_word && !final_pass && nrej > 0) {
            // ABORT: the first rejection stops the reordering; this window
            // only restores the standard form of its 2x2 blocks
            final_pass = true;
            if (tid == 0) atomicExch(abort_word, 1);
        }
        if (iter > 4 * WM * WM && !overflow) {
            if (tid == 0) atomicAdd(&ctr->step_overflow, 1);
            overflow = true;
        }
        for (int i = tid; i < w; i += nth) bst[i] = (i == 0) || (Sp[poff(i - 1) + i] == 0.0);
        if (tid < 3) tcnt2[pi][tid] = 0;
        if (tid < 15) pclaim[tid / 3][tid % 3] = 0;
        if (tid == 0) nsw = 0;
        __syncthreads();
        if (!overflow) list_swaps(pi, final_pass);
        __syncthreads();
        int ns = nsw;
        if (ns == 0 && !final_pass && !overflow) {
            // after the last swap: the pass that restores standard forms
            final_pass = true;
            __syncthreads();
            if (tid < 3) tcnt2[pi][tid] = 0;
            if (tid == 0) nsw = 0;
            __syncthreads();
            list_swaps(pi, true);
            __syncthreads();
            ns = nsw;
        }
        if (warp < NTW) {
            if (warp == NTW - 1 && ns > 0) prefix_sums(pi);
            bar_crit_wait();
            if (ns > 0) transforms(pi);
        } else {
            products(pp, ns_prev > 0);
        }
        __syncthreads();
        ns_prev = ns;
        if (ns == 0) break;
    }
    __shared__ unsigned long long wfl_sum;
    if (tid == 0) wfl_sum = 0;
    __syncthreads();
    for (int o = 16; o; o >>= 1) wflops += __shfl_xor_sync(0xffffffffu, wflops, o);
    if (lane == 0) atomicAdd(&wfl_sum, wflops);
    __syncthreads();
    wflops = wfl_sum;
    // store: window of S, selection, U
    for (int c = 0; c < w; ++c) {
        int rows = min(c + 2, w);
        for (int r = tid; r < rows; r += nth)
            S[cm(s0 + r, s0 + c, ldS)] = Sp[poff(c) + r];
    }
    for (int i = tid; i < w; i += nth)
        if (sel[i] != SEL_WALL) gsel[s0 + i] = sel[i];
    if constexpr (!WIDE) {
        for (int i = tid; i < w * w; i += nth) Ug[i] = U[i];
        if (uslices) write_u_slices(U, w, uslices);
    }
    if (tid == 0) {
        atomicAdd(&ctr->swaps, (unsigned long long)nacc);
        atomicAdd(&ctr->rejected, (unsigned long long)nrej);
        atomicAdd(&ctr->win_flops, wflops);
    }
}


// The shared-memory window task (w <= WMAX).
__device__ __forceinline__ void window_body(int n, double* __restrict__ S, int ldS, int s0, int w,
                                            uint8_t* __restrict__ gsel, double* __restrict__ Ug,
                                            int strong, DevCounters* __restrict__ ctr,
                                            unsigned char* smem_raw,
                                            unsigned char* __restrict__ uslices = nullptr,
                                            int* abort_word = nullptr, int* skip_out = nullptr) {
    window_body_t<WMAX>(n, S, ldS, s0, w, gsel, Ug, strong, ctr, smem_raw, uslices, abort_word,
                        skip_out, nullptr);
}

}  // namespace win
}  // namespace gbr
