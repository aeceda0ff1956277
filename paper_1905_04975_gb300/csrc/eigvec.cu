// Eigenvectors of a real Schur form (Section 2, Eq. 5) and their back-
// transformation (Eq. 6), with protection against floating-point overflow
// (the requirement of Section 3.1):
//
//   colmax_kernel   per column c of S: max |S[i, c]| over i < c and i < c - 1
//                   (the bounds the overflow guard multiplies with);
//   eigvec_kernel   one CTA per selected eigenvalue (a 1x1 block, or a 2x2
//                   block = a conjugate pair, stored as real and imaginary
//                   column): column-oriented back substitution over the
//                   diagonal blocks above it;
//   evgemm_kernel   X = Q Y with FP64 tensor-core products (DMMA); a column
//                   block of Y is nonzero only in its leading rows, so the
//                   inner dimension stops there;
//   evnorm_kernel   max |x_i| = 1 per real vector, max(|re| + |im|) = 1 per
//                   complex one.
//
// Back substitution: r = -S[0:j, B(j)] y[B(j)]; for each block B above,
// y[B] = (S[B,B] - lambda I)^-1 r[B] (one thread), then r[0:B0] -= S[0:B0, B]
// y[B] (all threads).  A pivot below smin = max(eps |lambda|, DBL_MIN / eps)
// is raised to smin.  rb bounds max|r| over the remaining rows (|z| = |re| +
// |im|); before a block is solved and before its update, the vector is
// scaled by 2^-512 (exact) while the next value or the new bound would exceed
// 2^900.  The right-hand side lives in shared memory when it fits.
#include "common.cuh"
#include "host.h"

#include <float.h>

namespace gbr {

namespace {

constexpr int EV_THREADS = 256;
constexpr double EV_BIG = 0x1p900;
constexpr double EV_SHRINK = 0x1p-512;

struct cd {
    double re, im;
};
__device__ __forceinline__ double cabs1(cd z) { return fabs(z.re) + fabs(z.im); }
__device__ __forceinline__ cd cmul(cd a, cd b) {
    return cd{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cd csub(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {  // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        const double t = b.im / b.re, d = fma(b.im, t, b.re);
        return cd{fma(a.im, t, a.re) / d, fma(-a.re, t, a.im) / d};
    }
    const double t = b.re / b.im, d = fma(b.re, t, b.im);
    return cd{fma(a.re, t, a.im) / d, fma(a.im, t, -a.re) / d};
}
__device__ __forceinline__ cd perturb(cd d, double smin) {
    const double m = cabs1(d);
    if (m >= smin) return d;
    if (m == 0.0) return cd{smin, 0.0};
    return cd{d.re * (smin / m), d.im * (smin / m)};
}

__global__ void colmax_kernel(int n, const double* __restrict__ S, int ldS, double* __restrict__ cmA,
                              double* __restrict__ cmB) {
    const int c = blockIdx.x;
    if (c >= n) return;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        const double v = fabs(__ldg(&S[cm(i, c, ldS)]));
        a = fmax(a, v);
        if (i < c - 1) b = fmax(b, v);
    }
    for (int o = 16; o; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    __shared__ double sa[32], sb[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { a = fmax(a, sa[i]); b = fmax(b, sb[i]); }
        cmA[c] = a;
        cmB[c] = b;
    }
}

// Block-wide max of v (EV_THREADS threads).
__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double m = red[0];
    for (int i = 1; i < EV_THREADS / 32; ++i) m = fmax(m, red[i]);
    return m;
}

// Inverse of the shifted diagonal block B = [b0, b0 + k), S[B,B] - lambda I,
// with a pivot (the 1x1 denominator or the 2x2 determinant) below smin
// raised to smin: inv[0..3] = row-major 2x2 (inv[0] alone for k = 1).
struct BlkInv {
    int b0, k;
    cd inv[4];
};

__device__ __forceinline__ BlkInv block_inverse(const double* __restrict__ S, int ldS, int b0,
                                                int k, double lr, double li, double smin) {
    BlkInv B;
    B.b0 = b0;
    B.k = k;
    const cd one{1.0, 0.0};
    if (k == 1) {
        const cd d = perturb(cd{__ldg(&S[cm(b0, b0, ldS)]) - lr, -li}, smin);
        B.inv[0] = cdiv(one, d);
        B.inv[1] = B.inv[2] = B.inv[3] = cd{0.0, 0.0};
        return B;
    }
    const cd m00 = cd{__ldg(&S[cm(b0, b0, ldS)]) - lr, -li};
    const cd m01 = cd{__ldg(&S[cm(b0, b0 + 1, ldS)]), 0.0};
    const cd m10 = cd{__ldg(&S[cm(b0 + 1, b0, ldS)]), 0.0};
    const cd m11 = cd{__ldg(&S[cm(b0 + 1, b0 + 1, ldS)]) - lr, -li};
    cd det = csub(cmul(m00, m11), cmul(m01, m10));
    const double mx = fmax(fmax(cabs1(m00), cabs1(m01)), fmax(cabs1(m10), cabs1(m11)));
    det = perturb(det, smin * fmax(mx, smin));
    const cd rd = cdiv(one, det);
    B.inv[0] = cmul(m11, rd);
    B.inv[1] = cmul(cd{-m01.re, -m01.im}, rd);
    B.inv[2] = cmul(cd{-m10.re, -m10.im}, rd);
    B.inv[3] = cmul(m00, rd);
    return B;
}

// x = inv r for one block; real arithmetic for real vectors.
template <bool CPLX>
__device__ __forceinline__ void apply_inv(const BlkInv& B, cd r0, cd r1, double f, cd& x0, cd& x1) {
    r0 = cd{r0.re * f, r0.im * f};
    r1 = cd{r1.re * f, r1.im * f};
    if (!CPLX) {
        x0 = cd{fma(B.inv[1].re, r1.re, B.inv[0].re * r0.re), 0.0};
        x1 = cd{fma(B.inv[3].re, r1.re, B.inv[2].re * r0.re), 0.0};
    } else {
        const cd a = cmul(B.inv[0], r0), b = cmul(B.inv[1], r1);
        const cd c = cmul(B.inv[2], r0), d = cmul(B.inv[3], r1);
        x0 = cd{a.re + b.re, a.im + b.im};
        x1 = cd{c.re + d.re, c.im + d.im};
    }
}

// The overflow guards of one block (one thread): scales by 2^-512 while the
// solution could exceed EV_BIG, then while the bound of the update of r by x
// could; returns the number of scalings, with x scaled and rb updated.
template <bool CPLX>
__device__ __forceinline__ int solve_guarded(const BlkInv& B, cd r0, cd r1, double cmx,
                                             double& rb, cd& x0, cd& x1) {
    int s = 0;
    double f = 1.0;
    apply_inv<CPLX>(B, r0, r1, 1.0, x0, x1);
    while (s < 8 && !(fmax(cabs1(x0), cabs1(x1)) <= EV_BIG)) {
        f *= EV_SHRINK;
        ++s;
        apply_inv<CPLX>(B, r0, r1, f, x0, x1);
    }
    rb *= f;
    if (B.b0 > 0) {
        double xm = fmax(cabs1(x0), cabs1(x1));
        int s2 = 0;
        while (s2 < 8 && rb + B.k * cmx * xm > EV_BIG) {
            x0 = cd{x0.re * EV_SHRINK, x0.im * EV_SHRINK};
            x1 = cd{x1.re * EV_SHRINK, x1.im * EV_SHRINK};
            rb *= EV_SHRINK;
            xm *= EV_SHRINK;
            ++s2;
        }
        rb += B.k * cmx * xm;
        s += s2;
    }
    return s;
}

// One eigenvector per CTA.  blocks[b] = (j, nb, column of Y, -); Y column-
// major (ldY), written for every row (zero below the vector's support).
// rscratch: per-CTA right-hand side and 2x2 flags in global memory (3 n
// doubles per CTA), used when rsm == 0; otherwise both are in dynamic shared
// memory.  nscale[col]: the number of 2^-512 scalings.
//
// Pipelined by one block: while warps 1..7 apply the update of block B_t to
// the rows below the next block, warp 0 applies it to the next block's rows
// and lane 0 solves the next block (its pending scaling is applied at the
// start of the following step, before anything else reads the rows).  The
// inverses of the shifted diagonal blocks are computed 32 blocks at a time
// by the lanes of warp 0 (one block per lane) into a ring, so that the
// serial step of lane 0 is a few multiplications and the guards.
template <bool CPLX>
__global__ void __launch_bounds__(EV_THREADS)
eigvec_kernel(int n, const double* __restrict__ S, int ldS, const int4* __restrict__ blocks,
              double* __restrict__ Y, int ldY, const double* __restrict__ cmA,
              const double* __restrict__ cmB, double* __restrict__ rscratch, int rsm,
              int* __restrict__ nscale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[EV_THREADS / 32];
    __shared__ cd xs[2][2];
    __shared__ int pend[2];
    __shared__ BlkInv ring[32];
    __shared__ int ring_b0[33];  // block starts of the ring's blocks (entry 32: one past)
    __shared__ int ring_first, ring_count;
    const int4 bk = blocks[blockIdx.x];
    const int j = bk.x, nb = bk.y, col = bk.z, top = j + nb;
    if ((nb == 2) != CPLX) return;  // launched per kind
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double* yr = Y + (size_t)col * ldY;
    double* yi = CPLX ? Y + (size_t)(col + 1) * ldY : nullptr;
    double* rr = rsm ? reinterpret_cast<double*>(smem_raw) : rscratch + (size_t)blockIdx.x * 3 * n;
    double* ri = rr + n;  // imaginary parts (complex vectors)
    uint8_t* sub = rsm ? smem_raw + sizeof(double) * 2 * (size_t)n
                       : reinterpret_cast<uint8_t*>(ri + n);  // 2x2 flag of rows i, i+1
    // eigenvalue and start vector
    double lr, li = 0.0, y1i = 0.0;
    if (!CPLX) {
        lr = __ldg(&S[cm(j, j, ldS)]);
    } else {
        const double a = __ldg(&S[cm(j, j, ldS)]), b = __ldg(&S[cm(j, j + 1, ldS)]);
        const double c = __ldg(&S[cm(j + 1, j, ldS)]);
        const double w = sqrt(-b * c);
        lr = a;
        li = w;
        y1i = w / b;
    }
    const double smin = fmax(DBL_EPSILON * (fabs(lr) + fabs(li)), DBL_MIN / DBL_EPSILON);
    // y rows >= j; r = -S[0:j, j:top] y[j:top]; the 2x2 pattern above j
    for (int i = j + tid; i < n; i += EV_THREADS) {
        yr[i] = (i == j) ? 1.0 : 0.0;
        if (CPLX) yi[i] = (i == j + 1) ? y1i : 0.0;
    }
    double m = 0.0;
    for (int i = tid; i < j; i += EV_THREADS) {
        const double s0 = __ldg(&S[cm(i, j, ldS)]);
        sub[i] = (i + 1 < j && __ldg(&S[cm(i + 1, i, ldS)]) != 0.0) ? 1 : 0;
        if (!CPLX) {
            rr[i] = -s0;
            m = fmax(m, fabs(s0));
        } else {
            const double s1 = __ldg(&S[cm(i, j + 1, ldS)]);
            rr[i] = -s0;
            ri[i] = -s1 * y1i;
            m = fmax(m, fabs(s0) + fabs(s1 * y1i));
        }
    }
    double rb = block_max(m, red);  // maintained by thread 0 only
    if (j == 0) {
        if (tid == 0 && nscale) {
            nscale[col] = 0;
            if (CPLX) nscale[col + 1] = 0;
        }
        return;
    }
    auto block_below = [&](int e) { return (e >= 2 && sub[e - 2]) ? e - 2 : e - 1; };
    auto colbound = [&](int b0, int k) { return (k == 1) ? cmA[b0] : fmax(cmA[b0], cmB[b0 + 1]); };
    // warp 0: the inverses of the next (up to) 32 blocks below e
    auto refill = [&](int e, int first) {
        if (lane == 0) {
            int cnt = 0, t = e;
            while (cnt < 32 && t > 0) {
                const int b = block_below(t);
                ring_b0[cnt++] = b;
                t = b;
            }
            ring_b0[cnt] = t;
            ring_count = cnt;
            ring_first = first;
        }
        __syncwarp();
        if (lane < ring_count) {
            const int b = ring_b0[lane], e2 = lane ? ring_b0[lane - 1] : e;
            ring[lane] = block_inverse(S, ldS, b, e2 - b, lr, li, smin);
        }
        __syncwarp();
    };
    int b1 = j, b0 = block_below(j);
    if (warp == 0) {
        refill(j, 0);
        if (lane == 0) {
            const BlkInv& Bi = ring[0];
            const int k = Bi.k;
            cd x0, x1;
            const int s = solve_guarded<CPLX>(
                Bi, cd{rr[b0], CPLX ? ri[b0] : 0.0},
                cd{k == 2 ? rr[b0 + 1] : 0.0, (CPLX && k == 2) ? ri[b0 + 1] : 0.0},
                b0 > 0 ? colbound(b0, k) : 0.0, rb, x0, x1);
            xs[0][0] = x0;
            xs[0][1] = x1;
            pend[0] = s;
            yr[b0] = x0.re;
            if (CPLX) yi[b0] = x0.im;
            if (k == 2) {
                yr[b0 + 1] = x1.re;
                if (CPLX) yi[b0 + 1] = x1.im;
            }
        }
    }
    __syncthreads();
    int cur = 0, step = 0, nsc = 0;
    if (tid == 0) nsc = pend[0];
    while (b0 > 0) {
        const int k = b1 - b0;
        const int s = pend[cur];
        const cd x0 = xs[cur][0], x1 = xs[cur][1];
        const int c1 = b0, c0 = block_below(b0), kn = c1 - c0;  // next block [c0, c1)
        double f = 1.0;
        if (s) {  // rare: the rows already computed move to the new scale
            for (int t = 0; t < s; ++t) f *= EV_SHRINK;
            for (int i = b1 + tid; i < top; i += EV_THREADS) {
                yr[i] *= f;
                if (CPLX) yi[i] *= f;
            }
        }
        if (warp == 0) {
            // the next block's rows: scale, update by B, then solve (lane 0)
            if (lane < kn) {
                const int i = c0 + lane;
                const double s0 = __ldg(&S[cm(i, b0, ldS)]);
                const double s1 = (k == 2) ? __ldg(&S[cm(i, b0 + 1, ldS)]) : 0.0;
                double v = s ? rr[i] * f : rr[i];
                v = fma(-s0, x0.re, v);
                if (k == 2) v = fma(-s1, x1.re, v);
                rr[i] = v;
                if (CPLX) {
                    double u = s ? ri[i] * f : ri[i];
                    u = fma(-s0, x0.im, u);
                    if (k == 2) u = fma(-s1, x1.im, u);
                    ri[i] = u;
                }
            }
            const int q = step + 1;  // index of the next block, counted from the eigenvalue
            if (q - ring_first >= ring_count) refill(c1, q);
            else __syncwarp();
            if (lane == 0) {
                const BlkInv& Bi = ring[q - ring_first];
                cd y0, y1;
                const int sn = solve_guarded<CPLX>(
                    Bi, cd{rr[c0], CPLX ? ri[c0] : 0.0},
                    cd{kn == 2 ? rr[c0 + 1] : 0.0, (CPLX && kn == 2) ? ri[c0 + 1] : 0.0},
                    c0 > 0 ? colbound(c0, kn) : 0.0, rb, y0, y1);
                xs[cur ^ 1][0] = y0;
                xs[cur ^ 1][1] = y1;
                pend[cur ^ 1] = sn;
                nsc += sn;
                yr[c0] = y0.re;
                if (CPLX) yi[c0] = y0.im;
                if (kn == 2) {
                    yr[c0 + 1] = y1.re;
                    if (CPLX) yi[c0 + 1] = y1.im;
                }
            }
        } else if (s) {
            // rows below the next block: scale, update by B
            for (int i = tid - 32; i < c0; i += EV_THREADS - 32) {
                const double s0 = __ldg(&S[cm(i, b0, ldS)]);
                const double s1 = (k == 2) ? __ldg(&S[cm(i, b0 + 1, ldS)]) : 0.0;
                double v = fma(-s0, x0.re, rr[i] * f);
                if (k == 2) v = fma(-s1, x1.re, v);
                rr[i] = v;
                if (CPLX) {
                    double u = fma(-s0, x0.im, ri[i] * f);
                    if (k == 2) u = fma(-s1, x1.im, u);
                    ri[i] = u;
                }
            }
        } else if (k == 1) {
            for (int i = tid - 32; i < c0; i += EV_THREADS - 32) {
                const double sv = __ldg(&S[cm(i, b0, ldS)]);
                rr[i] = fma(-sv, x0.re, rr[i]);
                if (CPLX) ri[i] = fma(-sv, x0.im, ri[i]);
            }
        } else {
            for (int i = tid - 32; i < c0; i += EV_THREADS - 32) {
                const double s0 = __ldg(&S[cm(i, b0, ldS)]), s1 = __ldg(&S[cm(i, b0 + 1, ldS)]);
                rr[i] = fma(-s1, x1.re, fma(-s0, x0.re, rr[i]));
                if (CPLX) ri[i] = fma(-s1, x1.im, fma(-s0, x0.im, ri[i]));
            }
        }
        __syncthreads();
        b1 = c1;
        b0 = c0;
        cur ^= 1;
        ++step;
    }
    // the last block's pending scaling: the rows already computed below it
    {
        const int s = pend[cur];
        if (s) {
            double f = 1.0;
            for (int t = 0; t < s; ++t) f *= EV_SHRINK;
            for (int i = b1 + tid; i < top; i += EV_THREADS) {
                yr[i] *= f;
                if (CPLX) yi[i] *= f;
            }
        }
    }
    if (tid == 0 && nscale) {
        nscale[col] = nsc;
        if (CPLX) nscale[col + 1] = nsc;
    }
}

// C (rows x cols) = A (rows x K) B (K x cols), column-major, K of column
// block cb limited to kmax[cb] (the vectors' support); DMMA m8n8k4.
constexpr int GM = 64, GN = 128, GK = 32;
constexpr int LDA_S = GK + 4, LDB_S = GN + 8;
constexpr size_t kGemmSmem = sizeof(double) * ((size_t)GM * LDA_S + (size_t)GK * LDB_S);

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256)
evgemm_kernel(int rows, int cols, const double* __restrict__ A, int ldA,
              const double* __restrict__ B, int ldB, double* __restrict__ C, int ldC,
              const int* __restrict__ kmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* As = reinterpret_cast<double*>(smem_raw);  // GM x LDA_S, row-major (k contiguous)
    double* Bs = As + GM * LDA_S;                       // GK x LDB_S, row-major (n contiguous)
    const int r0 = blockIdx.x * GM, c0 = blockIdx.y * GN;
    const int K = kmax[blockIdx.y];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    double acc[8][2][2];
#pragma unroll
    for (int rt = 0; rt < 8; ++rt)
#pragma unroll
        for (int ct = 0; ct < 2; ++ct) acc[rt][ct][0] = acc[rt][ct][1] = 0.0;
    for (int k0 = 0; k0 < K; k0 += GK) {
        __syncthreads();
        for (int i = tid; i < GM * GK; i += 256) {
            const int r = i % GM, k = i / GM;
            As[r * LDA_S + k] = (r0 + r < rows && k0 + k < K) ? __ldg(&A[cm(r0 + r, k0 + k, ldA)]) : 0.0;
        }
        for (int i = tid; i < GK * GN; i += 256) {
            const int k = i % GK, c = i / GK;
            Bs[k * LDB_S + c] = (c0 + c < cols && k0 + k < K) ? __ldg(&B[cm(k0 + k, c0 + c, ldB)]) : 0.0;
        }
        __syncthreads();
        const int cw = warp * 16;
#pragma unroll
        for (int kk = 0; kk < GK; kk += 4) {
            double a[8], bb[2];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt) a[rt] = As[(rt * 8 + gid) * LDA_S + kk + tig];
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) bb[ct] = Bs[(kk + tig) * LDB_S + cw + ct * 8 + gid];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt)
#pragma unroll
                for (int ct = 0; ct < 2; ++ct) dmma(acc[rt][ct][0], acc[rt][ct][1], a[rt], bb[ct]);
        }
    }
    // acc[rt][ct][v]: row rt*8 + gid, column warp*16 + ct*8 + 2*tig + v
#pragma unroll
    for (int rt = 0; rt < 8; ++rt) {
        const int r = r0 + rt * 8 + gid;
        if (r >= rows) continue;
#pragma unroll
        for (int ct = 0; ct < 2; ++ct)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int c = c0 + warp * 16 + ct * 8 + 2 * tig + v;
                if (c < cols) C[cm(r, c, ldC)] = acc[rt][ct][v];
            }
    }
}

// Normalizes the vector(s) of block b in place: X columns col (and col + 1).
__global__ void __launch_bounds__(EV_THREADS)
evnorm_kernel(int n, const int4* __restrict__ blocks, double* __restrict__ X, int ldX) {
    __shared__ double red[EV_THREADS / 32];
    const int4 bk = blocks[blockIdx.x];
    const int nb = bk.y, col = bk.z;
    double* xr = X + (size_t)col * ldX;
    double* xi = nb == 2 ? X + (size_t)(col + 1) * ldX : nullptr;
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += EV_THREADS)
        m = fmax(m, fabs(xr[i]) + (xi ? fabs(xi[i]) : 0.0));
    m = block_max(m, red);
    if (m == 0.0) return;
    for (int i = threadIdx.x; i < n; i += EV_THREADS) {
        xr[i] /= m;
        if (xi) xi[i] /= m;
    }
}

template <typename K>
cudaError_t smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Shared memory per CTA for the right-hand side of an n x n problem
// (complex: 2 n doubles); 0 if it does not fit and global scratch is used.
size_t eigvec_rhs_smem(int n) {
    const size_t b = sizeof(double) * 2 * (size_t)n + (size_t)n + 16;
    return b <= 96 * 1024 ? b : 0;
}

cudaError_t launch_colmax(int n, const double* S, int ldS, double* cmA, double* cmB,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    colmax_kernel<<<n, 128, 0, st>>>(n, S, ldS, cmA, cmB);
    return cudaGetLastError();
}

cudaError_t launch_eigvec(int n, const double* S, int ldS, const int4* d_blocks, int nblk,
                          int nreal, double* Y, int ldY, double* cmA, double* cmB,
                          double* rscratch, int* nscale, cudaStream_t st) {
    if (n == 0 || nblk == 0) return cudaSuccess;
    cudaError_t e;
    const size_t sm = eigvec_rhs_smem(n);
    e = smem_attr(eigvec_kernel<false>, sm);
    if (e != cudaSuccess) return e;
    e = smem_attr(eigvec_kernel<true>, sm);
    if (e != cudaSuccess) return e;
    // blocks are ordered real ones first (nreal of them), then the pairs
    if (nreal > 0)
        eigvec_kernel<false><<<nreal, EV_THREADS, sm, st>>>(n, S, ldS, d_blocks, Y, ldY, cmA, cmB,
                                                           rscratch, sm ? 1 : 0, nscale);
    if (nblk > nreal)
        eigvec_kernel<true><<<nblk - nreal, EV_THREADS, sm, st>>>(
            n, S, ldS, d_blocks + nreal, Y, ldY, cmA, cmB,
            rscratch ? rscratch + (size_t)nreal * 3 * n : nullptr, sm ? 1 : 0, nscale);
    return cudaGetLastError();
}

cudaError_t launch_evgemm(int rows, int cols, const double* A, int ldA, const double* B, int ldB,
                          double* C, int ldC, const int* d_kmax, cudaStream_t st) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    cudaError_t e = smem_attr(evgemm_kernel, kGemmSmem);
    if (e != cudaSuccess) return e;
    dim3 grid((rows + GM - 1) / GM, (cols + GN - 1) / GN);
    evgemm_kernel<<<grid, 256, kGemmSmem, st>>>(rows, cols, A, ldA, B, ldB, C, ldC, d_kmax);
    return cudaGetLastError();
}

int evgemm_col_block() { return GN; }

cudaError_t launch_evnorm(int n, const int4* d_blocks, int nblk, double* X, int ldX, cudaStream_t st) {
    if (n == 0 || nblk == 0) return cudaSuccess;
    evnorm_kernel<<<nblk, EV_THREADS, 0, st>>>(n, d_blocks, X, ldX);
    return cudaGetLastError();
}

}  // namespace gbr
