// Generalized reordering: the swap of two adjacent diagonal blocks of a
// matrix pair in generalized real Schur form, and the window task that
// reorders the selected blocks inside one diagonal window of (S, T) while
// accumulating the two orthogonal factors (Section 2, Eq. 7, second form:
// (S, T) = Q3 (S_hat, T_hat) Z3^T; Section 3.2 for the window structure).
//
// Swap of the p x p block (A11, B11) above the q x q block (A22, B22) of the
// k x k pair (A, B) (the paper leaves the method to the cited works; this is
// the direct method by a generalized Sylvester solve):
//   A11 R - L A22 = -gamma A12,  B11 R - L B22 = -gamma B12
// gives (A, B) [R; gamma I] = [L; gamma I] (A22, B22), so the orthogonal
// factors Qs, Zs of Householder QR factorizations of [L; gamma I] and
// [R; gamma I] make Qs^T (A, B) Zs block upper triangular with (A22, B22)'s
// eigenvalues first.  Weak test: the lower-left block of Qs^T A Zs (and of
// the B product) is at most 20 eps ||A||_F (||B||_F); strong test: the
// backward error of the result after zeroing it is within the same bound.
// Each new 2x2 diagonal block of T is then made upper triangular by a
// rotation of its two columns (folded into Zs).  Two 1x1 blocks with equal
// generalized eigenvalues (a11 b22 == a22 b11) are in order already.
//
// The window task mirrors the standard-form one (window_body.cuh): every
// selected block whose upper neighbour is unselected swaps with it in the
// same step (one thread computes one swap), then the left transformations
// (rows of S and T) and the right ones (columns of S and T, the columns of
// the accumulators UQ and UZ) are applied by all threads.
#pragma once

#include "common.cuh"

#include <float.h>

namespace gbr {
namespace gen {

constexpr int GW = 64;                 // largest generalized window
constexpr int GEN_THREADS = 512;
constexpr int GMAXSW = GW / 2;         // at most one swap per two positions
constexpr uint8_t GSEL_WALL = 3;       // window edge row of a 2x2 block cut by the edge

__host__ __device__ constexpr int gpoff(int c) { return (c * (c + 3)) / 2; }

// Shared memory of window_gen_body: UQ, UZ (GW x GW each), packed windows
// of S and T (column c keeps rows 0..c+1), Qs and Zs per swap slot.
constexpr size_t kGenWindowSmem =
    sizeof(double) * (2 * (size_t)GW * GW + 2 * (size_t)gpoff(GW) + (size_t)GMAXSW * 32) +
    sizeof(int) * 3 * GMAXSW + 2 * GW;

// |x| order through the bit pattern: for non-negative doubles the integer
// order of the bits is the numeric order (integer compares, no FP64 issue).
__device__ __forceinline__ unsigned long long mag(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Reflector (I - tau v v^T) on 4-vectors mapping x onto beta e_0, v[0] = 1;
// tau = 0 when x is a multiple of e_0 already.
__device__ __forceinline__ void house4(const double x[4], double v[4], double* tau) {
    const double sigma = x[1] * x[1] + x[2] * x[2] + x[3] * x[3];
    v[0] = 1.0;
    v[1] = x[1];
    v[2] = x[2];
    v[3] = x[3];
    *tau = 0.0;
    if (sigma != 0.0) {
        const double nrm = sqrt(x[0] * x[0] + sigma);
        const double beta = x[0] >= 0.0 ? -nrm : nrm;
        const double inv = 1.0 / (x[0] - beta);
        v[1] *= inv;
        v[2] *= inv;
        v[3] *= inv;
        *tau = (beta - x[0]) / beta;
    }
}

// Orthogonal factor Qo (4 x 4, column-major, identity beyond k) of the QR
// factorization of the k x q matrix [X; gamma I], X p x q (column-major,
// ld p): reflector H1 for column 0 on rows 0..3 (rows >= k are zero), H2 for
// column 1 on rows 1..3 when q == 2; Qo = H1 diag(1, H2).
__device__ __forceinline__ void qr_orth(int p, int q, const double* X, double gamma, double Qo[16]) {
    double M0[4], M1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        M0[i] = i < p ? X[i] : (i == p ? gamma : 0.0);
        M1[i] = (q == 2) ? (i < p ? X[i + p] : (i == p + 1 ? gamma : 0.0)) : 0.0;
    }
    double v1[4], v2[4], t1, t2 = 0.0;
    house4(M0, v1, &t1);
    v2[0] = 1.0; v2[1] = v2[2] = v2[3] = 0.0;
    if (q == 2) {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) d = fma(v1[i], M1[i], d);
        d *= t1;
        double x2[4];
#pragma unroll
        for (int i = 1; i < 4; ++i) x2[i - 1] = fma(-d, v1[i], M1[i]);
        x2[3] = 0.0;
        house4(x2, v2, &t2);
    }
    // H1 explicitly, then the right product with diag(1, H2) on columns 1..3
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) Qo[c * 4 + r] = (r == c ? 1.0 : 0.0) - t1 * v1[r] * v1[c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) d = fma(Qo[(i + 1) * 4 + r], v2[i], d);
        d *= t2;
#pragma unroll
        for (int i = 0; i < 3; ++i) Qo[(i + 1) * 4 + r] = fma(-d, v2[i], Qo[(i + 1) * 4 + r]);
    }
}

// Generalized Sylvester solve (see the file comment) on the Kronecker
// system of N = 2pq unknowns x = [vec R; vec L]; Gaussian elimination with
// complete pivoting, pivots below max(eps max|K|, DBL_MIN) raised to that
// value, and gamma <= 1 scaling the right-hand side so that no division in
// the back substitution overflows.  DA, DB: k x k (ld 4).  R, L: p x q
// (column-major, ld p).  Returns gamma.
__device__ __forceinline__ double gen_sylvester(int p, int q, const double* DA, const double* DB,
                                                double* R, double* L) {
    const int pq = p * q, N = 2 * pq;
    double K[64], b[8], y[8];
    int perm[8];
    for (int i = 0; i < 64; ++i) K[i] = 0.0;
    for (int e = 0; e < 2; ++e) {
        const double* D = e ? DB : DA;
        for (int c = 0; c < q; ++c)
            for (int i = 0; i < p; ++i) {
                const int row = e * pq + i + p * c;
                b[row] = -D[(p + c) * 4 + i];
                for (int l = 0; l < p; ++l) K[row * 8 + l + p * c] += D[l * 4 + i];
                for (int m = 0; m < q; ++m) K[row * 8 + pq + i + p * m] -= D[(p + c) * 4 + p + m];
            }
    }
    unsigned long long km = 0;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) km = max(km, mag(K[r * 8 + c]));
    double smin = DBL_EPSILON * __longlong_as_double((long long)km);
    smin = smin < DBL_MIN ? DBL_MIN : smin;
    for (int c = 0; c < N; ++c) perm[c] = c;
    for (int s = 0; s < N; ++s) {
        int pr = s, pc = s;
        unsigned long long best = 0;
        bool any = false;
        for (int r = s; r < N; ++r)
            for (int c = s; c < N; ++c) {
                const unsigned long long v = mag(K[r * 8 + c]);
                if (!any || v > best) { best = v; pr = r; pc = c; any = true; }
            }
        if (pr != s) {
            for (int c = 0; c < N; ++c) {
                const double t = K[s * 8 + c];
                K[s * 8 + c] = K[pr * 8 + c];
                K[pr * 8 + c] = t;
            }
            const double t = b[s]; b[s] = b[pr]; b[pr] = t;
        }
        if (pc != s) {
            for (int r = 0; r < N; ++r) {
                const double t = K[r * 8 + s];
                K[r * 8 + s] = K[r * 8 + pc];
                K[r * 8 + pc] = t;
            }
            const int t = perm[s]; perm[s] = perm[pc]; perm[pc] = t;
        }
        if (fabs(K[s * 8 + s]) < smin) K[s * 8 + s] = smin;
        const double piv = K[s * 8 + s];
        for (int r = s + 1; r < N; ++r) {
            const double f = K[r * 8 + s] / piv;
            K[r * 8 + s] = 0.0;
            for (int c = s + 1; c < N; ++c) K[r * 8 + c] = fma(-f, K[s * 8 + c], K[r * 8 + c]);
            b[r] = fma(-f, b[s], b[r]);
        }
    }
    double g = 1.0;
    const double big = DBL_MAX / 4.0;
    for (int s = N - 1; s >= 0; --s) {
        double acc = b[s];
        for (int c = s + 1; c < N; ++c) acc = fma(-K[s * 8 + c], y[c], acc);
        const double pv = fabs(K[s * 8 + s]);
        if (pv < 1.0 && fabs(acc) > big * pv) {
            const double f = (big * pv) / fabs(acc);
            for (int c = 0; c < N; ++c) b[c] *= f;
            for (int c = s + 1; c < N; ++c) y[c] *= f;
            acc *= f;
            g *= f;
        }
        y[s] = acc / K[s * 8 + s];
    }
    for (int c = 0; c < N; ++c) {
        const int u = perm[c];
        if (u < pq) R[u] = y[c];
        else L[u - pq] = y[c];
    }
    return g;
}

// C = X^T Y and C = X Y (4 x 4, column-major).
__device__ __forceinline__ void mm_tn(const double* X, const double* Y, double* C) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double s = 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) s = fma(X[r * 4 + t], Y[c * 4 + t], s);
            C[c * 4 + r] = s;
        }
}
__device__ __forceinline__ void mm_nn(const double* X, const double* Y, double* C) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double s = 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) s = fma(X[t * 4 + r], Y[c * 4 + t], s);
            C[c * 4 + r] = s;
        }
}

// Swap on the k x k pair (DA, DB; ld 4, zero beyond k).  On acceptance
// writes Qs, Zs (identity beyond k) and the new parts NA, NB and returns
// true; false if a stability test rejects it.
static __device__ __noinline__ bool gen_swap(int p, int q, const double* DA, const double* DB, bool strong,
                                      double* Qs, double* Zs, double* NA, double* NB) {
    const int k = p + q;
    double na = 0.0, nb = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        na = fma(DA[i], DA[i], na);
        nb = fma(DB[i], DB[i], nb);
    }
    const double tha = fmax(20.0 * DBL_EPSILON * sqrt(na), DBL_MIN);
    const double thb = fmax(20.0 * DBL_EPSILON * sqrt(nb), DBL_MIN);
    if (k == 2 && DA[0] * DB[5] == DA[5] * DB[0]) {
        // equal generalized eigenvalues: in order already
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            Qs[i] = Zs[i] = ((i & 3) == (i >> 2)) ? 1.0 : 0.0;
            NA[i] = DA[i];
            NB[i] = DB[i];
        }
        return true;
    }
    double R[4], L[4];
    const double g = gen_sylvester(p, q, DA, DB, R, L);
    qr_orth(p, q, L, g, Qs);
    qr_orth(p, q, R, g, Zs);
    double W[16];
    mm_tn(Qs, DA, W);
    mm_nn(W, Zs, NA);
    mm_tn(Qs, DB, W);
    mm_nn(W, Zs, NB);
    unsigned long long la = 0, lb = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 1; r < 4; ++r)
            if (c < q && r >= q && r < k) {
                la = max(la, mag(NA[c * 4 + r]));
                lb = max(lb, mag(NB[c * 4 + r]));
                NA[c * 4 + r] = 0.0;
                NB[c * 4 + r] = 0.0;
            }
    if (la > mag(tha) || lb > mag(thb)) return false;
    if (strong) {
        // D - Qs N Zs^T with the lower-left block zeroed
        for (int e = 0; e < 2; ++e) {
            const double* N0 = e ? NB : NA;
            const double* D = e ? DB : DA;
            double V[16];
            mm_nn(Qs, N0, V);
            unsigned long long err = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    double s = 0.0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) s = fma(V[t * 4 + r], Zs[t * 4 + c], s);
                    err = max(err, mag(s - D[c * 4 + r]));
                }
            if (err > mag(e ? thb : tha)) return false;
        }
    }
    // T stays upper triangular: rotate the columns of each new 2x2 block
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        const int sz = blk ? p : q, c0 = blk ? q : 0;
        if (sz != 2) continue;
        const double b10 = NB[c0 * 4 + c0 + 1], b11 = NB[(c0 + 1) * 4 + c0 + 1];
        if (b10 == 0.0) continue;
        const double h = hypot(b10, b11);
        const double cs = b11 / h, sn = -b10 / h;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            double x = NA[c0 * 4 + r], y = NA[(c0 + 1) * 4 + r];
            NA[c0 * 4 + r] = fma(cs, x, sn * y);
            NA[(c0 + 1) * 4 + r] = fma(cs, y, -sn * x);
            x = NB[c0 * 4 + r]; y = NB[(c0 + 1) * 4 + r];
            NB[c0 * 4 + r] = fma(cs, x, sn * y);
            NB[(c0 + 1) * 4 + r] = fma(cs, y, -sn * x);
            x = Zs[c0 * 4 + r]; y = Zs[(c0 + 1) * 4 + r];
            Zs[c0 * 4 + r] = fma(cs, x, sn * y);
            Zs[(c0 + 1) * 4 + r] = fma(cs, y, -sn * x);
        }
        NB[c0 * 4 + c0 + 1] = 0.0;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Window task of the pair: window [s0, s0 + w) of (S, T), w <= GW; writes
// the accumulated factors UQ, UZ (w x w, column-major, ld w) to UQg, UZg.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void window_gen_body(int n, double* __restrict__ S, int ldS,
                                                double* __restrict__ T, int ldT, int s0, int w,
                                                uint8_t* __restrict__ gsel, double* __restrict__ UQg,
                                                double* __restrict__ UZg, int strong,
                                                DevCounters* __restrict__ ctr,
                                                unsigned char* smem_raw) {
    double* UQ = reinterpret_cast<double*>(smem_raw);     // GW * GW
    double* UZ = UQ + GW * GW;                            // GW * GW
    double* Sp = UZ + GW * GW;                            // packed window of S
    double* Tp = Sp + gpoff(GW);                          // packed window of T
    double* QZ = Tp + gpoff(GW);                          // per slot: Qs (16), Zs (16)
    int* swj = reinterpret_cast<int*>(QZ + GMAXSW * 32);  // per slot: first row
    int* swk = swj + GMAXSW;                              // k, 0 = rejected
    int* swp = swk + GMAXSW;                              // p, or the stuck block's row
    uint8_t* bst = reinterpret_cast<uint8_t*>(swp + GMAXSW);
    uint8_t* sel = bst + GW;
    __shared__ int nsw, nrej, nacc;
    __shared__ int wall_top, wall_bot;
    unsigned long long wflops = 0;
    const int tid = threadIdx.x, nth = blockDim.x;

    for (int c = 0; c < w; ++c) {
        const int rows = min(c + 2, w);
        for (int r = tid; r < rows; r += nth) {
            Sp[gpoff(c) + r] = __ldcg(&S[cm(s0 + r, s0 + c, ldS)]);
            Tp[gpoff(c) + r] = __ldcg(&T[cm(s0 + r, s0 + c, ldT)]);
        }
    }
    for (int i = tid; i < w * w; i += nth) {
        const double v = ((i % w) == (i / w)) ? 1.0 : 0.0;
        UQ[i] = v;
        UZ[i] = v;
    }
    for (int i = tid; i < w; i += nth) sel[i] = __ldcg(&gsel[s0 + i]);
    if (tid == 0) {
        nrej = 0;
        nacc = 0;
        wall_top = s0 > 0 && __ldcg(&S[cm(s0, s0 - 1, ldS)]) != 0.0;
        wall_bot = s0 + w < n && __ldcg(&S[cm(s0 + w, s0 + w - 1, ldS)]) != 0.0;
    }
    __syncthreads();
    if (tid == 0 && wall_top) sel[0] = GSEL_WALL;
    if (tid == 0 && wall_bot) sel[w - 1] = GSEL_WALL;

    // every accepted swap moves a selected block up and every rejected one
    // retires a block, so the loop ends within w * w steps; the cap only
    // guards against a logic error (reported through the counters)
    for (int iter = 0;; ++iter) {
        __syncthreads();
        if (iter > 4 * GW * GW) {
            if (tid == 0) atomicAdd(&ctr->step_overflow, 1);
            break;
        }
        for (int i = tid; i < w; i += nth) bst[i] = (i == 0) || (Sp[gpoff(i - 1) + i] == 0.0);
        if (tid == 0) nsw = 0;
        __syncthreads();
        // find this step's swaps: a selected block below an unselected one
        for (int t = tid; t < w; t += nth) {
            if (t == 0 || !bst[t] || sel[t] != SEL_YES) continue;
            const int ja = bst[t - 1] ? t - 1 : t - 2;
            if (sel[ja] != SEL_NO) continue;
            const int p = t - ja;
            const int q = (t + 1 < w && !bst[t + 1]) ? 2 : 1;
            const int slot = atomicAdd(&nsw, 1);
            swj[slot] = ja;
            swk[slot] = p + q;
            swp[slot] = p;
        }
        __syncthreads();
        const int ns = nsw;
        if (ns == 0) break;
        // one thread per swap
        if (tid < ns) {
            const int slot = tid, ja = swj[slot], k = swk[slot], p = swp[slot], q = k - p;
            double DA[16], DB[16], NA[16], NB[16];
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const bool in = c < k && r < k && r <= c + 1;
                    DA[c * 4 + r] = in ? Sp[gpoff(ja + c) + ja + r] : 0.0;
                    DB[c * 4 + r] = in ? Tp[gpoff(ja + c) + ja + r] : 0.0;
                }
            double* Qs = &QZ[slot * 32];
            double* Zs = Qs + 16;
            if (gen_swap(p, q, DA, DB, strong != 0, Qs, Zs, NA, NB)) {
                for (int c = 0; c < k; ++c)
                    for (int r = 0; r <= min(c + 1, k - 1); ++r) {
                        Sp[gpoff(ja + c) + ja + r] = NA[c * 4 + r];
                        Tp[gpoff(ja + c) + ja + r] = NB[c * 4 + r];
                    }
                atomicAdd(&nacc, 1);
            } else {
                swk[slot] = 0;
                swp[slot] = ja + p;   // the stuck (selected) block
                atomicAdd(&nrej, 1);
            }
        }
        __syncthreads();
        // left: rows [j, j+k) of S and T, columns [j+k, w), by Qs^T
        for (int it = tid; it < ns * w; it += nth) {
            const int slot = it / w, c = it - slot * w;
            const int j = swj[slot], k = swk[slot];
            if (k == 0 || c < j + k) continue;
            const double* Qs = &QZ[slot * 32];
            double xs[4], xt[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                xs[r] = r < k ? Sp[gpoff(c) + j + r] : 0.0;
                xt[r] = r < k ? Tp[gpoff(c) + j + r] : 0.0;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r >= k) break;
                double as = 0.0, at = 0.0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    as = fma(Qs[r * 4 + i], xs[i], as);
                    at = fma(Qs[r * 4 + i], xt[i], at);
                }
                Sp[gpoff(c) + j + r] = as;
                Tp[gpoff(c) + j + r] = at;
            }
        }
        __syncthreads();
        // right: columns [j, j+k) of S and T rows [0, j) by Zs; of UQ by Qs
        // and UZ by Zs, rows [0, w)
        for (int it = tid; it < ns * 2 * w; it += nth) {
            const int slot = it / (2 * w), t = it - slot * 2 * w;
            const int j = swj[slot], k = swk[slot];
            if (k == 0) continue;
            const double* Qs = &QZ[slot * 32];
            const double* Zs = Qs + 16;
            if (t < w) {
                const int r = t;
                if (r >= j) continue;
                double xs[4], xt[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    xs[i] = i < k ? Sp[gpoff(j + i) + r] : 0.0;
                    xt[i] = i < k ? Tp[gpoff(j + i) + r] : 0.0;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c >= k) break;
                    double as = 0.0, at = 0.0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        as = fma(xs[i], Zs[c * 4 + i], as);
                        at = fma(xt[i], Zs[c * 4 + i], at);
                    }
                    Sp[gpoff(j + c) + r] = as;
                    Tp[gpoff(j + c) + r] = at;
                }
            } else {
                const int r = t - w;
                double xq[4], xz[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    xq[i] = i < k ? UQ[(j + i) * w + r] : 0.0;
                    xz[i] = i < k ? UZ[(j + i) * w + r] : 0.0;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c >= k) break;
                    double aq = 0.0, az = 0.0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        aq = fma(xq[i], Qs[c * 4 + i], aq);
                        az = fma(xz[i], Zs[c * 4 + i], az);
                    }
                    UQ[(j + c) * w + r] = aq;
                    UZ[(j + c) * w + r] = az;
                }
            }
        }
        __syncthreads();
        // move the selection flags with the blocks
        for (int sw = tid; sw < ns; sw += nth) {
            const int j = swj[sw], k = swk[sw];
            if (k == 0) {
                sel[swp[sw]] = SEL_STUCK;
                continue;
            }
            // left (S, T) + right (S, T) + UQ + UZ: k x k applied to
            // 2 (w - j - k) + 2 j + 2 w vectors
            wflops += 2ull * k * k * (unsigned long long)(2 * (w - j - k) + 2 * j + 2 * w);
            const int p = swp[sw], q = k - p;
            for (int i = 0; i < q; ++i) sel[j + i] = SEL_YES;
            for (int i = q; i < k; ++i) sel[j + i] = SEL_NO;
        }
        __syncthreads();
        for (int t = tid; t + 1 < w; t += nth)
            if (sel[t] == SEL_STUCK && Sp[gpoff(t) + t + 1] != 0.0) sel[t + 1] = SEL_STUCK;
    }
    __syncthreads();
    for (int c = 0; c < w; ++c) {
        const int rows = min(c + 2, w);
        for (int r = tid; r < rows; r += nth) {
            S[cm(s0 + r, s0 + c, ldS)] = Sp[gpoff(c) + r];
            T[cm(s0 + r, s0 + c, ldT)] = Tp[gpoff(c) + r];
        }
    }
    for (int i = tid; i < w; i += nth)
        if (sel[i] != GSEL_WALL) gsel[s0 + i] = sel[i];
    for (int i = tid; i < w * w; i += nth) {
        UQg[i] = UQ[i];
        UZg[i] = UZ[i];
    }
    if (wflops) atomicAdd(&ctr->win_flops, wflops);
    if (tid == 0) {
        atomicAdd(&ctr->swaps, (unsigned long long)nacc);
        atomicAdd(&ctr->rejected, (unsigned long long)nrej);
    }
}

}  // namespace gen
}  // namespace gbr
