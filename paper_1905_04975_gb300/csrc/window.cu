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

#include <float.h>

namespace gbr {

namespace {

constexpr int WIN_THREADS = 512;
constexpr int MAXSW = WMAX / 2;  // at most one swap per two positions

__device__ __forceinline__ int poff(int c) { return (c * (c + 3)) >> 1; }

// ---------------------------------------------------------------------------
// Small dense helpers on k x k column-major matrices with leading dim 4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mm4(int k, const double* A, bool tA, const double* B, bool tB,
                                    double* C) {
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            double acc = 0.0;
            for (int l = 0; l < k; ++l) {
                double a = tA ? A[i * 4 + l] : A[l * 4 + i];
                double b = tB ? B[l * 4 + j] : B[j * 4 + l];
                acc = fma(a, b, acc);
            }
            C[j * 4 + i] = acc;
        }
}

// Rotation (cs, sn) that brings the 2x2 block M = [[a, b], [c, d]] to
// standard form: equal diagonal with bc < 0 (complex pair, *cplx = true), or
// upper triangular (real pair, *cplx = false).
__device__ void std_rotation(double a, double b, double c, double d, double* cs, double* sn,
                             bool* cplx) {
    *cs = 1.0;
    *sn = 0.0;
    *cplx = false;
    if (c == 0.0) return;
    double p = 0.5 * (a - d);
    double disc = fma(p, p, b * c);
    if (disc >= 0.0) {
        // Schur vector of the eigenvalue (a + d)/2 + sign(p) sqrt(disc)
        double x = (p >= 0.0) ? p + sqrt(disc) : p - sqrt(disc);
        double h = hypot(x, c);
        *cs = x / h;
        *sn = c / h;
        return;
    }
    *cplx = true;
    double sig = b + c;
    double r = hypot(2.0 * p, sig);
    if (r == 0.0) return;
    double sg = (sig >= 0.0) ? 1.0 : -1.0;
    double c2 = sg * sig / r;          // cos 2t >= 0
    double s2 = -sg * 2.0 * p / r;     // sin 2t
    double cc = sqrt(0.5 * (1.0 + c2));
    *cs = cc;
    *sn = s2 / (2.0 * cc);
}

// Applies the rotation to the 2x2 block in place and fixes its structure.
// Returns the rotation actually used (a second one is composed in when
// rounding turned a complex pair real).
__device__ void standardize2(double* m /* 2x2, ld 4 */, double* cs, double* sn) {
    bool cplx;
    std_rotation(m[0], m[4], m[1], m[5], cs, sn, &cplx);
    double c = *cs, s = *sn;
    // N = R^T M R, R = [[c, -s], [s, c]]
    double a11 = fma(c, m[0], s * m[1]), a12 = fma(c, m[4], s * m[5]);
    double a21 = fma(c, m[1], -s * m[0]), a22 = fma(c, m[5], -s * m[4]);
    double n11 = fma(a11, c, a12 * s), n12 = fma(a12, c, -a11 * s);
    double n21 = fma(a21, c, a22 * s), n22 = fma(a22, c, -a21 * s);
    if (!cplx) {
        n21 = 0.0;
    } else {
        double avg = 0.5 * (n11 + n22);
        n11 = n22 = avg;
        if (!(n12 * n21 < 0.0)) {
            double c2, s2;
            bool cx2;
            std_rotation(n11, n12, n21, n22, &c2, &s2, &cx2);
            double b11 = fma(c2, n11, s2 * n21), b12 = fma(c2, n12, s2 * n22);
            double b21 = fma(c2, n21, -s2 * n11), b22 = fma(c2, n22, -s2 * n12);
            n11 = fma(b11, c2, b12 * s2);
            n12 = fma(b12, c2, -b11 * s2);
            n22 = fma(b22, c2, -b21 * s2);
            n21 = 0.0;
            double cc = c * c2 - s * s2, ss = s * c2 + c * s2;
            *cs = cc;
            *sn = ss;
        }
    }
    m[0] = n11; m[1] = n21; m[4] = n12; m[5] = n22;
}

// Householder vector for x[0..len): (I - tau v v^T) x = beta e_0, v[0] = 1.
__device__ void house(int len, const double* x, double* v, double* tau) {
    double alpha = x[0], sig = 0.0;
    for (int i = 1; i < len; ++i) sig = fma(x[i], x[i], sig);
    v[0] = 1.0;
    if (sig == 0.0) {
        for (int i = 1; i < len; ++i) v[i] = 0.0;
        *tau = 0.0;
        return;
    }
    double nrm = sqrt(fma(alpha, alpha, sig));
    double beta = (alpha >= 0.0) ? -nrm : nrm;
    double inv = 1.0 / (alpha - beta);
    for (int i = 1; i < len; ++i) v[i] = x[i] * inv;
    *tau = (beta - alpha) / beta;
}

// Solves T11 X - X T22 = gamma T12 for the p x q matrix X (Kronecker form,
// Gaussian elimination with complete pivoting; tiny pivots are raised to
// eps * max|K|; gamma <= 1 guards against overflow).  D holds the k x k
// block [[T11, T12], [0, T22]] with leading dimension 4.  X is p x q, ld 2.
__device__ void sylvester(const double* D, int p, int q, double* X, double* gamma) {
    const int N = p * q;
    double K[16], b[4];
    int perm[4];
    double kmax = 0.0;
    for (int r = 0; r < N; ++r) {
        int i = r % p, kk = r / p;
        b[r] = D[(p + kk) * 4 + i];                 // T12(i, kk)
        for (int c = 0; c < N; ++c) {
            int l = c % p, mm = c / p;
            double v = 0.0;
            if (kk == mm) v += D[l * 4 + i];        // T11(i, l)
            if (i == l) v -= D[(p + kk) * 4 + p + mm];  // T22(mm, kk)
            K[c * 4 + r] = v;
            kmax = fmax(kmax, fabs(v));
        }
    }
    for (int c = 0; c < 4; ++c) perm[c] = c;
    double smin = fmax(DBL_EPSILON * kmax, DBL_MIN);
    for (int st = 0; st < N; ++st) {
        int pr = st, pc = st;
        double best = -1.0;
        for (int c = st; c < N; ++c)
            for (int r = st; r < N; ++r) {
                double a = fabs(K[c * 4 + r]);
                if (a > best) { best = a; pr = r; pc = c; }
            }
        if (pr != st) {
            for (int c = 0; c < N; ++c) {
                double t = K[c * 4 + st]; K[c * 4 + st] = K[c * 4 + pr]; K[c * 4 + pr] = t;
            }
            double t = b[st]; b[st] = b[pr]; b[pr] = t;
        }
        if (pc != st) {
            for (int r = 0; r < N; ++r) {
                double t = K[st * 4 + r]; K[st * 4 + r] = K[pc * 4 + r]; K[pc * 4 + r] = t;
            }
            int t = perm[st]; perm[st] = perm[pc]; perm[pc] = t;
        }
        double piv = K[st * 4 + st];
        if (fabs(piv) < smin) { piv = smin; K[st * 4 + st] = smin; }
        double ipiv = 1.0 / piv;
        for (int r = st + 1; r < N; ++r) {
            double f = K[st * 4 + r] * ipiv;
            for (int c = st + 1; c < N; ++c) K[c * 4 + r] = fma(-f, K[c * 4 + st], K[c * 4 + r]);
            b[r] = fma(-f, b[st], b[r]);
        }
    }
    double g = 1.0, y[4];
    const double big = DBL_MAX / 4.0;
    for (int st = N - 1; st >= 0; --st) {
        double acc = b[st];
        for (int c = st + 1; c < N; ++c) acc = fma(-K[c * 4 + st], y[c], acc);
        double piv = fabs(K[st * 4 + st]);
        if (piv < 1.0 && fabs(acc) > big * piv) {
            double f = big * piv / fabs(acc);
            for (int c = 0; c < N; ++c) b[c] *= f;
            for (int c = st + 1; c < N; ++c) y[c] *= f;
            acc *= f;
            g *= f;
        }
        y[st] = acc / K[st * 4 + st];
    }
    for (int c = 0; c < N; ++c) {
        int u = perm[c];
        X[(u / p) * 2 + (u % p)] = y[c];
    }
    *gamma = g;
}

// Orthogonal Z (k x k, ld 4) and new block Dn (ld 4) with Z^T D Z = Dn and
// the blocks exchanged; false if the swap fails the stability test.
__device__ bool swap_transform(const double* D, int p, int q, bool strong, double* Z,
                               double* Dn) {
    const int k = p + q;
    for (int i = 0; i < 16; ++i) { Z[i] = 0.0; Dn[i] = 0.0; }
    if (k == 2) {
        double t11 = D[0], t12 = D[4], t22 = D[5];
        if (t11 == t22) {
            Z[0] = Z[5] = 1.0;
            Dn[0] = t11; Dn[4] = t12; Dn[5] = t22;
            return true;
        }
        double d = t22 - t11;
        double h = hypot(t12, d);
        double c = t12 / h, s = d / h;
        Z[0] = c; Z[1] = s; Z[4] = -s; Z[5] = c;
        // (Z^T D Z)_{12} with row 1 of Z^T D = (c t11, c t12 + s t22)
        double r12 = fma(c, t12, s * t22);
        Dn[0] = t22;
        Dn[4] = fma(r12, c, -(c * t11) * s);
        Dn[5] = t11;
        return true;
    }
    double dnorm = 0.0;
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) dnorm = fmax(dnorm, fabs(D[c * 4 + r]));
    const double thresh = fmax(10.0 * DBL_EPSILON * dnorm, DBL_MIN);

    double X[4], gamma;
    sylvester(D, p, q, X, &gamma);

    // Householder QR of M = [-X; gamma I_q] (k x q), Qs = H1 H2 explicit.
    double M[8];
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < k; ++i)
            M[j * 4 + i] = (i < p) ? -X[j * 2 + i] : ((i - p == j) ? gamma : 0.0);
    double v1[4], t1, v2[4] = {0, 0, 0, 0}, t2 = 0.0;
    house(k, &M[0], v1, &t1);
    if (q == 2) {
        // apply H1 to column 2 of M, then reflect its rows 1..k-1
        double w = 0.0;
        for (int i = 0; i < k; ++i) w = fma(v1[i], M[4 + i], w);
        w *= t1;
        for (int i = 0; i < k; ++i) M[4 + i] = fma(-w, v1[i], M[4 + i]);
        house(k - 1, &M[5], v2, &t2);
    }
    double Qs[16];
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) Qs[j * 4 + i] = (i == j) ? 1.0 : 0.0;
    if (q == 2) {  // Qs <- H2 (acting on indices 1..k-1)
        for (int j = 1; j < k; ++j) {
            double w = 0.0;
            for (int i = 1; i < k; ++i) w = fma(v2[i - 1], Qs[j * 4 + i], w);
            w *= t2;
            for (int i = 1; i < k; ++i) Qs[j * 4 + i] = fma(-w, v2[i - 1], Qs[j * 4 + i]);
        }
    }
    for (int j = 0; j < k; ++j) {  // Qs <- H1 Qs
        double w = 0.0;
        for (int i = 0; i < k; ++i) w = fma(v1[i], Qs[j * 4 + i], w);
        w *= t1;
        for (int i = 0; i < k; ++i) Qs[j * 4 + i] = fma(-w, v1[i], Qs[j * 4 + i]);
    }

    double T[16], Dt[16];
    mm4(k, Qs, true, D, false, T);     // Qs^T D
    mm4(k, T, false, Qs, false, Dt);   // Qs^T D Qs

    double low = 0.0;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) low = fmax(low, fabs(Dt[c * 4 + r]));
    if (!(low <= thresh)) return false;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) Dt[c * 4 + r] = 0.0;
    if (strong) {
        mm4(k, Qs, false, Dt, false, T);   // Qs Dt0
        double E[16];
        mm4(k, T, false, Qs, true, E);     // Qs Dt0 Qs^T
        double err = 0.0;
        for (int c = 0; c < k; ++c)
            for (int r = 0; r < k; ++r) err = fmax(err, fabs(E[c * 4 + r] - D[c * 4 + r]));
        if (!(err <= thresh)) return false;
    }

    // Standardize the new 2x2 blocks: R = diag(R1, R2); Z = Qs R; Dn = R^T Dt0 R.
    double R[16];
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) R[j * 4 + i] = (i == j) ? 1.0 : 0.0;
    double blk1[16], blk2[16];
    if (q == 2) {
        blk1[0] = Dt[0]; blk1[1] = Dt[1]; blk1[4] = Dt[4]; blk1[5] = Dt[5];
        double c, s;
        standardize2(blk1, &c, &s);
        R[0] = c; R[1] = s; R[4] = -s; R[5] = c;
    }
    if (p == 2) {
        int o = q;
        blk2[0] = Dt[o * 4 + o]; blk2[1] = Dt[o * 4 + o + 1];
        blk2[4] = Dt[(o + 1) * 4 + o]; blk2[5] = Dt[(o + 1) * 4 + o + 1];
        double c, s;
        standardize2(blk2, &c, &s);
        R[o * 4 + o] = c; R[o * 4 + o + 1] = s; R[(o + 1) * 4 + o] = -s; R[(o + 1) * 4 + o + 1] = c;
    }
    mm4(k, Qs, false, R, false, Z);
    mm4(k, R, true, Dt, false, T);
    mm4(k, T, false, R, false, Dn);
    // exact structure: zero lower-left block, standardized 2x2 blocks
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) Dn[c * 4 + r] = 0.0;
    if (q == 2) { Dn[0] = blk1[0]; Dn[1] = blk1[1]; Dn[4] = blk1[4]; Dn[5] = blk1[5]; }
    else if (k > 1) { Dn[1] = 0.0; }
    if (p == 2) {
        int o = q;
        Dn[o * 4 + o] = blk2[0]; Dn[o * 4 + o + 1] = blk2[1];
        Dn[(o + 1) * 4 + o] = blk2[4]; Dn[(o + 1) * 4 + o + 1] = blk2[5];
    }
    // entries two or more below the diagonal are structurally zero
    for (int c = 0; c < k; ++c)
        for (int r = c + 2; r < k; ++r) Dn[c * 4 + r] = 0.0;
    return true;
}

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
