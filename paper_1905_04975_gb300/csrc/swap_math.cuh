// FP64 math of one adjacent block swap (Section 3.2: Givens rotations and
// Householder reflectors), shared by the window kernels.  Host-callable too,
// so the same code can be exercised on the CPU.
#pragma once

#include <float.h>
#include <math.h>
#include <string.h>

#ifdef __CUDACC__
#define GBR_HD __host__ __device__ __forceinline__
#define GBR_HD_NOINLINE static __host__ __device__ __noinline__
#else
#define GBR_HD inline
#define GBR_HD_NOINLINE static inline
#endif

namespace gbr {

// ---------------------------------------------------------------------------
// Small dense helpers on k x k column-major matrices with leading dim 4.
// ---------------------------------------------------------------------------
GBR_HD void mm4(int k, const double* A, bool tA, const double* B, bool tB,
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
GBR_HD void std_rotation(double a, double b, double c, double d, double* cs, double* sn,
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
GBR_HD void standardize2(double* m /* 2x2, ld 4 */, double* cs, double* sn) {
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
GBR_HD void house(int len, const double* x, double* v, double* tau) {
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
GBR_HD void sylvester(const double* D, int p, int q, double* X, double* gamma) {
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

// Error-free transformations (Knuth's TwoSum; TwoProduct through fma).
GBR_HD void two_sum(double a, double b, double* s, double* e) {
    double x = a + b, bb = x - a;
    *e = (a - (x - bb)) + (b - bb);
    *s = x;
}

// max_ij |(Qs Dt Qs^T - D)_ij| evaluated in compensated arithmetic: each
// entry is the sum of the k*k triple products Qs_ia Dt_ab Qs_jb and -D_ij,
// every product split exactly into high and low parts and summed with
// TwoSum, so the result is accurate to a few units in the last place of the
// residual itself rather than of the terms.
GBR_HD double recon_err_compensated(int k, const double* Qs, const double* Dt, const double* D) {
    double worst = 0.0;
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            double s = -D[j * 4 + i], comp = 0.0;
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) {
                    double qa = Qs[a * 4 + i], dab = Dt[b * 4 + a], qb = Qs[b * 4 + j];
                    double ph = qa * dab, pl = fma(qa, dab, -ph);   // qa dab = ph + pl
                    double th = ph * qb, tl = fma(ph, qb, -th);     // ph qb = th + tl
                    double e;
                    two_sum(s, th, &s, &e);
                    comp += e + tl + pl * qb;
                }
            worst = fmax(worst, fabs(s + comp));
        }
    return worst;
}

// Given the swap's orthogonal Qs and Dt0 = Qs^T D Qs with its lower-left block
// zeroed: rotations that restore the standard form of the new 2x2 blocks,
// R = diag(R1, R2), then Z = Qs R and Dn = R^T Dt0 R with exact structure.
GBR_HD void finish_swap(int p, int q, const double* Qs, const double* Dt, double* Z, double* Dn) {
    const int k = p + q;
    double T[16];
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
}

// Orthogonal Z (k x k, ld 4) and new block Dn (ld 4) with Z^T D Z = Dn and
// the blocks exchanged, in plain FP64; false if the swap fails the stability
// test as evaluated here.
GBR_HD bool swap_transform_fast(const double* D, int p, int q, bool strong, double* Z,
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

    // Orthogonal Qs whose leading q columns span [-X; gamma I_q].
    //  p=2, q=1: one 3x3 reflector mapping [-X; gamma] to a multiple of e_1;
    //  p=1, q=2: one 3x3 reflector mapping u = (gamma, x11, x12), which is
    //            orthogonal to both columns of [-X; gamma I], to a multiple of
    //            e_3 (its first two columns then span the subspace);
    //  p=2, q=2: Householder QR of the 4x2 matrix [-X; gamma I] (two reflectors).
    double M[8];
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < k; ++i)
            M[j * 4 + i] = (i < p) ? -X[j * 2 + i] : ((i - p == j) ? gamma : 0.0);
    double v1[4], t1, v2[4] = {0, 0, 0, 0}, t2 = 0.0;
    if (p == 1 && q == 2) {
        // reflector for the reversed vector (x12, x11, gamma) -> e_1, then reversed back
        double ur[3] = {X[2], X[0], gamma}, vr[3];
        house(3, ur, vr, &t1);
        v1[0] = vr[2]; v1[1] = vr[1]; v1[2] = vr[0]; v1[3] = 0.0;
    } else {
        house(k, &M[0], v1, &t1);
    }
    if (p == 2 && q == 2) {
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
    if (p == 2 && q == 2) {  // Qs <- H2 (acting on indices 1..3)
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
        // Rounding in this check alone can reach the threshold for
        // well-conditioned swaps; decide on the accurately evaluated residual.
        if (!(err <= thresh) && !(recon_err_compensated(k, Qs, Dt, D) <= thresh)) return false;
    }

    finish_swap(p, q, Qs, Dt, Z, Dn);
    return true;
}

// ---------------------------------------------------------------------------
// Fast k = 3 swap without re-standardization (the window kernel restores the
// standard form of its 2x2 blocks once, at the end of the window).
//
// 2|1: D = [[A, c], [0, lam]] with A 2x2.  X solves (A - lam I) X = c; the one
// reflector H with H (-x0, -x1, 1)^T = beta e_1 gives Dt = H D H with lam first.
// 1|2 is mapped onto 2|1 by the flip D' = F D^T F (F reverses the indices):
// if Z'^T D' Z' = Dt' then Z = F Z' F and Dt = F Dt'^T F.
// Integer comparisons of |x| bit patterns keep the tests off the FP64 pipe.
// Returns false when the fast path cannot decide (tiny pivot) or the swap
// fails the weak or strong test; the caller then uses the full transform.
// ---------------------------------------------------------------------------
GBR_HD unsigned long long abs_bits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
#else
    unsigned long long u;
    memcpy(&u, &x, 8);
    return u & 0x7fffffffffffffffULL;
#endif
}
GBR_HD double bits_double(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

// D, Z, Dn: 3x3 column-major with leading dimension 4 (entries [c*4 + r]).
GBR_HD bool swap21_fast(const double* D, bool strong, double* Z, double* Dn) {
    unsigned long long mx = 0;
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) {
            unsigned long long b = abs_bits(D[c * 4 + r]);
            mx = b > mx ? b : mx;
        }
    const double thresh = fmax(10.0 * DBL_EPSILON * bits_double(mx), DBL_MIN);
    const unsigned long long tb = abs_bits(thresh);
    const double lam = D[10];
    const double a00 = D[0] - lam, a01 = D[4], a10 = D[1], a11 = D[5] - lam;
    const double c0 = D[8], c1 = D[9];
    const double det = fma(a00, a11, -(a01 * a10));
    // partial-pivoting quality check: |det| must not be tiny against the entries
    unsigned long long am = abs_bits(a00);
    am = abs_bits(a01) > am ? abs_bits(a01) : am;
    am = abs_bits(a10) > am ? abs_bits(a10) : am;
    am = abs_bits(a11) > am ? abs_bits(a11) : am;
    const double amax = bits_double(am);
    if (!(abs_bits(det) > abs_bits(1e-4 * amax * amax))) return false;
    const double rdet = 1.0 / det;
    const double x0 = fma(a11, c0, -(a01 * c1)) * rdet;
    const double x1 = fma(a00, c1, -(a10 * c0)) * rdet;
    // reflector for u = (-x0, -x1, 1)
    const double alpha = -x0;
    const double sig = fma(x1, x1, 1.0);
    const double nrm = sqrt(fma(alpha, alpha, sig));
    const double beta = alpha >= 0.0 ? -nrm : nrm;
    const double dd = alpha - beta;
    const double rdd = 1.0 / dd;
    const double v0 = 1.0, v1 = -x1 * rdd, v2 = rdd;
    const double tau = -dd / beta;
    // Dt = H D H, H = I - tau v v^T
    double T[9];
    for (int c = 0; c < 3; ++c) {
        double w = fma(v2, D[c * 4 + 2], fma(v1, D[c * 4 + 1], v0 * D[c * 4 + 0])) * tau;
        T[c * 3 + 0] = fma(-w, v0, D[c * 4 + 0]);
        T[c * 3 + 1] = fma(-w, v1, D[c * 4 + 1]);
        T[c * 3 + 2] = fma(-w, v2, D[c * 4 + 2]);
    }
    for (int r = 0; r < 3; ++r) {
        double w = fma(T[6 + r], v2, fma(T[3 + r], v1, T[r] * v0)) * tau;
        Dn[0 * 4 + r] = fma(-w, v0, T[r]);
        Dn[1 * 4 + r] = fma(-w, v1, T[3 + r]);
        Dn[2 * 4 + r] = fma(-w, v2, T[6 + r]);
    }
    // weak test: the block that must vanish, rows 1..2 of column 0
    if (abs_bits(Dn[1]) > tb || abs_bits(Dn[2]) > tb) return false;
    Dn[1] = 0.0;
    Dn[2] = 0.0;
    if (strong) {
        // E = H Dt0 H - D
        for (int c = 0; c < 3; ++c) {
            double w = fma(v2, Dn[c * 4 + 2], fma(v1, Dn[c * 4 + 1], v0 * Dn[c * 4 + 0])) * tau;
            T[c * 3 + 0] = fma(-w, v0, Dn[c * 4 + 0]);
            T[c * 3 + 1] = fma(-w, v1, Dn[c * 4 + 1]);
            T[c * 3 + 2] = fma(-w, v2, Dn[c * 4 + 2]);
        }
        for (int r = 0; r < 3; ++r) {
            double w = fma(T[6 + r], v2, fma(T[3 + r], v1, T[r] * v0)) * tau;
            double e0 = fma(-w, v0, T[r]) - D[0 * 4 + r];
            double e1 = fma(-w, v1, T[3 + r]) - D[1 * 4 + r];
            double e2 = fma(-w, v2, T[6 + r]) - D[2 * 4 + r];
            if (abs_bits(e0) > tb || abs_bits(e1) > tb || abs_bits(e2) > tb) return false;
        }
    }
    // Z = H (symmetric)
    const double tv0 = tau * v0, tv1 = tau * v1, tv2 = tau * v2;
    Z[0] = fma(-tv0, v0, 1.0); Z[1] = -tv0 * v1;          Z[2] = -tv0 * v2;
    Z[4] = Z[1];               Z[5] = fma(-tv1, v1, 1.0); Z[6] = -tv1 * v2;
    Z[8] = Z[2];               Z[9] = Z[6];               Z[10] = fma(-tv2, v2, 1.0);
    return true;
}

// 1|2 is solved as 2|1 on the flipped block F D^T F (F the exchange matrix)
// and flipped back.  The flip is a select between registers, not a branch:
// the lanes of a warp that serve 1|2 and 2|1 swaps then run one instruction
// stream (on the GPU every FP64 instruction a warp issues costs the same
// whether one lane or all of them need it).
GBR_HD bool swap3_fast(const double* D, int p, bool strong, double* Z, double* Dn) {
    const bool f = (p == 1);
    double Df[16], Zf[16], Dnf[16];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) Df[c * 4 + r] = f ? D[(2 - r) * 4 + (2 - c)] : D[c * 4 + r];
    if (!swap21_fast(Df, strong, Zf, Dnf)) return false;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Z[c * 4 + r] = f ? Zf[(2 - c) * 4 + (2 - r)] : Zf[c * 4 + r];
            Dn[c * 4 + r] = f ? Dnf[(2 - r) * 4 + (2 - c)] : Dnf[c * 4 + r];
        }
    return true;
}

// ---------------------------------------------------------------------------
// Accurate retry in double-double arithmetic (a value is hi + lo with
// |lo| <= ulp(hi)/2; Dekker's and Knuth's error-free transformations).
// For moderately ill-conditioned swaps (||X|| ~ 1e2) the rounding of a
// plain-FP64 transform alone can reach the 10 eps max|D| threshold; the
// retry builds the same reflectors and Qs^T D Qs in ~106-bit arithmetic, so
// that only a genuinely unstable swap (large residual of the Sylvester
// solution, seen by the weak test) is rejected.
// ---------------------------------------------------------------------------
struct dd { double hi, lo; };

GBR_HD dd dd_from(double a) { return dd{a, 0.0}; }
GBR_HD dd dd_norm(double s, double e) {
    double h = s + e;
    return dd{h, e - (h - s)};
}
GBR_HD dd dd_add(dd a, dd b) {
    double s, e;
    two_sum(a.hi, b.hi, &s, &e);
    e += a.lo + b.lo;
    return dd_norm(s, e);
}
GBR_HD dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
GBR_HD dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
GBR_HD dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return dd_norm(p, e);
}
GBR_HD dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(b, dd_from(q1)));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(b, dd_from(q2)));
    double q3 = r.hi / b.hi;
    return dd_add(dd_norm(q1, q2), dd_from(q3));
}
GBR_HD dd dd_sqrt(dd a) {
    if (a.hi <= 0.0) return dd_from(0.0);
    double x = sqrt(a.hi);
    dd x2 = dd_mul(dd_from(x), dd_from(x));
    double corr = (dd_sub(a, x2).hi) / (2.0 * x);
    return dd_norm(x, corr);
}

// (I - tau v v^T) x = beta e_0, v[0] = 1, in double-double.
GBR_HD void house_dd(int len, const dd* x, dd* v, dd* tau) {
    dd sig = dd_from(0.0);
    for (int i = 1; i < len; ++i) sig = dd_add(sig, dd_mul(x[i], x[i]));
    v[0] = dd_from(1.0);
    if (sig.hi == 0.0) {
        for (int i = 1; i < len; ++i) v[i] = dd_from(0.0);
        *tau = dd_from(0.0);
        return;
    }
    dd nrm = dd_sqrt(dd_add(dd_mul(x[0], x[0]), sig));
    dd beta = (x[0].hi >= 0.0) ? dd_neg(nrm) : nrm;
    dd den = dd_sub(x[0], beta);
    for (int i = 1; i < len; ++i) v[i] = dd_div(x[i], den);
    *tau = dd_div(dd_sub(beta, x[0]), beta);
}

GBR_HD_NOINLINE bool swap_transform_accurate(const double* D, int p, int q, bool strong, double* Z,
                                    double* Dn) {
    const int k = p + q;
    double dnorm = 0.0;
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) dnorm = fmax(dnorm, fabs(D[c * 4 + r]));
    const double thresh = fmax(10.0 * DBL_EPSILON * dnorm, DBL_MIN);

    // X from the FP64 solve, refined once with a double-double residual:
    // r = gamma T12 - (T11 X - X T22); T11 dX - dX T22 = r.
    double X[4], gamma;
    sylvester(D, p, q, X, &gamma);
    dd Xd[4], R[4];
    double Rh[16];
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < p; ++i) {
            dd acc = dd_mul(dd_from(gamma), dd_from(D[(p + j) * 4 + i]));
            for (int l = 0; l < p; ++l)
                acc = dd_sub(acc, dd_mul(dd_from(D[l * 4 + i]), dd_from(X[j * 2 + l])));
            for (int l = 0; l < q; ++l)
                acc = dd_add(acc, dd_mul(dd_from(X[l * 2 + i]), dd_from(D[(p + j) * 4 + p + l])));
            R[j * 2 + i] = acc;
        }
    for (int i = 0; i < 16; ++i) Rh[i] = 0.0;
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) Rh[j * 4 + i] = D[j * 4 + i];
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < p; ++i) Rh[(p + j) * 4 + i] = R[j * 2 + i].hi;
    double dX[4], g2;
    sylvester(Rh, p, q, dX, &g2);
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < p; ++i)
            Xd[j * 2 + i] = dd_add(dd_from(X[j * 2 + i]), dd_from(g2 > 0.0 ? dX[j * 2 + i] / g2 : 0.0));

    // reflectors (same construction as the fast path), in double-double
    dd v1[4], t1, v2[3] = {dd_from(0), dd_from(0), dd_from(0)}, t2 = dd_from(0.0);
    dd g = dd_from(gamma);
    if (p == 1 && q == 2) {
        dd ur[3] = {Xd[2], Xd[0], g}, vr[3];
        house_dd(3, ur, vr, &t1);
        v1[0] = vr[2]; v1[1] = vr[1]; v1[2] = vr[0]; v1[3] = dd_from(0.0);
    } else {
        dd c0[4];
        for (int i = 0; i < k; ++i)
            c0[i] = (i < p) ? dd_neg(Xd[i]) : ((i == p) ? g : dd_from(0.0));
        house_dd(k, c0, v1, &t1);
        if (p == 2 && q == 2) {
            dd c1[4] = {dd_neg(Xd[2]), dd_neg(Xd[3]), dd_from(0.0), g};
            dd w = dd_from(0.0);
            for (int i = 0; i < 4; ++i) w = dd_add(w, dd_mul(v1[i], c1[i]));
            w = dd_mul(w, t1);
            for (int i = 0; i < 4; ++i) c1[i] = dd_sub(c1[i], dd_mul(w, v1[i]));
            house_dd(3, &c1[1], v2, &t2);
        }
    }
    // Qs = H1 H2 explicit, double-double
    dd Qd[16];
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) Qd[j * 4 + i] = dd_from(i == j ? 1.0 : 0.0);
    if (p == 2 && q == 2)
        for (int j = 1; j < 4; ++j) {
            dd w = dd_from(0.0);
            for (int i = 1; i < 4; ++i) w = dd_add(w, dd_mul(v2[i - 1], Qd[j * 4 + i]));
            w = dd_mul(w, t2);
            for (int i = 1; i < 4; ++i) Qd[j * 4 + i] = dd_sub(Qd[j * 4 + i], dd_mul(w, v2[i - 1]));
        }
    for (int j = 0; j < k; ++j) {
        dd w = dd_from(0.0);
        for (int i = 0; i < k; ++i) w = dd_add(w, dd_mul(v1[i], Qd[j * 4 + i]));
        w = dd_mul(w, t1);
        for (int i = 0; i < k; ++i) Qd[j * 4 + i] = dd_sub(Qd[j * 4 + i], dd_mul(w, v1[i]));
    }
    // Dt = Qs^T D Qs
    dd T[16], Dtd[16];
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            dd acc = dd_from(0.0);
            for (int l = 0; l < k; ++l) acc = dd_add(acc, dd_mul(Qd[i * 4 + l], dd_from(D[j * 4 + l])));
            T[j * 4 + i] = acc;
        }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            dd acc = dd_from(0.0);
            for (int l = 0; l < k; ++l) acc = dd_add(acc, dd_mul(T[l * 4 + i], Qd[j * 4 + l]));
            Dtd[j * 4 + i] = acc;
        }
    double Qs[16], Dt[16];
    for (int i = 0; i < 16; ++i) { Qs[i] = 0.0; Dt[i] = 0.0; }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
            Qs[j * 4 + i] = Qd[j * 4 + i].hi + Qd[j * 4 + i].lo;
            Dt[j * 4 + i] = Dtd[j * 4 + i].hi + Dtd[j * 4 + i].lo;
        }
    double low = 0.0;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) low = fmax(low, fabs(Dt[c * 4 + r]));
    if (!(low <= thresh)) return false;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) Dt[c * 4 + r] = 0.0;
    if (strong && !(recon_err_compensated(k, Qs, Dt, D) <= thresh)) return false;
    finish_swap(p, q, Qs, Dt, Z, Dn);
    return true;
}

// A swap: the fast FP64 transform, and the double-double retry when the fast
// one fails the stability test.  The window task reaches it only when its
// specialized paths decline a swap, so it stays out of line: the window
// task's step loop must fit the instruction caches.
GBR_HD_NOINLINE bool swap_transform(const double* D, int p, int q, bool strong, double* Z, double* Dn) {
    if (swap_transform_fast(D, p, q, strong, Z, Dn)) return true;
    if (p + q == 2) return false;
    return swap_transform_accurate(D, p, q, strong, Z, Dn);
}

}  // namespace gbr
