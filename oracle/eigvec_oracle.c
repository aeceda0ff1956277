/*
 * CPU oracle for the eigenvectors of a real Schur form -- TEST INFRASTRUCTURE.
 *
 * Section 2 (Eq. 5): for an eigenvalue lambda of S (upper quasi-triangular,
 * standardized 2x2 blocks [[a, b], [c, a]], bc < 0) a vector y != 0 with
 * (S - lambda I) y = 0; Eq. 6 back-transforms it with the orthogonal factor
 * (x = Q y, done by the caller of this file).  The paper leaves the method to
 * the cited works and requires protection against floating-point overflow
 * (Section 3.1); the steps here are the plain definition:
 *
 *   - lambda from a 1x1 block at j: y[j] = 1, y[i] = 0 for i > j; for a 2x2
 *     block at (j, j+1) with lambda = a + i w (w = sqrt(-bc) > 0): the
 *     complex vector with y[j] = 1, y[j+1] = i w / b (the null vector of the
 *     block minus lambda), zero below;
 *   - back substitution upwards, one diagonal block at a time, column
 *     oriented: r = -S[0:j0, block(j)] y[block(j)]; for each block B above,
 *     y[B] = (S[B,B] - lambda I)^-1 r[B], then r[0:B0] -= S[0:B0, B] y[B];
 *   - a pivot (a 1x1 denominator or a 2x2 determinant) of magnitude below
 *     smin = max(eps |lambda|, DBL_MIN / eps) is replaced by smin;
 *   - overflow protection: rb bounds max|r| over the rows still to be solved
 *     (|z| = |re| + |im| for complex values).  Before a block is solved, and
 *     before its update of r, the vector is scaled by 2^-512 (exact) while the
 *     next value or the new bound would exceed BIG = 2^900;
 *     (each scaling loop stops after 8 passes; finite input needs at most 3);
 *   - the result is normalized: max |y_i| = 1 for a real vector,
 *     max (|re y_i| + |im y_i|) = 1 for a complex one.
 *
 * A complex vector is returned as two columns (real part, imaginary part),
 * for the eigenvalue with positive imaginary part, as in LAPACK.
 * Plain C, binary64; no blocking, no BLAS.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

static const double BIG = 0x1p900;
static const double SHRINK = 0x1p-512;

/* size of the diagonal block starting at j (1 or 2) */
static int blk(int n, const double *S, int ldS, int j) {
    return (j + 1 < n && AT(S, ldS, j + 1, j) != 0.0) ? 2 : 1;
}

typedef struct { double re, im; } cplx;

static double cabs1(cplx z) { return fabs(z.re) + fabs(z.im); }
static cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static cplx csub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
static cplx cdiv(cplx a, cplx b) {
    /* Smith's algorithm */
    cplx r;
    if (fabs(b.re) >= fabs(b.im)) {
        double t = b.im / b.re, d = b.re + b.im * t;
        r.re = (a.re + a.im * t) / d;
        r.im = (a.im - a.re * t) / d;
    } else {
        double t = b.re / b.im, d = b.re * t + b.im;
        r.re = (a.re * t + a.im) / d;
        r.im = (a.im * t - a.re) / d;
    }
    return r;
}

/* replaces a pivot of magnitude below smin by smin (keeping its direction) */
static cplx perturb(cplx d, double smin) {
    double m = cabs1(d);
    if (m >= smin) return d;
    if (m == 0.0) { cplx r = {smin, 0.0}; return r; }
    cplx r = {d.re * (smin / m), d.im * (smin / m)};
    return r;
}

/*
 * One eigenvector.  j: first row of the eigenvalue's block (size nb); y: n
 * complex entries out (imaginary parts zero for a real eigenvalue), already
 * normalized.  Returns the number of 2^-512 scalings applied.
 */
static int eigvec_one(int n, const double *S, int ldS, int j, int nb, cplx *y) {
    cplx lam;
    int top = j + nb; /* rows [0, top) are the vector's support */
    for (int i = 0; i < n; ++i) y[i].re = y[i].im = 0.0;
    if (nb == 1) {
        lam.re = AT(S, ldS, j, j);
        lam.im = 0.0;
        y[j].re = 1.0;
    } else {
        double a = AT(S, ldS, j, j), b = AT(S, ldS, j, j + 1), c = AT(S, ldS, j + 1, j);
        double w = sqrt(-b * c);
        lam.re = a;
        lam.im = w;
        y[j].re = 1.0;
        y[j + 1].im = w / b;
    }
    const double smin = fmax(DBL_EPSILON * cabs1(lam), DBL_MIN / DBL_EPSILON);
    /* r = -S[0:j, j:top] y[j:top] */
    cplx *r = (cplx *)calloc((size_t)(j > 0 ? j : 1), sizeof(cplx));
    double rb = 0.0;
    for (int i = 0; i < j; ++i) {
        cplx s = {0.0, 0.0};
        for (int t = j; t < top; ++t) {
            s.re -= AT(S, ldS, i, t) * y[t].re;
            s.im -= AT(S, ldS, i, t) * y[t].im;
        }
        r[i] = s;
        if (cabs1(s) > rb) rb = cabs1(s);
    }
    int nscale = 0;
    int b1 = j; /* blocks above: [b0, b1) */
    while (b1 > 0) {
        const int b0 = (b1 >= 2 && AT(S, ldS, b1 - 1, b1 - 2) != 0.0) ? b1 - 2 : b1 - 1;
        const int k = b1 - b0;
        cplx x[2];
        /* solve (S[B,B] - lambda I) x = r[B], scaling first if |x| could exceed BIG */
        if (k == 1) {
            cplx d = {AT(S, ldS, b0, b0) - lam.re, -lam.im};
            d = perturb(d, smin);
            for (int it = 0; it < 8 && cabs1(r[b0]) > BIG * cabs1(d); ++it) {
                for (int i = 0; i < top; ++i) { y[i].re *= SHRINK; y[i].im *= SHRINK; }
                for (int i = 0; i < b1; ++i) { r[i].re *= SHRINK; r[i].im *= SHRINK; }
                rb *= SHRINK;
                ++nscale;
            }
            x[0] = cdiv(r[b0], d);
        } else {
            /* M = S[B,B] - lambda I; x = adj(M) r / det(M) */
            cplx m00 = {AT(S, ldS, b0, b0) - lam.re, -lam.im};
            cplx m01 = {AT(S, ldS, b0, b0 + 1), 0.0};
            cplx m10 = {AT(S, ldS, b0 + 1, b0), 0.0};
            cplx m11 = {AT(S, ldS, b0 + 1, b0 + 1) - lam.re, -lam.im};
            cplx det = csub(cmul(m00, m11), cmul(m01, m10));
            double mx = fmax(fmax(cabs1(m00), cabs1(m01)), fmax(cabs1(m10), cabs1(m11)));
            det = perturb(det, smin * fmax(mx, smin));
            for (int it = 0;; ++it) {
                cplx u0 = csub(cmul(m11, r[b0]), cmul(m01, r[b0 + 1]));
                cplx u1 = csub(cmul(m00, r[b0 + 1]), cmul(m10, r[b0]));
                double um = fmax(cabs1(u0), cabs1(u1));
                if (um <= BIG * cabs1(det) || it == 8) {
                    x[0] = cdiv(u0, det);
                    x[1] = cdiv(u1, det);
                    break;
                }
                for (int i = 0; i < top; ++i) { y[i].re *= SHRINK; y[i].im *= SHRINK; }
                for (int i = 0; i < b1; ++i) { r[i].re *= SHRINK; r[i].im *= SHRINK; }
                rb *= SHRINK;
                ++nscale;
            }
        }
        for (int t = 0; t < k; ++t) y[b0 + t] = x[t];
        /* r[0:b0] -= S[0:b0, B] x, scaling first if the bound could exceed BIG */
        if (b0 > 0) {
            double cm = 0.0;
            for (int i = 0; i < b0; ++i)
                for (int t = 0; t < k; ++t) cm = fmax(cm, fabs(AT(S, ldS, i, b0 + t)));
            double xm = 0.0;
            for (int t = 0; t < k; ++t) xm = fmax(xm, cabs1(x[t]));
            for (int it = 0; it < 8 && rb + k * cm * xm > BIG; ++it) {
                for (int i = 0; i < top; ++i) { y[i].re *= SHRINK; y[i].im *= SHRINK; }
                for (int i = 0; i < b1; ++i) { r[i].re *= SHRINK; r[i].im *= SHRINK; }
                for (int t = 0; t < k; ++t) { x[t].re *= SHRINK; x[t].im *= SHRINK; }
                rb *= SHRINK;
                xm *= SHRINK;
                ++nscale;
            }
            rb += k * cm * xm;
            for (int i = 0; i < b0; ++i)
                for (int t = 0; t < k; ++t) {
                    r[i].re -= AT(S, ldS, i, b0 + t) * x[t].re;
                    r[i].im -= AT(S, ldS, i, b0 + t) * x[t].im;
                }
        }
        b1 = b0;
    }
    free(r);
    double mx = 0.0;
    for (int i = 0; i < top; ++i) mx = fmax(mx, cabs1(y[i]));
    if (mx > 0.0)
        for (int i = 0; i < top; ++i) { y[i].re /= mx; y[i].im /= mx; }
    return nscale;
}

/*
 * Eigenvectors of the selected eigenvalues, in diagonal order.
 *   select: n ints (a 2x2 block is selected if either of its rows is), or
 *           NULL for all;
 *   Y:      n x m column-major (ldY), m = number of selected positions; a
 *           real eigenvalue gives one column, a conjugate pair two (real and
 *           imaginary part of the vector of the eigenvalue with positive
 *           imaginary part);
 *   nscale: per column, the number of 2^-512 scalings (or NULL).
 * Returns m.
 */
int orc_eigvec(int n, const double *S, int ldS, const int *select, double *Y, int ldY,
               int *nscale) {
    cplx *y = (cplx *)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int j = 0; j < n;) {
        const int nb = blk(n, S, ldS, j);
        int sel = select ? (select[j] != 0 || (nb == 2 && select[j + 1] != 0)) : 1;
        if (sel) {
            int ns = eigvec_one(n, S, ldS, j, nb, y);
            for (int i = 0; i < n; ++i) AT(Y, ldY, i, m) = y[i].re;
            if (nscale) nscale[m] = ns;
            if (nb == 2) {
                for (int i = 0; i < n; ++i) AT(Y, ldY, i, m + 1) = y[i].im;
                if (nscale) nscale[m + 1] = ns;
            }
            m += nb;
        }
        j += nb;
    }
    free(y);
    return m;
}
