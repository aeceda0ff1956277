/*
 * Plain CPU oracle for real Schur-form eigenvalue reordering.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  It shares no code, header, table
 * or helper with the GPU library, and the GPU library never calls it.
 *
 * What it computes (Section 2, Eq. 7): given S in standard real Schur form
 * (Eq. 4: upper quasi-triangular with 1x1 and standardized 2x2 diagonal
 * blocks), an orthogonal Q and a selection of eigenvalues, an orthogonal
 * Q3 such that S_hat = Q3^T S Q3 is again in standard real Schur form with
 * the selected eigenvalues in its leading diagonal blocks; S is overwritten
 * by S_hat and Q by Q Q3.
 *
 * How (Section 3.2, Fig. 1a, "scalar updates"): every selected block is
 * moved up by swaps with the block directly above it, top to bottom, and
 * every local transformation -- a Givens rotation for two 1x1 blocks, 3x3
 * (or two 4x4/3x3) Householder reflectors otherwise, then one rotation per
 * new 2x2 block to restore the standard form -- is applied at once to the
 * whole rows/columns of S and to the columns of Q.  No windows, no
 * accumulation, no blocking.
 *
 * The paper names the transformation types only.  The swap itself is the
 * direct swap of adjacent diagonal blocks by a Sylvester solve (Bai and
 * Demmel), written here from its mathematics:
 *   T11 X - X T22 = gamma T12 ;   D [-X; gamma I] = [-X; gamma I] T22,
 * so an orthogonal Qs whose leading q columns span [-X; gamma I] moves the
 * eigenvalues of T22 to the top:  Qs^T D Qs = [[R T22 R^-1, *], [0, *]].
 * A swap is accepted only if the lower-left block of Qs^T D Qs and the
 * back-transformation error are both below 10 eps max|D| (weak and strong
 * stability tests); otherwise nothing is applied and the swap is rejected.
 *
 * Floating point: IEEE binary64, round to nearest, built with
 * -ffp-contract=off (no fused multiply-add).
 */
#include <float.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EPS DBL_EPSILON   /* 2^-52 */
#define ORC_SMALL DBL_MIN     /* smallest normal */

#define EL(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* ---------------------------------------------------------------------- */
/* Structure of a standard real Schur form (Eq. 4).                       */
/* ---------------------------------------------------------------------- */

/* Size of the diagonal block starting at position j (j must be a start). */
static int block_size(int n, const double *S, int ldS, int j)
{
    return (j + 1 < n && EL(S, ldS, j + 1, j) != 0.0) ? 2 : 1;
}

/* 0 if S is in standard real Schur form, else -(1 + first bad column). */
int orc_validate(int n, const double *S, int ldS)
{
    for (int j = 0; j < n; ++j) {
        for (int i = j + 2; i < n; ++i)
            if (EL(S, ldS, i, j) != 0.0) return -(1 + j);
        if (j + 1 < n && EL(S, ldS, j + 1, j) != 0.0) {
            if (j + 2 < n && EL(S, ldS, j + 2, j + 1) != 0.0) return -(1 + j);
            if (EL(S, ldS, j, j) != EL(S, ldS, j + 1, j + 1)) return -(1 + j);
            if (!(EL(S, ldS, j, j + 1) * EL(S, ldS, j + 1, j) < 0.0)) return -(1 + j);
        }
    }
    return 0;
}

/* Eigenvalues from the diagonal blocks: a 1x1 block s gives (s, 0); a
 * standardized 2x2 block [[a, b], [c, a]] gives a +- i sqrt(-bc), the one
 * with positive imaginary part first. */
void orc_eigenvalues(int n, const double *S, int ldS, double *wr, double *wi)
{
    int j = 0;
    while (j < n) {
        if (block_size(n, S, ldS, j) == 1) {
            wr[j] = EL(S, ldS, j, j);
            wi[j] = 0.0;
            j += 1;
        } else {
            double a = EL(S, ldS, j, j);
            double im = sqrt(fabs(EL(S, ldS, j, j + 1))) * sqrt(fabs(EL(S, ldS, j + 1, j)));
            wr[j] = a;
            wr[j + 1] = EL(S, ldS, j + 1, j + 1);
            wi[j] = im;
            wi[j + 1] = -im;
            j += 2;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Elementary orthogonal transformations applied to the whole matrix.     */
/* ---------------------------------------------------------------------- */

/* The four loops below are the long ones (a whole row or column range of S,
 * or all rows of Q).  Built with -fopenmp (the CPU baseline's multi-core
 * timing only), each is split over the host cores when it is long; every
 * element is still computed by the same operations, so the result is
 * bitwise the same as the single-threaded build, where the pragmas are
 * ignored. */
#ifndef ORC_OMP_MIN
#define ORC_OMP_MIN 2048
#endif

/* Rotation G = [[c, -s], [s, c]] on index pair (i, i+1):
 *   rows    i, i+1 of A, columns [c0, c1):   [x; y] <- G^T [x; y]
 *   columns i, i+1 of A, rows    [r0, r1):   [x, y] <- [x, y] G      */
static void rot_rows(double *A, int ld, int i, int c0, int c1, double c, double s)
{
#pragma omp parallel for schedule(static) if (c1 - c0 >= ORC_OMP_MIN)
    for (int k = c0; k < c1; ++k) {
        double x = EL(A, ld, i, k), y = EL(A, ld, i + 1, k);
        EL(A, ld, i, k) = c * x + s * y;
        EL(A, ld, i + 1, k) = c * y - s * x;
    }
}

static void rot_cols(double *A, int ld, int i, int r0, int r1, double c, double s)
{
#pragma omp parallel for schedule(static) if (r1 - r0 >= ORC_OMP_MIN)
    for (int k = r0; k < r1; ++k) {
        double x = EL(A, ld, k, i), y = EL(A, ld, k, i + 1);
        EL(A, ld, k, i) = c * x + s * y;
        EL(A, ld, k, i + 1) = c * y - s * x;
    }
}

/* Householder reflector H = I - tau v v^T on indices [i, i+len), v[0..len).
 * H is symmetric, so left and right application use the same H. */
static void house_rows(double *A, int ld, int i, int len, const double *v, double tau,
                       int c0, int c1)
{
#pragma omp parallel for schedule(static) if (c1 - c0 >= ORC_OMP_MIN)
    for (int k = c0; k < c1; ++k) {
        double w = 0.0;
        for (int t = 0; t < len; ++t) w += v[t] * EL(A, ld, i + t, k);
        w *= tau;
        for (int t = 0; t < len; ++t) EL(A, ld, i + t, k) -= w * v[t];
    }
}

static void house_cols(double *A, int ld, int i, int len, const double *v, double tau,
                       int r0, int r1)
{
#pragma omp parallel for schedule(static) if (r1 - r0 >= ORC_OMP_MIN)
    for (int k = r0; k < r1; ++k) {
        double w = 0.0;
        for (int t = 0; t < len; ++t) w += EL(A, ld, k, i + t) * v[t];
        w *= tau;
        for (int t = 0; t < len; ++t) EL(A, ld, k, i + t) -= w * v[t];
    }
}

/* Reflector that maps x (length len) onto beta e_t:
 *   (I - tau v v^T) x = beta e_t,  v[t] = 1.
 * If x is already a multiple of e_t, tau = 0 (H = I). */
static void house_gen(int len, const double *x, int t, double *v, double *tau)
{
    double alpha = x[t], sigma = 0.0;
    for (int i = 0; i < len; ++i)
        if (i != t) sigma += x[i] * x[i];
    for (int i = 0; i < len; ++i) v[i] = x[i];
    v[t] = 1.0;
    if (sigma == 0.0) {
        *tau = 0.0;
        return;
    }
    double norm = sqrt(alpha * alpha + sigma);
    double beta = alpha >= 0.0 ? -norm : norm;
    double d = alpha - beta;
    for (int i = 0; i < len; ++i)
        if (i != t) v[i] = x[i] / d;
    *tau = (beta - alpha) / beta;
}

/* ---------------------------------------------------------------------- */
/* Small Sylvester equation  T11 X - X T22 = gamma T12,  p, q in {1, 2}.  */
/* ---------------------------------------------------------------------- */

/* Kronecker form: unknown x_(i + p k) = X[i][k];
 *   K[(i,k),(l,m)] = T11[i][l] delta(k,m) - delta(i,l) T22[m][k].
 * Gaussian elimination with complete pivoting; pivots smaller than
 * smin = max(eps max|K|, smallest normal) are replaced by smin, and gamma
 * (<= 1) scales the right-hand side so that no division overflows.
 * Matrices are column-major with the given leading dimension. Returns 1 if
 * a pivot was perturbed, else 0. */
int orc_sylvester(int p, int q, const double *T11, int ld11, const double *T22, int ld22,
                  const double *T12, int ld12, double *X, int ldX, double *gamma)
{
    int N = p * q;
    double K[4][4], b[4];
    int colperm[4];
    double kmax = 0.0;
    for (int k = 0; k < q; ++k)
        for (int i = 0; i < p; ++i) {
            int r = i + p * k;
            b[r] = EL(T12, ld12, i, k);
            for (int m = 0; m < q; ++m)
                for (int l = 0; l < p; ++l) {
                    int c = l + p * m;
                    double v = 0.0;
                    if (k == m) v += EL(T11, ld11, i, l);
                    if (i == l) v -= EL(T22, ld22, m, k);
                    K[r][c] = v;
                    if (fabs(v) > kmax) kmax = fabs(v);
                }
        }
    for (int c = 0; c < N; ++c) colperm[c] = c;
    double smin = ORC_EPS * kmax;
    if (smin < ORC_SMALL) smin = ORC_SMALL;
    int perturbed = 0;
    for (int s = 0; s < N; ++s) {
        int pr = s, pc = s;
        double best = -1.0;
        for (int r = s; r < N; ++r)
            for (int c = s; c < N; ++c)
                if (fabs(K[r][c]) > best) {
                    best = fabs(K[r][c]);
                    pr = r;
                    pc = c;
                }
        if (pr != s) {
            for (int c = 0; c < N; ++c) {
                double t = K[s][c]; K[s][c] = K[pr][c]; K[pr][c] = t;
            }
            double t = b[s]; b[s] = b[pr]; b[pr] = t;
        }
        if (pc != s) {
            for (int r = 0; r < N; ++r) {
                double t = K[r][s]; K[r][s] = K[r][pc]; K[r][pc] = t;
            }
            int t = colperm[s]; colperm[s] = colperm[pc]; colperm[pc] = t;
        }
        if (fabs(K[s][s]) < smin) {
            K[s][s] = smin;
            perturbed = 1;
        }
        for (int r = s + 1; r < N; ++r) {
            double f = K[r][s] / K[s][s];
            K[r][s] = 0.0;
            for (int c = s + 1; c < N; ++c) K[r][c] -= f * K[s][c];
            b[r] -= f * b[s];
        }
    }
    /* back substitution with overflow guard */
    double g = 1.0, y[4];
    const double big = DBL_MAX / 4.0;
    for (int s = N - 1; s >= 0; --s) {
        double acc = b[s];
        for (int c = s + 1; c < N; ++c) acc -= K[s][c] * y[c];
        double piv = fabs(K[s][s]);
        if (piv < 1.0 && fabs(acc) > big * piv) {
            double f = (big * piv) / fabs(acc);
            for (int c = 0; c < N; ++c) b[c] *= f;
            for (int c = s + 1; c < N; ++c) y[c] *= f;
            acc *= f;
            g *= f;
        }
        y[s] = acc / K[s][s];
    }
    for (int c = 0; c < N; ++c) {
        int u = colperm[c];
        EL(X, ldX, u % p, u / p) = y[c];
    }
    *gamma = g;
    return perturbed;
}

/* ---------------------------------------------------------------------- */
/* Standardization of a 2x2 diagonal block.                               */
/* ---------------------------------------------------------------------- */

/* Rotation Z = [[c, -s], [s, c]] such that Z^T M Z is either
 *   [[a', b'], [c', a']] with b'c' < 0   (complex pair), or
 *   upper triangular                      (real pair; the block splits).
 * M = [[m11, m12], [m21, m22]]. Writes the new block to out[4] (column-major)
 * with its diagonal made exactly equal, or its (2,1) entry exactly zero. */
void orc_std2(double m11, double m12, double m21, double m22,
              double *cs, double *sn, double *out)
{
    double c = 1.0, s = 0.0;
    double n11, n12, n21, n22;
    int real_case = 0;
    if (m21 == 0.0) {
        c = 1.0; s = 0.0;
        real_case = 1;
    } else if (m12 == 0.0) {
        c = 0.0; s = 1.0;
        real_case = 1;
    } else {
        double p = 0.5 * (m11 - m22);
        double disc = p * p + m12 * m21;
        if (disc >= 0.0) {
            /* real eigenvalues: Schur vector (lambda - m22, m21) with
             * lambda = (m11 + m22)/2 + sign(p) sqrt(disc) */
            double r = sqrt(disc);
            double x1 = p >= 0.0 ? p + r : p - r;
            double x2 = m21;
            double h = hypot(x1, x2);
            c = x1 / h;
            s = x2 / h;
            real_case = 1;
        } else {
            /* complex pair: equalize the diagonal,
             * cos2t (m11 - m22) + sin2t (m12 + m21) = 0 */
            double sig = m12 + m21;
            double r2 = hypot(2.0 * p, sig);
            if (r2 == 0.0) {
                c = 1.0; s = 0.0;
            } else {
                double sg = sig >= 0.0 ? 1.0 : -1.0;
                double cos2 = sg * sig / r2;
                double sin2 = -sg * 2.0 * p / r2;
                c = sqrt(0.5 * (1.0 + cos2));
                s = sin2 / (2.0 * c);
            }
        }
    }
    /* N = Z^T M Z */
    double a11 = c * m11 + s * m21, a12 = c * m12 + s * m22;   /* Z^T M */
    double a21 = c * m21 - s * m11, a22 = c * m22 - s * m12;
    n11 = a11 * c + a12 * s;
    n12 = a12 * c - a11 * s;
    n21 = a21 * c + a22 * s;
    n22 = a22 * c - a21 * s;
    if (real_case) {
        n21 = 0.0;
    } else {
        double avg = 0.5 * (n11 + n22);
        n11 = avg;
        n22 = avg;
        if (!(n12 * n21 < 0.0)) {
            /* rounding made the pair real: triangularize the new block */
            double c2, s2, o2[4];
            orc_std2(n11, n12, n21, n22, &c2, &s2, o2);
            /* compose Z <- Z Z2 */
            double cc = c * c2 - s * s2, ss = s * c2 + c * s2;
            c = cc; s = ss;
            n11 = o2[0]; n21 = o2[1]; n12 = o2[2]; n22 = o2[3];
        }
    }
    *cs = c;
    *sn = s;
    out[0] = n11; out[1] = n21; out[2] = n12; out[3] = n22;
}

/* Standardize the 2x2 block at j of the whole matrix (and Q). */
static void standardize_block(int n, double *S, int ldS, double *Q, int ldQ, int j)
{
    double c, s, blk[4];
    orc_std2(EL(S, ldS, j, j), EL(S, ldS, j, j + 1), EL(S, ldS, j + 1, j),
             EL(S, ldS, j + 1, j + 1), &c, &s, blk);
    rot_rows(S, ldS, j, j + 2, n, c, s);
    rot_cols(S, ldS, j, 0, j, c, s);
    if (Q) rot_cols(Q, ldQ, j, 0, n, c, s);
    EL(S, ldS, j, j) = blk[0];
    EL(S, ldS, j + 1, j) = blk[1];
    EL(S, ldS, j, j + 1) = blk[2];
    EL(S, ldS, j + 1, j + 1) = blk[3];
}

/* ---------------------------------------------------------------------- */
/* Swap of two adjacent diagonal blocks.                                  */
/* ---------------------------------------------------------------------- */

/* Swap the p x p block at j with the q x q block at j+p (p, q in {1,2}).
 * strong != 0 enables the strong stability test in addition to the weak
 * one.  Returns 0 if the swap was applied, 1 if it was rejected (S and Q
 * are then unchanged). */
int orc_swap(int n, double *S, int ldS, double *Q, int ldQ, int j, int p, int q, int strong)
{
    int k = p + q;
    if (k == 2) {
        /* two 1x1 blocks: the rotation whose first column is the
         * eigenvector (t12, t22 - t11) of the eigenvalue t22 */
        double t11 = EL(S, ldS, j, j), t12 = EL(S, ldS, j, j + 1);
        double t22 = EL(S, ldS, j + 1, j + 1);
        if (t11 == t22) return 0; /* equal eigenvalues: already in order */
        double h = hypot(t12, t22 - t11);
        double c = t12 / h, s = (t22 - t11) / h;
        rot_rows(S, ldS, j, j + 2, n, c, s);
        rot_cols(S, ldS, j, 0, j, c, s);
        if (Q) rot_cols(Q, ldQ, j, 0, n, c, s);
        /* new block [[t22, t12'], [0, t11]] with t12' = (G^T D G)_{12},
         * D = [[t11, t12], [0, t22]]; row 1 of G^T D is (c t11, c t12 + s t22) */
        double a11 = c * t11, a12 = c * t12 + s * t22;
        double t12n = a12 * c - a11 * s;
        EL(S, ldS, j, j) = t22;
        EL(S, ldS, j + 1, j + 1) = t11;
        EL(S, ldS, j + 1, j) = 0.0;
        EL(S, ldS, j, j + 1) = t12n;
        return 0;
    }

    double D[16], Dt[16];   /* local copies, column-major 4x4 (ld 4) */
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) D[c * 4 + r] = EL(S, ldS, j + r, j + c);
    double dnorm = 0.0;
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r)
            if (fabs(D[c * 4 + r]) > dnorm) dnorm = fabs(D[c * 4 + r]);
    double thresh = 10.0 * ORC_EPS * dnorm;
    if (thresh < ORC_SMALL) thresh = ORC_SMALL;

    /* Sylvester solve  T11 X - X T22 = gamma T12 */
    double X[4], gamma;
    orc_sylvester(p, q, &D[0], 4, &D[p * 4 + p], 4, &D[p * 4], 4, X, 2, &gamma);

    /* Reflectors spanning [-X; gamma I] (leading q columns of Qs). */
    double v1[4], v2[4], tau1 = 0.0, tau2 = 0.0;
    int nref;
    if (p == 2 && q == 1) {
        double x[3] = {-X[0], -X[1], gamma};
        house_gen(3, x, 0, v1, &tau1);
        nref = 1;
    } else if (p == 1 && q == 2) {
        /* u = (gamma, X11, X12) is orthogonal to both columns of
         * [-X; gamma I]; a reflector sending u to e_3 has its last column
         * along u and its first two spanning the subspace. */
        double u[3] = {gamma, X[0], X[2]};
        house_gen(3, u, 2, v1, &tau1);
        nref = 1;
    } else {
        /* p = q = 2: Householder QR of the 4x2 matrix M = [-X; gamma I] */
        double M[8] = {-X[0], -X[1], gamma, 0.0, -X[2], -X[3], 0.0, gamma};
        house_gen(4, M, 0, v1, &tau1);
        double w = 0.0;
        for (int t = 0; t < 4; ++t) w += v1[t] * M[4 + t];
        w *= tau1;
        for (int t = 0; t < 4; ++t) M[4 + t] -= w * v1[t];
        house_gen(3, &M[5], 0, v2, &tau2);
        nref = 2;
    }

    /* Dt = Qs^T D Qs, Qs = H1 (H2 acting on rows/cols 1..3) */
    memcpy(Dt, D, sizeof D);
    house_rows(Dt, 4, 0, (p == 2 && q == 2) ? 4 : 3, v1, tau1, 0, k);
    house_cols(Dt, 4, 0, (p == 2 && q == 2) ? 4 : 3, v1, tau1, 0, k);
    if (nref == 2) {
        house_rows(Dt, 4, 1, 3, v2, tau2, 0, k);
        house_cols(Dt, 4, 1, 3, v2, tau2, 0, k);
    }

    /* weak test: the block that must vanish, rows [q,k) x cols [0,q) */
    double lower = 0.0;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r)
            if (fabs(Dt[c * 4 + r]) > lower) lower = fabs(Dt[c * 4 + r]);
    if (lower > thresh) return 1;

    /* zero it, then the strong test: D - Qs Dt0 Qs^T must be small */
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) Dt[c * 4 + r] = 0.0;
    if (strong) {
        double E[16];
        memcpy(E, Dt, sizeof E);
        if (nref == 2) {
            house_rows(E, 4, 1, 3, v2, tau2, 0, k);
            house_cols(E, 4, 1, 3, v2, tau2, 0, k);
        }
        house_rows(E, 4, 0, (p == 2 && q == 2) ? 4 : 3, v1, tau1, 0, k);
        house_cols(E, 4, 0, (p == 2 && q == 2) ? 4 : 3, v1, tau1, 0, k);
        double err = 0.0;
        for (int c = 0; c < k; ++c)
            for (int r = 0; r < k; ++r) {
                double e = fabs(E[c * 4 + r] - D[c * 4 + r]);
                if (e > err) err = e;
            }
        if (err > thresh) return 1;
    }

    /* accepted: apply the reflectors to the rest of S and to Q */
    int len1 = (p == 2 && q == 2) ? 4 : 3;
    house_rows(S, ldS, j, len1, v1, tau1, j + k, n);
    house_cols(S, ldS, j, len1, v1, tau1, 0, j);
    if (Q) house_cols(Q, ldQ, j, len1, v1, tau1, 0, n);
    if (nref == 2) {
        house_rows(S, ldS, j + 1, 3, v2, tau2, j + k, n);
        house_cols(S, ldS, j + 1, 3, v2, tau2, 0, j);
        if (Q) house_cols(Q, ldQ, j + 1, 3, v2, tau2, 0, n);
    }
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) EL(S, ldS, j + r, j + c) = Dt[c * 4 + r];
    /* 1x1 blocks keep an exact zero below them */
    if (q == 1 && p == 2) { /* new order: 1x1 at j, 2x2 at j+1 */
        EL(S, ldS, j + 1, j) = 0.0;
    }
    if (q == 2 && p == 1) { /* new order: 2x2 at j, 1x1 at j+2 */
        EL(S, ldS, j + 2, j + 1) = 0.0;
        EL(S, ldS, j + 2, j) = 0.0;
    }
    /* restore the standard form of the new 2x2 blocks */
    if (q == 2) standardize_block(n, S, ldS, Q, ldQ, j);
    if (p == 2) standardize_block(n, S, ldS, Q, ldQ, j + q);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Reordering.                                                            */
/* ---------------------------------------------------------------------- */

/*
 * Reorder S (n x n, column-major, leading dimension ldS) so that the
 * selected eigenvalues lead.  select[i] != 0 selects the eigenvalue at
 * diagonal position i; a 2x2 block is selected if either of its positions
 * is.  Selected blocks keep their relative order, and so do unselected ones.
 * Q (nullable) is overwritten by Q Q3.
 *
 * abort_on_reject != 0: stop at the first rejected swap (S, Q partially
 * reordered).  Otherwise the rejected block stays where it is and later
 * selected blocks stop below it.
 *
 * Outputs (nullable): wr, wi eigenvalues of the result; *m the number of
 * selected eigenvalues; *nswaps successful swaps; *nrej rejected swaps;
 * selout[n] the final per-position selection flags.
 * Returns the number of rejected swaps (>= 0), -1 if n < 0 or ldS < n,
 * -2 if S is not in standard real Schur form, -3 if out of memory,
 * -4 if ldQ < n.
 */
int orc_reorder(int n, double *S, int ldS, double *Q, int ldQ, const int *select,
                double *wr, double *wi, int *m, int abort_on_reject, int strong,
                long long *nswaps, long long *nrej, unsigned char *selout)
{
    if (n < 0 || ldS < (n > 1 ? n : 1)) return -1;
    if (Q && ldQ < (n > 1 ? n : 1)) return -4;
    if (orc_validate(n, S, ldS) != 0) return -2;
    long long swaps = 0, rej = 0;
    if (n == 0) {
        if (m) *m = 0;
        if (nswaps) *nswaps = 0;
        if (nrej) *nrej = 0;
        return 0;
    }
    unsigned char *sel = (unsigned char *)malloc((size_t)n);
    if (!sel) return -3;
    for (int i = 0; i < n; ++i) sel[i] = select[i] ? 1 : 0;
    for (int j = 0; j < n;) {
        if (block_size(n, S, ldS, j) == 2) {
            unsigned char s2 = sel[j] | sel[j + 1];
            sel[j] = sel[j + 1] = s2;
            j += 2;
        } else {
            j += 1;
        }
    }
    int msel = 0;
    for (int i = 0; i < n; ++i) msel += sel[i];

    int ks = 0;
    for (;;) {
        int pos = ks;
        while (pos < n && !sel[pos]) pos += block_size(n, S, ldS, pos);
        if (pos >= n) break;
        if (pos == ks) {
            ks += block_size(n, S, ldS, ks);
            continue;
        }
        int here = pos, ok = 1;
        while (here > ks) {
            int q = block_size(n, S, ldS, here);
            int pa = (here - 2 >= ks && EL(S, ldS, here - 1, here - 2) != 0.0) ? 2 : 1;
            int j = here - pa;
            if (orc_swap(n, S, ldS, Q, ldQ, j, pa, q, strong) != 0) {
                ok = 0;
                ++rej;
                break;
            }
            ++swaps;
            for (int i = j; i < j + q; ++i) sel[i] = 1;
            for (int i = j + q; i < j + q + pa; ++i) sel[i] = 0;
            here = j;
        }
        if (!ok && abort_on_reject) break;
        ks = here + block_size(n, S, ldS, here);
    }
    if (wr && wi) orc_eigenvalues(n, S, ldS, wr, wi);
    if (selout) memcpy(selout, sel, (size_t)n);
    free(sel);
    if (m) *m = msel;
    if (nswaps) *nswaps = swaps;
    if (nrej) *nrej = rej;
    return (int)rej;
}
