/*
 * Plain CPU oracle for generalized real Schur-form eigenvalue reordering.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  It shares no code, header, table
 * or helper with the GPU library (nor with the standard-form oracle: the
 * file compiles on its own), and the GPU library never calls it.
 *
 * What it computes (Section 2, Eq. 7, second form): given a matrix pair
 * (S, T) in generalized real Schur form -- S upper quasi-triangular with 1x1
 * and 2x2 diagonal blocks, a 2x2 block carrying a complex-conjugate pair of
 * generalized eigenvalues, T upper triangular -- orthogonal Q, Z and a
 * selection, orthogonal Q3, Z3 such that (S_hat, T_hat) = Q3^T (S, T) Z3 is
 * again in that form with the selected eigenvalues in its leading diagonal
 * blocks; (S, T) is overwritten by (S_hat, T_hat), Q by Q Q3 and Z by Z Z3.
 *
 * How (Section 3.2, Fig. 1a, "scalar updates", as for the standard form):
 * every selected block is moved up by swaps with the block directly above
 * it, top to bottom, and each swap's orthogonal transformations are applied
 * at once to the whole rows/columns of S and T and to the columns of Q, Z.
 *
 * The paper leaves the swap of a matrix pair to the cited works.  The swap
 * here is the direct method (a generalized Sylvester solve), written from
 * its mathematics.  For D = (A, B) = the k x k diagonal part of (S, T)
 * holding the p x p block (A11, B11) above the q x q block (A22, B22):
 *
 *   A11 R - L A22 = -gamma A12,   B11 R - L B22 = -gamma B12
 *
 * gives A [R; gamma I] = [L; gamma I] A22 and B [R; gamma I] = [L; gamma I]
 * B22, so orthogonal Qs, Zs whose leading q columns span [L; gamma I] and
 * [R; gamma I] move (A22, B22) to the top: Qs^T (A, B) Zs is block upper
 * triangular with the q x q block first.  Qs and Zs are the orthogonal
 * factors of Householder QR factorizations of those k x q matrices.
 *
 *   - weak test: the lower-left (k-q) x q block of Qs^T A Zs and of
 *     Qs^T B Zs has magnitude <= 20 eps ||A||_F (resp. ||B||_F);
 *   - strong test: after zeroing that block, A - Qs (Qs^T A Zs) Zs^T and the
 *     same for B stay below the same thresholds (max norm);
 *   - T stays upper triangular: each new 2x2 diagonal block of T is made
 *     upper triangular by one rotation of its two columns (folded into Zs);
 *   - a rejected swap changes nothing; two 1x1 blocks with equal generalized
 *     eigenvalues (a11 b22 == a22 b11) are already in order.
 *
 * Floating point: IEEE binary64, round to nearest, built with
 * -ffp-contract=off (no fused multiply-add).
 */
#include <float.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define G_EPS DBL_EPSILON
#define G_SMALL DBL_MIN

#define EL(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* Size of the diagonal block of the pair starting at position j. */
static int gblock(int n, const double *S, int ldS, int j)
{
    return (j + 1 < n && EL(S, ldS, j + 1, j) != 0.0) ? 2 : 1;
}

/* Coefficients of det(Sb - lambda Tb) = a lambda^2 - b lambda + c for the
 * 2x2 block at j (Tb upper triangular). */
static void pencil2(const double *S, int ldS, const double *T, int ldT, int j,
                    double *a, double *b, double *c)
{
    double s11 = EL(S, ldS, j, j), s12 = EL(S, ldS, j, j + 1);
    double s21 = EL(S, ldS, j + 1, j), s22 = EL(S, ldS, j + 1, j + 1);
    double t11 = EL(T, ldT, j, j), t12 = EL(T, ldT, j, j + 1), t22 = EL(T, ldT, j + 1, j + 1);
    *a = t11 * t22;
    *b = s11 * t22 + s22 * t11 - s21 * t12;
    *c = s11 * s22 - s12 * s21;
}

/* 0 if (S, T) is in generalized real Schur form, else -(1 + first bad
 * column): S zero below its subdiagonal, no two adjacent subdiagonal
 * nonzeros, T zero below its diagonal, and every 2x2 block of the pair with
 * a complex-conjugate pair (b^2 < 4 a c). */
int orc_gen_validate(int n, const double *S, int ldS, const double *T, int ldT)
{
    for (int j = 0; j < n; ++j) {
        for (int i = j + 2; i < n; ++i)
            if (EL(S, ldS, i, j) != 0.0) return -(1 + j);
        for (int i = j + 1; i < n; ++i)
            if (EL(T, ldT, i, j) != 0.0) return -(1 + j);
        if (j + 1 < n && EL(S, ldS, j + 1, j) != 0.0) {
            if (j + 2 < n && EL(S, ldS, j + 2, j + 1) != 0.0) return -(1 + j);
            double a, b, c;
            pencil2(S, ldS, T, ldT, j, &a, &b, &c);
            if (!(b * b < 4.0 * a * c)) return -(1 + j);
        }
    }
    return 0;
}

/* Generalized eigenvalues lambda = alpha / beta from the diagonal blocks: a
 * 1x1 block gives s / t (+-inf if t = 0); a 2x2 block the roots of
 * a lambda^2 - b lambda + c, b / 2a +- i sqrt(4ac - b^2) / 2|a|, the one with
 * positive imaginary part first (a real pair, possible only after rounding
 * in a swap, gives its two real roots, larger first). */
void orc_gen_eigenvalues(int n, const double *S, int ldS, const double *T, int ldT,
                         double *wr, double *wi)
{
    int j = 0;
    while (j < n) {
        if (gblock(n, S, ldS, j) == 1) {
            wr[j] = EL(S, ldS, j, j) / EL(T, ldT, j, j);
            wi[j] = 0.0;
            j += 1;
        } else {
            double a, b, c;
            pencil2(S, ldS, T, ldT, j, &a, &b, &c);
            double d = 4.0 * a * c - b * b;
            if (d > 0.0) {
                double re = b / (2.0 * a), im = sqrt(d) / (2.0 * fabs(a));
                wr[j] = re; wi[j] = im;
                wr[j + 1] = re; wi[j + 1] = -im;
            } else {
                double r = sqrt(-d) / (2.0 * fabs(a)), m = b / (2.0 * a);
                wr[j] = m + r; wi[j] = 0.0;
                wr[j + 1] = m - r; wi[j + 1] = 0.0;
            }
            j += 2;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Generalized Sylvester equation, p, q in {1, 2}.                        */
/* ---------------------------------------------------------------------- */

/*
 * A11 R - L A22 = -gamma A12,  B11 R - L B22 = -gamma B12  for R, L (p x q).
 * D holds the k x k diagonal part (column-major, ld 4) of A (DA) and B (DB).
 * Kronecker form with unknowns x = [vec R; vec L] (column-major vec) and
 * equations [vec of the first; vec of the second]:
 *   row (i, c) of the first:  sum_l A11[i][l] R[l][c] - sum_m L[i][m] A22[m][c]
 * Gaussian elimination with complete pivoting; pivots below
 * smin = max(eps max|K|, smallest normal) are replaced by smin and gamma
 * (<= 1) scales the right-hand side so that no division overflows.  Writes
 * R and L column-major (ld p) and returns gamma.
 */
double orc_gen_sylvester(int p, int q, const double *DA, const double *DB, double *R, double *L)
{
    const int pq = p * q, N = 2 * pq;
    double K[8][8], b[8];
    int colperm[8];
    double kmax = 0.0;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) K[r][c] = 0.0;
    for (int e = 0; e < 2; ++e) {
        const double *D = e ? DB : DA;
        for (int c = 0; c < q; ++c)
            for (int i = 0; i < p; ++i) {
                const int row = e * pq + i + p * c;
                b[row] = -D[(p + c) * 4 + i];               /* -X12[i][c] */
                for (int l = 0; l < p; ++l)                 /* X11[i][l] R[l][c] */
                    K[row][l + p * c] += D[l * 4 + i];
                for (int m = 0; m < q; ++m)                 /* -L[i][m] X22[m][c] */
                    K[row][pq + i + p * m] -= D[(p + c) * 4 + p + m];
            }
    }
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c)
            if (fabs(K[r][c]) > kmax) kmax = fabs(K[r][c]);
    for (int c = 0; c < N; ++c) colperm[c] = c;
    double smin = G_EPS * kmax;
    if (smin < G_SMALL) smin = G_SMALL;
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
        if (fabs(K[s][s]) < smin) K[s][s] = smin;
        for (int r = s + 1; r < N; ++r) {
            double f = K[r][s] / K[s][s];
            K[r][s] = 0.0;
            for (int c = s + 1; c < N; ++c) K[r][c] -= f * K[s][c];
            b[r] -= f * b[s];
        }
    }
    double g = 1.0, y[8];
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
        const int u = colperm[c];
        if (u < pq) R[u] = y[c];
        else L[u - pq] = y[c];
    }
    return g;
}

/* ---------------------------------------------------------------------- */
/* Orthogonal factors.                                                    */
/* ---------------------------------------------------------------------- */

/* Reflector I - tau v v^T (v[0] = 1) mapping x (length len) onto beta e_0;
 * tau = 0 if x is already a multiple of e_0. */
static void house0(int len, const double *x, double *v, double *tau)
{
    double alpha = x[0], sigma = 0.0;
    for (int i = 1; i < len; ++i) sigma += x[i] * x[i];
    v[0] = 1.0;
    for (int i = 1; i < len; ++i) v[i] = x[i];
    if (sigma == 0.0) {
        *tau = 0.0;
        return;
    }
    double norm = sqrt(alpha * alpha + sigma);
    double beta = alpha >= 0.0 ? -norm : norm;
    double d = alpha - beta;
    for (int i = 1; i < len; ++i) v[i] = x[i] / d;
    *tau = (beta - alpha) / beta;
}

/* Orthogonal factor (k x k, column-major, ld 4) of the Householder QR of the
 * k x q matrix [X; gamma I] (X p x q, ld p): H1 for column 0, then H2 on
 * rows 1..k-1 for column 1 (q = 2).  Its leading q columns span [X; gamma I]. */
static void qr_factor(int p, int q, const double *X, double gamma, double *Qo)
{
    const int k = p + q;
    double M[4][2];
    for (int c = 0; c < q; ++c) {
        for (int i = 0; i < p; ++i) M[i][c] = X[i + p * c];
        for (int i = 0; i < q; ++i) M[p + i][c] = (i == c) ? gamma : 0.0;
    }
    double v1[4], v2[4], tau1, tau2 = 0.0, x[4];
    for (int i = 0; i < k; ++i) x[i] = M[i][0];
    house0(k, x, v1, &tau1);
    if (q == 2) {
        double w = 0.0;
        for (int i = 0; i < k; ++i) w += v1[i] * M[i][1];
        w *= tau1;
        for (int i = 0; i < k; ++i) M[i][1] -= w * v1[i];
        for (int i = 1; i < k; ++i) x[i - 1] = M[i][1];
        house0(k - 1, x, v2, &tau2);
    }
    /* Qo = H1 diag(1, H2): start from I, apply diag(1, H2) then H1 on the left */
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) Qo[c * 4 + r] = (r == c) ? 1.0 : 0.0;
    if (q == 2)
        for (int c = 0; c < k; ++c) {
            double w = 0.0;
            for (int i = 1; i < k; ++i) w += v2[i - 1] * Qo[c * 4 + i];
            w *= tau2;
            for (int i = 1; i < k; ++i) Qo[c * 4 + i] -= w * v2[i - 1];
        }
    for (int c = 0; c < k; ++c) {
        double w = 0.0;
        for (int i = 0; i < k; ++i) w += v1[i] * Qo[c * 4 + i];
        w *= tau1;
        for (int i = 0; i < k; ++i) Qo[c * 4 + i] -= w * v1[i];
    }
}

/* C = op(X) Y Z-ish helpers on k x k blocks, column-major ld 4. */
static void mul_tn(int k, const double *X, const double *Y, double *C)   /* C = X^T Y */
{
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += X[r * 4 + t] * Y[c * 4 + t];
            C[c * 4 + r] = s;
        }
}

static void mul_nn(int k, const double *X, const double *Y, double *C)   /* C = X Y */
{
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += X[t * 4 + r] * Y[c * 4 + t];
            C[c * 4 + r] = s;
        }
}

static void mul_nt(int k, const double *X, const double *Y, double *C)   /* C = X Y^T */
{
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += X[t * 4 + r] * Y[t * 4 + c];
            C[c * 4 + r] = s;
        }
}

/* Rotation of columns c0, c0+1 of the k x k block M (ld 4):
 * [x, y] <- [x, y] [[c, -s], [s, c]]. */
static void rot_cols4(int k, double *M, int c0, double c, double s)
{
    for (int r = 0; r < k; ++r) {
        double x = M[c0 * 4 + r], y = M[(c0 + 1) * 4 + r];
        M[c0 * 4 + r] = c * x + s * y;
        M[(c0 + 1) * 4 + r] = c * y - s * x;
    }
}

/* ---------------------------------------------------------------------- */
/* Swap of two adjacent diagonal blocks of the pair.                      */
/* ---------------------------------------------------------------------- */

/*
 * Computes the swap of the p x p block at j with the q x q block at j+p on
 * the k x k diagonal part only.  DA, DB: the k x k parts (ld 4).  On
 * acceptance fills Qs, Zs (k x k, ld 4) and the new diagonal parts NA, NB and
 * returns 0; returns 1 if a stability test rejects the swap.
 */
int orc_gen_swap_local(int p, int q, const double *DA, const double *DB, int strong, double *Qs,
                       double *Zs, double *NA, double *NB)
{
    const int k = p + q;
    double na = 0.0, nb = 0.0;
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) {
            na += DA[c * 4 + r] * DA[c * 4 + r];
            nb += DB[c * 4 + r] * DB[c * 4 + r];
        }
    double tha = 20.0 * G_EPS * sqrt(na), thb = 20.0 * G_EPS * sqrt(nb);
    if (tha < G_SMALL) tha = G_SMALL;
    if (thb < G_SMALL) thb = G_SMALL;

    double R[4], L[4];
    double gamma = orc_gen_sylvester(p, q, DA, DB, R, L);
    qr_factor(p, q, L, gamma, Qs);
    qr_factor(p, q, R, gamma, Zs);

    double W[16];
    mul_tn(k, Qs, DA, W);
    mul_nn(k, W, Zs, NA);
    mul_tn(k, Qs, DB, W);
    mul_nn(k, W, Zs, NB);

    double lowa = 0.0, lowb = 0.0;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) {
            if (fabs(NA[c * 4 + r]) > lowa) lowa = fabs(NA[c * 4 + r]);
            if (fabs(NB[c * 4 + r]) > lowb) lowb = fabs(NB[c * 4 + r]);
        }
    if (lowa > tha || lowb > thb) return 1;
    for (int c = 0; c < q; ++c)
        for (int r = q; r < k; ++r) NA[c * 4 + r] = NB[c * 4 + r] = 0.0;

    if (strong) {
        double E[16], V[16];
        for (int e = 0; e < 2; ++e) {
            const double *N0 = e ? NB : NA, *D = e ? DB : DA;
            mul_nn(k, Qs, N0, V);
            mul_nt(k, V, Zs, E);
            double err = 0.0;
            for (int c = 0; c < k; ++c)
                for (int r = 0; r < k; ++r)
                    if (fabs(E[c * 4 + r] - D[c * 4 + r]) > err) err = fabs(E[c * 4 + r] - D[c * 4 + r]);
            if (err > (e ? thb : tha)) return 1;
        }
    }

    /* T stays upper triangular: rotate the two columns of each new 2x2
     * block so that its (2,1) entry in T vanishes */
    for (int blk = 0; blk < 2; ++blk) {
        const int sz = blk ? p : q, c0 = blk ? q : 0;
        if (sz != 2) continue;
        double b10 = NB[c0 * 4 + c0 + 1], b11 = NB[(c0 + 1) * 4 + c0 + 1];
        if (b10 == 0.0) continue;
        double h = hypot(b10, b11);
        double c = b11 / h, s = -b10 / h;
        rot_cols4(k, NA, c0, c, s);
        rot_cols4(k, NB, c0, c, s);
        rot_cols4(k, Zs, c0, c, s);
        NB[c0 * 4 + c0 + 1] = 0.0;
    }
    return 0;
}

/* Swap on the whole pair: applies the local transformations to rows
 * [j, j+k) (columns to the right), columns [j, j+k) (rows above) of S and T,
 * and to the columns [j, j+k) of Q and Z (either may be NULL). */
int orc_gen_swap(int n, double *S, int ldS, double *T, int ldT, double *Q, int ldQ, double *Z,
                 int ldZ, int j, int p, int q, int strong)
{
    const int k = p + q;
    if (k == 2 && EL(S, ldS, j, j) * EL(T, ldT, j + 1, j + 1) ==
                      EL(S, ldS, j + 1, j + 1) * EL(T, ldT, j, j))
        return 0; /* equal eigenvalues: already in order */
    double DA[16], DB[16], Qs[16], Zs[16], NA[16], NB[16];
    for (int c = 0; c < k; ++c)
        for (int r = 0; r < k; ++r) {
            DA[c * 4 + r] = EL(S, ldS, j + r, j + c);
            DB[c * 4 + r] = EL(T, ldT, j + r, j + c);
        }
    if (orc_gen_swap_local(p, q, DA, DB, strong, Qs, Zs, NA, NB)) return 1;
    double x[4];
    for (int e = 0; e < 2; ++e) {
        double *A = e ? T : S;
        const int ld = e ? ldT : ldS;
        for (int c = j + k; c < n; ++c) {                 /* rows: A <- Qs^T A */
            for (int r = 0; r < k; ++r) {
                double s = 0.0;
                for (int t = 0; t < k; ++t) s += Qs[r * 4 + t] * EL(A, ld, j + t, c);
                x[r] = s;
            }
            for (int r = 0; r < k; ++r) EL(A, ld, j + r, c) = x[r];
        }
        for (int r = 0; r < j; ++r) {                     /* columns: A <- A Zs */
            for (int c = 0; c < k; ++c) {
                double s = 0.0;
                for (int t = 0; t < k; ++t) s += EL(A, ld, r, j + t) * Zs[c * 4 + t];
                x[c] = s;
            }
            for (int c = 0; c < k; ++c) EL(A, ld, r, j + c) = x[c];
        }
        const double *N = e ? NB : NA;
        for (int c = 0; c < k; ++c)
            for (int r = 0; r < k; ++r) EL(A, ld, j + r, j + c) = N[c * 4 + r];
    }
    for (int e = 0; e < 2; ++e) {
        double *X = e ? Z : Q;
        const int ld = e ? ldZ : ldQ;
        const double *F = e ? Zs : Qs;
        if (!X) continue;
        for (int r = 0; r < n; ++r) {
            for (int c = 0; c < k; ++c) {
                double s = 0.0;
                for (int t = 0; t < k; ++t) s += EL(X, ld, r, j + t) * F[c * 4 + t];
                x[c] = s;
            }
            for (int c = 0; c < k; ++c) EL(X, ld, r, j + c) = x[c];
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Reordering.                                                            */
/* ---------------------------------------------------------------------- */

/*
 * Reorder (S, T) so that the selected generalized eigenvalues lead.
 * select[i] != 0 selects the eigenvalue at diagonal position i; a 2x2 block
 * is selected if either of its positions is.  Selected blocks keep their
 * relative order, and so do unselected ones.  Q, Z (nullable) are
 * overwritten by Q Q3 and Z Z3.  A rejected swap leaves the block where it
 * is and later selected blocks stop below it.
 *
 * Outputs (nullable): wr, wi eigenvalues of the result; *m the number of
 * selected eigenvalues; *nswaps, *nrej accepted and rejected swaps.
 * Returns the number of rejected swaps (>= 0), -1 for a bad size or leading
 * dimension, -2 if (S, T) is not in generalized real Schur form, -3 if out
 * of memory.
 */
int orc_gen_reorder(int n, double *S, int ldS, double *T, int ldT, double *Q, int ldQ, double *Z,
                    int ldZ, const int *select, double *wr, double *wi, int *m, int strong,
                    long long *nswaps, long long *nrej)
{
    const int ld1 = n > 1 ? n : 1;
    if (n < 0 || ldS < ld1 || ldT < ld1 || (Q && ldQ < ld1) || (Z && ldZ < ld1)) return -1;
    if (orc_gen_validate(n, S, ldS, T, ldT) != 0) return -2;
    long long swaps = 0, rej = 0;
    unsigned char *sel = (unsigned char *)malloc((size_t)(n > 0 ? n : 1));
    if (!sel) return -3;
    for (int i = 0; i < n; ++i) sel[i] = select[i] ? 1 : 0;
    for (int j = 0; j < n;) {
        if (gblock(n, S, ldS, j) == 2) {
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
        while (pos < n && !sel[pos]) pos += gblock(n, S, ldS, pos);
        if (pos >= n) break;
        if (pos == ks) {
            ks += gblock(n, S, ldS, ks);
            continue;
        }
        int here = pos;
        while (here > ks) {
            const int q = gblock(n, S, ldS, here);
            const int pa = (here - 2 >= ks && EL(S, ldS, here - 1, here - 2) != 0.0) ? 2 : 1;
            const int j = here - pa;
            if (orc_gen_swap(n, S, ldS, T, ldT, Q, ldQ, Z, ldZ, j, pa, q, strong) != 0) {
                ++rej;
                break;
            }
            ++swaps;
            for (int i = j; i < j + q; ++i) sel[i] = 1;
            for (int i = j + q; i < j + q + pa; ++i) sel[i] = 0;
            here = j;
        }
        ks = here + gblock(n, S, ldS, here);
    }
    if (wr && wi) orc_gen_eigenvalues(n, S, ldS, T, ldT, wr, wi);
    free(sel);
    if (m) *m = msel;
    if (nswaps) *nswaps = swaps;
    if (nrej) *nrej = rej;
    return (int)rej;
}
