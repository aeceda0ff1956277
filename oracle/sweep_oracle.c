/*
 * CPU oracle for one bulge-chasing sweep of the Schur reduction.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only callers.  It shares no code with the GPU
 * library (nor with the other oracle files: it compiles on its own).
 *
 * What it computes (Section 3.2, "Bulge Chasing and Eigenvalue
 * Reordering"): one pipelined QR iteration on an upper Hessenberg matrix H.
 * A set of bulges, one per pair of shifts, is introduced at the top of H and
 * chased down the diagonal by overlapping 3x3 Householder reflectors; each
 * reflector P is applied as H <- P H P (P symmetric orthogonal) and
 * accumulated as Q <- Q P.  The result is again upper Hessenberg.
 *
 * The paper names the transformations only; the steps here are the
 * pipelined small-bulge sweep, written from its mathematics:
 *   - shifts come in pairs (two real shifts or a complex-conjugate pair),
 *     given by s = sigma1 + sigma2 and p = sigma1 sigma2 (both real);
 *   - at chase step tau, bulge j (j = 0 introduced first) sits at
 *     k_j = tau - 3 j - 1; within a step the bulges are processed from the
 *     lowest (j = 0) to the highest, so that each reflector's input column is
 *     untouched by the others of its step;
 *   - introduction (k = -1): the first column of (H - sigma1 I)(H - sigma2 I)
 *     has three nonzeros
 *         x0 = h00^2 + h01 h10 - s h00 + p,  x1 = h10 (h00 + h11 - s),
 *         x2 = h10 h21,
 *     and the reflector with P x = beta e_0 acts on rows / columns 0..2;
 *   - chase (0 <= k <= n - 3): the reflector maps H[k+1 .. k+3, k] (two
 *     entries at k = n - 3) onto beta e_0 and acts on rows / columns
 *     k+1 .. k+3; the entries it annihilates are set to exact zeros;
 *   - a reflector is applied to rows k+1..k+3 of H for columns max(k, 0) ..
 *     n-1, to columns k+1..k+3 for rows 0 .. min(k+4, n-1) (the other
 *     entries it could touch are zero), and to the columns of Q.
 * n < 3 is left unchanged.
 *
 * Floating point: IEEE binary64, round to nearest, -ffp-contract=off.
 */
#include <math.h>
#include <stddef.h>

#define EL(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* Reflector I - tau v v^T (v[0] = 1) mapping x (length len) onto beta e_0;
 * tau = 0 when x is already a multiple of e_0. */
static void refl(int len, const double *x, double *v, double *tau, double *beta)
{
    double alpha = x[0], sigma = 0.0;
    for (int i = 1; i < len; ++i) sigma += x[i] * x[i];
    v[0] = 1.0;
    for (int i = 1; i < len; ++i) v[i] = x[i];
    if (sigma == 0.0) {
        *tau = 0.0;
        *beta = alpha;
        return;
    }
    double norm = sqrt(alpha * alpha + sigma);
    double b = alpha >= 0.0 ? -norm : norm;
    double d = alpha - b;
    for (int i = 1; i < len; ++i) v[i] = x[i] / d;
    *tau = (b - alpha) / b;
    *beta = b;
}

/* Applies P = I - tau v v^T on the indices r0 .. r0+len-1: rows of H for
 * columns [c0, n), columns of H for rows [0, rend), columns of Q. */
static void apply(int n, double *H, int ldH, double *Q, int ldQ, int r0, int len, const double *v,
                  double tau, int c0, int rend)
{
    if (tau == 0.0) return;
    for (int c = c0; c < n; ++c) {
        double w = 0.0;
        for (int i = 0; i < len; ++i) w += v[i] * EL(H, ldH, r0 + i, c);
        w *= tau;
        for (int i = 0; i < len; ++i) EL(H, ldH, r0 + i, c) -= w * v[i];
    }
    for (int r = 0; r < rend; ++r) {
        double w = 0.0;
        for (int i = 0; i < len; ++i) w += EL(H, ldH, r, r0 + i) * v[i];
        w *= tau;
        for (int i = 0; i < len; ++i) EL(H, ldH, r, r0 + i) -= w * v[i];
    }
    if (Q)
        for (int r = 0; r < n; ++r) {
            double w = 0.0;
            for (int i = 0; i < len; ++i) w += EL(Q, ldQ, r, r0 + i) * v[i];
            w *= tau;
            for (int i = 0; i < len; ++i) EL(Q, ldQ, r, r0 + i) -= w * v[i];
        }
}

/* One step of bulge j at position k (see the file comment). */
static void bulge_step(int n, double *H, int ldH, double *Q, int ldQ, int k, double s, double p)
{
    double x[3], v[3], tau, beta;
    if (k < 0) {
        const double h00 = EL(H, ldH, 0, 0), h01 = EL(H, ldH, 0, 1), h10 = EL(H, ldH, 1, 0);
        const double h11 = EL(H, ldH, 1, 1), h21 = EL(H, ldH, 2, 1);
        x[0] = h00 * h00 + h01 * h10 - s * h00 + p;
        x[1] = h10 * (h00 + h11 - s);
        x[2] = h10 * h21;
        refl(3, x, v, &tau, &beta);
        apply(n, H, ldH, Q, ldQ, 0, 3, v, tau, 0, n < 4 ? n : 4);
        return;
    }
    const int len = (k + 3 <= n - 1) ? 3 : 2;
    for (int i = 0; i < len; ++i) x[i] = EL(H, ldH, k + 1 + i, k);
    refl(len, x, v, &tau, &beta);
    const int rend = (k + 5 < n) ? k + 5 : n;
    apply(n, H, ldH, Q, ldQ, k + 1, len, v, tau, k, rend);
    EL(H, ldH, k + 1, k) = beta;
    for (int i = 1; i < len; ++i) EL(H, ldH, k + 1 + i, k) = 0.0;
}

/*
 * One sweep on H (n x n upper Hessenberg, column-major, ldH) with nshifts
 * shifts sr[i] + i si[i] (nshifts even; the shifts of each pair are either
 * both real or complex conjugates).  Q (nullable) is overwritten by Q Q3.
 * Returns 0, -1 for a bad argument (n < 0, ldH < n, odd or negative
 * nshifts, a pair that is neither real nor conjugate), -2 if H is not upper
 * Hessenberg.
 */
int orc_qr_sweep(int n, double *H, int ldH, double *Q, int ldQ, int nshifts, const double *sr,
                 const double *si)
{
    if (n < 0 || ldH < (n > 1 ? n : 1) || nshifts < 0 || (nshifts & 1)) return -1;
    if (Q && ldQ < (n > 1 ? n : 1)) return -1;
    for (int j = 0; j < n; ++j)
        for (int i = j + 2; i < n; ++i)
            if (EL(H, ldH, i, j) != 0.0) return -2;
    const int nb = nshifts / 2;
    for (int b = 0; b < nb; ++b) {
        const double a1 = sr[2 * b], b1 = si[2 * b], a2 = sr[2 * b + 1], b2 = si[2 * b + 1];
        if (!((b1 == 0.0 && b2 == 0.0) || (a1 == a2 && b1 == -b2))) return -1;
    }
    if (n < 3 || nb == 0) return 0;
    const int last = (n - 3) + 3 * (nb - 1) + 1; /* the last bulge reaches k = n - 3 */
    for (int tau = 0; tau <= last; ++tau)
        for (int b = 0; b < nb; ++b) {
            const int k = tau - 3 * b - 1;
            if (k < -1 || k > n - 3) continue;
            const double s = sr[2 * b] + sr[2 * b + 1];
            const double p = sr[2 * b] * sr[2 * b + 1] - si[2 * b] * si[2 * b + 1];
            bulge_step(n, H, ldH, Q, ldQ, k, s, p);
        }
    return 0;
}
