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
// same step (8 lanes compute one swap, the octets of a warp on swaps of one
// size), then the left transformations (rows of S and T) and the right ones
// (columns of S and T, the columns of the accumulators UQ and UZ) are
// applied by all warps, split among the swap sizes by their work.
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
// of S and T (column c keeps rows 0..c+1), a 128-double scratch per swap
// slot (gen_swap_octet: its Qs and Zs stay there for the updates).
constexpr int GSLOT = 128;
constexpr size_t kGenWindowSmem =
    sizeof(double) * (2 * (size_t)GW * GW + 2 * (size_t)gpoff(GW) + 2 * (size_t)GMAXSW * GSLOT) +
    sizeof(int) * 2 * 3 * GMAXSW + 2 * GW;

// |x| order through the bit pattern: for non-negative doubles the integer
// order of the bits is the numeric order (integer compares, no FP64 issue).
__device__ __forceinline__ unsigned long long mag(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// ---------------------------------------------------------------------------
// Swap of one pair of adjacent blocks by an octet: 8 lanes of a warp.
//
// An FP64 instruction costs the same issue slot for 1 or 32 active lanes, so
// the swap's arithmetic is spread over 8 lanes instead of running on one:
//   - the Kronecker system (N = 2pq <= 8 unknowns): lane r owns row r;
//     complete pivoting by an octet arg-max (integer compares on the bit
//     patterns), row and column exchanges by shuffles, one division per
//     elimination step; back substitution column by column;
//   - the two QR factors: lanes 0-3 build column l of Qs, lanes 4-7 column
//     l - 4 of Zs (each half from its own reflectors);
//   - the 4 x 4 products, the tests and the rotations of T's new 2x2 blocks:
//     lane l owns entries 2l, 2l + 1 (column l / 2) of each k x k result,
//     exchanged through the slot's shared-memory scratch.
// All loops have the same trip counts on the 8 lanes; shuffles and
// __syncwarp name the octet's lanes only.
// ---------------------------------------------------------------------------

// Per-slot scratch (doubles, column-major 4 x 4 each, zero / identity beyond
// k): DA DB Qs Zs WA WB NA NB.
constexpr int SC_DA = 0, SC_DB = 16, SC_Q = 32, SC_Z = 48, SC_WA = 64, SC_WB = 80, SC_NA = 96,
              SC_NB = 112;
static_assert(SC_NB + 16 <= GSLOT, "slot scratch");

__device__ __forceinline__ double pick8(const double (&v)[8], int i) {
    double r = v[0];
#pragma unroll
    for (int c = 1; c < 8; ++c) r = (i == c) ? v[c] : r;
    return r;
}

// Reflector (I - tau v v^T) on 4-vectors mapping x onto beta e_0, v[0] = 1;
// tau = 0 when x is a multiple of e_0 already.
__device__ __forceinline__ void house4(const double x[4], double v[4], double* tau) {
    const double sigma = fma(x[1], x[1], fma(x[2], x[2], x[3] * x[3]));
    v[0] = 1.0;
    v[1] = x[1];
    v[2] = x[2];
    v[3] = x[3];
    *tau = 0.0;
    if (sigma != 0.0) {
        const double nrm = sqrt(fma(x[0], x[0], sigma));
        const double beta = x[0] >= 0.0 ? -nrm : nrm;
        const double inv = 1.0 / (x[0] - beta);
        v[1] *= inv;
        v[2] *= inv;
        v[3] *= inv;
        *tau = (beta - x[0]) / beta;
    }
}

// Returns true (on all 8 lanes) if the swap of the p x p block at ja with the
// q x q block below it is accepted; sc (the slot's scratch) then holds Qs,
// Zs and the new diagonal parts NA, NB.  l: lane in the octet; ob: lane of
// the octet's lane 0 in the warp; om: the octet's lane mask.
__device__ __forceinline__ bool gen_swap_octet(int p, int q, const double* __restrict__ Sp,
                                               const double* __restrict__ Tp, int ja, bool strong,
                                               int l, int ob, unsigned om, double* __restrict__ sc) {
    const int k = p + q, pq = p * q, N = 2 * pq;
    // own entries e = 2l, 2l+1: column c0 = l / 2, rows r0, r0 + 1
    const int ec = l >> 1, er = (l & 1) * 2;
    double pa = 0.0, pb = 0.0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int r = er + t;
        const bool in = ec < k && r < k && r <= ec + 1;
        const double a = in ? Sp[gpoff(ja + ec) + ja + r] : 0.0;
        const double b = in ? Tp[gpoff(ja + ec) + ja + r] : 0.0;
        sc[SC_DA + ec * 4 + r] = a;
        sc[SC_DB + ec * 4 + r] = b;
        pa = fma(a, a, pa);
        pb = fma(b, b, pb);
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        pa += __shfl_xor_sync(om, pa, o);
        pb += __shfl_xor_sync(om, pb, o);
    }
    const double tha = fmax(20.0 * DBL_EPSILON * sqrt(pa), DBL_MIN);
    const double thb = fmax(20.0 * DBL_EPSILON * sqrt(pb), DBL_MIN);
    __syncwarp(om);
    const double* DA = sc + SC_DA;
    const double* DB = sc + SC_DB;
    if (k == 2 && DA[0] * DB[5] == DA[5] * DB[0]) {
        // equal generalized eigenvalues: in order already (identity factors)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int e = 2 * l + t;
            const double id = ((e & 3) == (e >> 2)) ? 1.0 : 0.0;
            sc[SC_Q + e] = id;
            sc[SC_Z + e] = id;
            sc[SC_NA + e] = DA[e];
            sc[SC_NB + e] = DB[e];
        }
        __syncwarp(om);
        return true;
    }

    // --- Kronecker row l: unknowns [vec R; vec L], equations [first; second]
    double K[8], b = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) K[c] = 0.0;
    if (l < N) {
        const int e = l / pq, rem = l - e * pq, i = rem % p, cc = rem / p;
        const double* D = e ? DB : DA;
        b = -D[(p + cc) * 4 + i];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            double v = 0.0;
            if (c < pq) {
                if (c / p == cc) v += D[(c % p) * 4 + i];          // X11[i][l'] R[l'][cc]
            } else if (c < N) {
                const int u = c - pq;
                if (u % p == i) v -= D[(p + cc) * 4 + p + u / p];  // -L[i][m] X22[m][cc]
            }
            K[c] = v;
        }
    }
    unsigned long long km = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) km = max(km, mag(K[c]));
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const unsigned long long v = __shfl_xor_sync(om, km, o);
        km = max(km, v);
    }
    const double smin = fmax(DBL_EPSILON * __longlong_as_double((long long)km), DBL_MIN);
    int perm = l;
    double rpiv = 1.0;
    for (int s = 0; s < N; ++s) {
        // arg-max over rows >= s, columns [s, N): (magnitude, row * 8 + col),
        // the first in row-major order on ties
        unsigned long long bm = 0;
        int bi = 64;
        if (l >= s && l < N) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const unsigned long long v = mag(K[c]);
                if (c >= s && c < N && (bi == 64 || v > bm)) { bm = v; bi = l * 8 + c; }
            }
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const unsigned long long v = __shfl_xor_sync(om, bm, o);
            const int vi = __shfl_xor_sync(om, bi, o);
            if (vi != 64 && (bi == 64 || v > bm || (v == bm && vi < bi))) { bm = v; bi = vi; }
        }
        const int pr = bi >> 3, pc = bi & 7;
        // rows s <-> pr
        const int prt = (l == s) ? pr : (l == pr ? s : l);
#pragma unroll
        for (int c = 0; c < 8; ++c) K[c] = __shfl_sync(om, K[c], ob + prt);
        b = __shfl_sync(om, b, ob + prt);
        // columns s <-> pc
        {
            const double vs = pick8(K, s), vp = pick8(K, pc);
#pragma unroll
            for (int c = 0; c < 8; ++c) K[c] = (c == s) ? vp : ((c == pc) ? vs : K[c]);
            const int pct = (l == s) ? pc : (l == pc ? s : l);
            perm = __shfl_sync(om, perm, ob + pct);
        }
        if (l == s && mag(pick8(K, s)) < mag(smin)) {
#pragma unroll
            for (int c = 0; c < 8; ++c) K[c] = (c == s) ? smin : K[c];
        }
        // eliminate below the pivot
        double prow[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) prow[c] = __shfl_sync(om, K[c], ob + s);
        const double pbv = __shfl_sync(om, b, ob + s);
        // one reciprocal per pivot, kept by the pivot's lane for the back
        // substitution (no division there)
        const double rinv = 1.0 / pick8(prow, s);
        if (l == s) rpiv = rinv;
        if (l > s && l < N) {
            const double f = pick8(K, s) * rinv;
#pragma unroll
            for (int c = 0; c < 8; ++c) K[c] = (c > s) ? fma(-f, prow[c], K[c]) : (c == s ? 0.0 : K[c]);
            b = fma(-f, pbv, b);
        }
    }
    // back substitution, column by column: acc holds row l's remaining sum
    double acc = b, y = 0.0, g = 1.0;
    const double big = DBL_MAX / 4.0;
    for (int s = N - 1; s >= 0; --s) {
        double f = 1.0;
        if (l == s) {
            const double pv = fabs(pick8(K, s));
            if (pv < 1.0 && fabs(acc) > big * pv) f = (big * pv) / fabs(acc);
        }
        f = __shfl_sync(om, f, ob + s);
        if (f != 1.0) {
            acc *= f;
            y *= f;
            g *= f;
        }
        if (l == s) y = acc * rpiv;
        const double ys = __shfl_sync(om, y, ob + s);
        if (l < s) acc = fma(-pick8(K, s), ys, acc);
    }
    // unknown perm[c] = y of lane c: gather R (lanes 0-3 need L, 4-7 need R)
    double X[4] = {0.0, 0.0, 0.0, 0.0};
    const bool zhalf = l >= 4;
    for (int c = 0; c < N; ++c) {
        const double v = __shfl_sync(om, y, ob + c);
        const int u = __shfl_sync(om, perm, ob + c);
        const int want = zhalf ? (u < pq ? u : -1) : u - pq;   // R for Zs, L for Qs
#pragma unroll
        for (int t = 0; t < 4; ++t) X[t] = (want == t) ? v : X[t];
    }
    // --- QR factor: column (l & 3) of Qs (lanes 0-3, from [L; g I]) or of
    // Zs (lanes 4-7, from [R; g I]); H1 for column 0, H2 on rows 1..3
    {
        double M0[4], M1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            M0[i] = i < p ? X[i] : (i == p ? g : 0.0);
            M1[i] = (q == 2) ? (i < p ? X[i + p] : (i == p + 1 ? g : 0.0)) : 0.0;
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
        // column c of H1 diag(1, H2): w = diag(1, H2) e_c, then H1 w
        const int c = l & 3;
        double w[4];
        w[0] = (c == 0) ? 1.0 : 0.0;
#pragma unroll
        for (int i = 1; i < 4; ++i)
            w[i] = (c == 0) ? 0.0 : (((i == c) ? 1.0 : 0.0) - t2 * v2[i - 1] * v2[c - 1]);
        double d = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) d = fma(v1[i], w[i], d);
        d *= t1;
        double* out = sc + (zhalf ? SC_Z : SC_Q) + c * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = fma(-d, v1[i], w[i]);
    }
    __syncwarp(om);
    const double* Qs = sc + SC_Q;
    const double* Zs = sc + SC_Z;
    // --- W = Qs^T D (own entries), then N = W Zs
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int r = er + t;
        double wa = 0.0, wb = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            wa = fma(Qs[r * 4 + a], DA[ec * 4 + a], wa);
            wb = fma(Qs[r * 4 + a], DB[ec * 4 + a], wb);
        }
        sc[SC_WA + ec * 4 + r] = wa;
        sc[SC_WB + ec * 4 + r] = wb;
    }
    __syncwarp(om);
    bool low = false;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int r = er + t;
        double na = 0.0, nb = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            na = fma(sc[SC_WA + a * 4 + r], Zs[ec * 4 + a], na);
            nb = fma(sc[SC_WB + a * 4 + r], Zs[ec * 4 + a], nb);
        }
        // weak test on the block that must vanish: rows [q, k) x columns [0, q)
        if (ec < q && r >= q && r < k) {
            low |= mag(na) > mag(tha) || mag(nb) > mag(thb);
            na = 0.0;
            nb = 0.0;
        }
        sc[SC_NA + ec * 4 + r] = na;
        sc[SC_NB + ec * 4 + r] = nb;
    }
    if (__any_sync(om, low)) return false;
    __syncwarp(om);
    if (strong) {
        // V = Qs N (into W), then D - V Zs^T must stay below the thresholds
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int r = er + t;
            double va = 0.0, vb = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                va = fma(Qs[a * 4 + r], sc[SC_NA + ec * 4 + a], va);
                vb = fma(Qs[a * 4 + r], sc[SC_NB + ec * 4 + a], vb);
            }
            sc[SC_WA + ec * 4 + r] = va;
            sc[SC_WB + ec * 4 + r] = vb;
        }
        __syncwarp(om);
        bool bad = false;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int r = er + t;
            double ea = 0.0, eb = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                ea = fma(sc[SC_WA + a * 4 + r], Zs[a * 4 + ec], ea);
                eb = fma(sc[SC_WB + a * 4 + r], Zs[a * 4 + ec], eb);
            }
            bad |= mag(ea - DA[ec * 4 + r]) > mag(tha) || mag(eb - DB[ec * 4 + r]) > mag(thb);
        }
        if (__any_sync(om, bad)) return false;
    }
    // --- T stays upper triangular: rotate the two columns of each new 2x2
    // block (lanes 0-3: rows of NA, lanes 4-7: rows of NB, then all of Zs).
    // The two blocks own disjoint columns, so both rotations are computed
    // first (independent chains) and applied one after the other.
    double rc[2], rs[2];
    bool act[2];
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        const int sz = blk ? p : q, c0 = blk ? q : 0;
        act[blk] = false;
        rc[blk] = 1.0;
        rs[blk] = 0.0;
        if (sz == 2) {
            const double b10 = sc[SC_NB + c0 * 4 + c0 + 1], b11 = sc[SC_NB + (c0 + 1) * 4 + c0 + 1];
            if (b10 != 0.0) {
                const double rh = 1.0 / hypot(b10, b11);
                act[blk] = true;
                rc[blk] = b11 * rh;
                rs[blk] = -b10 * rh;
            }
        }
    }
    __syncwarp(om);
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        if (!act[blk]) continue;
        const int c0 = blk ? q : 0;
        const double cs = rc[blk], sn = rs[blk];
        {
            double* M = sc + (zhalf ? SC_NB : SC_NA);
            const int r = l & 3;
            const double x = M[c0 * 4 + r], yv = M[(c0 + 1) * 4 + r];
            M[c0 * 4 + r] = fma(cs, x, sn * yv);
            M[(c0 + 1) * 4 + r] = fma(cs, yv, -sn * x);
        }
        if (l < 4) {
            double* M = sc + SC_Z;
            const double x = M[c0 * 4 + l], yv = M[(c0 + 1) * 4 + l];
            M[c0 * 4 + l] = fma(cs, x, sn * yv);
            M[(c0 + 1) * 4 + l] = fma(cs, yv, -sn * x);
        }
        __syncwarp(om);
        if (l == 0) sc[SC_NB + c0 * 4 + c0 + 1] = 0.0;
        __syncwarp(om);
    }
    return true;
}

// Warps [base[g], base[g+1]) serve group g (k = g + 2): counts in proportion
// to tot[g] k^2, at least one warp for a group with items, nwarps in all.
// Every thread computes the same split.
__device__ __forceinline__ void split_warps(const int tot[3], int nwarps, int base[4]) {
    int wt[3], c[3], sum = 0;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        wt[g] = tot[g] * (g + 2) * (g + 2);
        sum += wt[g];
    }
    int used = 0;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        c[g] = tot[g] == 0 ? 0 : max(1, (int)((long long)wt[g] * nwarps / (sum > 0 ? sum : 1)));
        used += c[g];
    }
    // fix the total: take from the group with the most warps, give to the
    // group with the most work per warp
    while (used > nwarps) {
        int gi = 0;
        for (int g = 1; g < 3; ++g) if (c[g] > c[gi]) gi = g;
        --c[gi];
        --used;
    }
    while (used < nwarps && sum > 0) {
        int gi = -1;
        for (int g = 0; g < 3; ++g)
            if (c[g] > 0 && (gi < 0 || (long long)wt[g] * c[gi] > (long long)wt[gi] * c[g])) gi = g;
        if (gi < 0) break;
        ++c[gi];
        ++used;
    }
    base[0] = 0;
    base[1] = c[0];
    base[2] = c[0] + c[1];
    base[3] = c[0] + c[1] + c[2];
}

// Left items of group k: item it of the group's flat list (prefix sums pre
// over its cnt slots) is column j + k + (it - pre[i]) of swap list[i].
template <int K>
__device__ __forceinline__ void apply_left(int first, int stride, int total, int cnt, const int* pre,
                                           const int* list, const int* swj, const double* SCR,
                                           double* Sp, double* Tp) {
    for (int it = first; it < total; it += stride) {
        int lo = 0, hi = cnt - 1;   // last i with pre[i] <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const int slot = list[lo], j = swj[slot];
        const int c = j + K + (it - pre[lo]);
        const double* Qs = SCR + slot * GSLOT + SC_Q;
        double xs[K], xt[K];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            xs[r] = Sp[gpoff(c) + j + r];
            xt[r] = Tp[gpoff(c) + j + r];
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            double as = 0.0, at = 0.0;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                as = fma(Qs[r * 4 + i], xs[i], as);
                at = fma(Qs[r * 4 + i], xt[i], at);
            }
            Sp[gpoff(c) + j + r] = as;
            Tp[gpoff(c) + j + r] = at;
        }
    }
}

// Right items of group k: rows [0, j) of S and T for the columns [j, j+k)
// of swap list[i].
template <int K>
__device__ __forceinline__ void apply_right(int first, int stride, int total, int cnt, const int* pre,
                                            const int* list, const int* swj, const double* SCR,
                                            double* Sp, double* Tp) {
    for (int it = first; it < total; it += stride) {
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= it) lo = mid; else hi = mid - 1;
        }
        const int slot = list[lo], j = swj[slot];
        const int rr = it - pre[lo];
        const double* Zs = SCR + slot * GSLOT + SC_Z;
        double x1[K], x2[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            x1[i] = Sp[gpoff(j + i) + rr];
            x2[i] = Tp[gpoff(j + i) + rr];
        }
#pragma unroll
        for (int c = 0; c < K; ++c) {
            double a1 = 0.0, a2 = 0.0;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                a1 = fma(x1[i], Zs[c * 4 + i], a1);
                a2 = fma(x2[i], Zs[c * 4 + i], a2);
            }
            Sp[gpoff(j + c) + rr] = a1;
            Tp[gpoff(j + c) + rr] = a2;
        }
    }
}

// Row r of UQ and UZ, columns [j, j + K) <- (those columns) Qs and Zs (the
// right transformations of one swap, applied to the accumulators).
template <int K>
__device__ __forceinline__ void right_uqz_row(double* __restrict__ UQ, double* __restrict__ UZ,
                                              int w, int j, int r, const double* __restrict__ Qs,
                                              const double* __restrict__ Zs) {
    double x1[K], x2[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        x1[i] = UQ[(j + i) * w + r];
        x2[i] = UZ[(j + i) * w + r];
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
        double a1 = 0.0, a2 = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            a1 = fma(x1[i], Qs[c * 4 + i], a1);
            a2 = fma(x2[i], Zs[c * 4 + i], a2);
        }
        UQ[(j + c) * w + r] = a1;
        UZ[(j + c) * w + r] = a2;
    }
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
    // The state of a step (swaps, their scratch with Qs and Zs, item prefix
    // sums) is kept for two steps, by the step's parity: the rows of UQ and
    // UZ of a step's right transformations (read by no later swap) are
    // applied during the next step's swap transforms, by warps whose
    // sub-partition carries no k = 3 or 4 pair swap.
    double* SCRbuf = Tp + gpoff(GW);                      // [2][GMAXSW * GSLOT]
    int* swbuf = reinterpret_cast<int*>(SCRbuf + 2 * GMAXSW * GSLOT);  // [2][3][GMAXSW]
    uint8_t* bst = reinterpret_cast<uint8_t*>(swbuf + 2 * 3 * GMAXSW);
    uint8_t* sel = bst + GW;
    __shared__ int nsw, nrej, nacc;
    __shared__ int wall_top, wall_bot;
    __shared__ int gcnt2[2][3], glist2[2][3][GMAXSW];   // slots per block-size sum k = 2, 3, 4
    __shared__ int gpl[3][GMAXSW + 1], gps[3][GMAXSW + 1];  // left / right S, T item prefix sums
    __shared__ int gpu2[2][3][GMAXSW + 1];      // right UQ, UZ item prefix sums
    __shared__ short urlo[GW], urhi[GW];        // nonzero rows of each column of UQ, UZ
    __shared__ short slo2[2][GMAXSW], shi2[2][GMAXSW];  // per slot: rows of UQ, UZ it updates
    __shared__ int pu_par, pu_next;             // step whose UQ, UZ rows are pending (-1: none)
    unsigned long long wflops = 0;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane_ = tid & 31;
    // the UQ, UZ rows of the step of parity pp, claimed by whole warps in
    // chunks of 32 (pu_next)
    auto pending_uqz = [&](int pp) {
        const int* pj = swbuf + pp * 3 * GMAXSW;
        const int* pk = pj + GMAXSW;
        const int T0 = gpu2[pp][0][gcnt2[pp][0]], T1 = gpu2[pp][1][gcnt2[pp][1]];
        const int total = T0 + T1 + gpu2[pp][2][gcnt2[pp][2]];
        for (;;) {
            int base = 0;
            if (lane_ == 0) base = atomicAdd(&pu_next, 32);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= total) break;
            const int it = base + lane_;
            if (it >= total) continue;
            const int g = it < T0 ? 0 : (it < T0 + T1 ? 1 : 2);
            const int itg = it - (g == 0 ? 0 : (g == 1 ? T0 : T0 + T1));
            const int* pre = gpu2[pp][g];
            int lo = 0, hi = gcnt2[pp][g] - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= itg) lo = mid; else hi = mid - 1;
            }
            const int slot = glist2[pp][g][lo];
            if (pk[slot] == 0) continue;  // rejected
            const int j = pj[slot];
            const int r = slo2[pp][slot] + (itg - pre[lo]);
            const double* sc = SCRbuf + (size_t)pp * GMAXSW * GSLOT + slot * GSLOT;
            if (g == 0) right_uqz_row<2>(UQ, UZ, w, j, r, sc + SC_Q, sc + SC_Z);
            else if (g == 1) right_uqz_row<3>(UQ, UZ, w, j, r, sc + SC_Q, sc + SC_Z);
            else right_uqz_row<4>(UQ, UZ, w, j, r, sc + SC_Q, sc + SC_Z);
        }
    };

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
    for (int i = tid; i < w; i += nth) {
        sel[i] = __ldcg(&gsel[s0 + i]);
        urlo[i] = (short)i;
        urhi[i] = (short)i;
    }
    if (tid == 0) {
        nrej = 0;
        nacc = 0;
        pu_par = -1;
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
        const int par = iter & 1;
        double* SCR = SCRbuf + (size_t)par * GMAXSW * GSLOT;
        int* swj = swbuf + par * 3 * GMAXSW;
        int* swk = swj + GMAXSW;
        int* swp = swk + GMAXSW;
        int* gcnt = gcnt2[par];
        int (*glist)[GMAXSW] = glist2[par];
        int (*gpu)[GMAXSW + 1] = gpu2[par];
        short* slo = slo2[par];
        short* shi = shi2[par];
        __syncthreads();
        if (iter > 4 * GW * GW) {
            if (tid == 0) atomicAdd(&ctr->step_overflow, 1);
            break;
        }
        for (int i = tid; i < w; i += nth) bst[i] = (i == 0) || (Sp[gpoff(i - 1) + i] == 0.0);
        if (tid == 0) nsw = 0;
        if (tid < 3) gcnt[tid] = 0;
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
            glist[p + q - 2][atomicAdd(&gcnt[p + q - 2], 1)] = slot;
        }
        __syncthreads();
        const int ns = nsw;
        if (ns == 0) break;  // the pending rows are applied after the loop
        // One octet (8 lanes) per swap, the four octets of a warp on swaps of
        // the same sizes (k = 4 first, then 3, then 2), so that they follow
        // one instruction stream with the same trip counts.  At most 32
        // swaps need at most 11 of the 16 warps.
        {
            const int lane = tid & 31, warp = tid >> 5;
            const int nw4 = (gcnt[2] + 3) >> 2, nw3 = (gcnt[1] + 3) >> 2;
            const int g = warp < nw4 ? 2 : (warp < nw4 + nw3 ? 1 : 0);
            const int wbase = g == 2 ? 0 : (g == 1 ? nw4 : nw4 + nw3);
            const int idx = (warp - wbase) * 4 + (lane >> 3);
            const int l = lane & 7, ob = lane & ~7;
            const unsigned om = 0xffu << ob;
            if (idx < gcnt[g]) {
                const int slot = glist[g][idx], ja = swj[slot], k = swk[slot], p = swp[slot],
                          q = k - p;
                double* sc = SCR + slot * GSLOT;
                if (gen_swap_octet(p, q, Sp, Tp, ja, strong != 0, l, ob, om, sc)) {
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int e = 2 * l + t, r = e & 3, c = e >> 2;
                        if (c < k && r < k && r <= c + 1) {
                            Sp[gpoff(ja + c) + ja + r] = sc[SC_NA + e];
                            Tp[gpoff(ja + c) + ja + r] = sc[SC_NB + e];
                        }
                    }
                    if (l == 0) atomicAdd(&nacc, 1);
                } else if (l == 0) {
                    swk[slot] = 0;
                    swp[slot] = ja + p;   // the stuck (selected) block
                    atomicAdd(&nrej, 1);
                }
            }
            // the previous step's UQ, UZ rows, by the warps of the
            // sub-partitions that carry no k = 3 or 4 swap chain
            if (pu_par >= 0 && (warp & 3) >= min(nw4 + nw3, 4)) pending_uqz(pu_par);
        }
        __syncthreads();
        // what is left of them (UQ, UZ only: no conflict with the steps below)
        if (pu_par >= 0) pending_uqz(pu_par);
        // Work lists of the updates, per block-size sum k (so that a warp
        // applies one k): prefix sums of the left items (columns [j+k, w) of
        // rows [j, j+k) of S and T) and of the right items (rows [0, j) of
        // columns [j, j+k) of S and T, then the rows [lo, hi] of UQ and UZ
        // holding the nonzeros of those columns: UQ and UZ start as I and a
        // swap mixes only its own columns, the same ones in both).  Warp g
        // scans group g; rejected swaps have no items.
        {
            const int lane = tid & 31, warp = tid >> 5;
            if (warp < 3) {
                const int g = warp, k = g + 2, cnt = gcnt[g];
                int il = 0, ir = 0, iu = 0;
                if (lane < cnt) {
                    const int slot = glist[g][lane], j = swj[slot];
                    if (swk[slot] != 0) {
                        int lo = urlo[j], hi = urhi[j];
                        for (int c = 1; c < k; ++c) {
                            lo = min(lo, (int)urlo[j + c]);
                            hi = max(hi, (int)urhi[j + c]);
                        }
                        slo[slot] = (short)lo;
                        shi[slot] = (short)hi;
                        il = w - j - k;
                        ir = j;
                        iu = hi - lo + 1;
                    }
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int a2 = __shfl_up_sync(0xffffffffu, il, o);
                    const int b2 = __shfl_up_sync(0xffffffffu, ir, o);
                    const int c2 = __shfl_up_sync(0xffffffffu, iu, o);
                    if (lane >= o) { il += a2; ir += b2; iu += c2; }
                }
                if (lane < cnt) { gpl[g][lane + 1] = il; gps[g][lane + 1] = ir; gpu[g][lane + 1] = iu; }
                if (lane == 0) { gpl[g][0] = 0; gps[g][0] = 0; gpu[g][0] = 0; }
            }
        }
        __syncthreads();
        // The warps are split among the three k groups in proportion to
        // their FP64 work (items x k^2), so that every warp applies one k
        // and the sub-partitions carry equal shares; then the left products
        // (rows [j, j+k) of S and T, columns [j+k, w), by Qs^T) and, after a
        // barrier, the right ones (columns [j, j+k) of S and T for rows
        // [0, j) by Zs, of UQ by Qs and UZ by Zs for rows [lo, hi]).
        {
            const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
            int tl[3], tr[3], bl[4], br[4];
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                tl[g] = gcnt[g] ? gpl[g][gcnt[g]] : 0;
                tr[g] = gcnt[g] ? gps[g][gcnt[g]] : 0;
            }
            split_warps(tl, nwarps, bl);
            split_warps(tr, nwarps, br);
            const int gL = warp < bl[1] ? 0 : (warp < bl[2] ? 1 : 2);
            if (warp < bl[3]) {
                const int first = (warp - bl[gL]) * 32 + lane, stride = (bl[gL + 1] - bl[gL]) * 32;
                if (gL == 0) apply_left<2>(first, stride, tl[0], gcnt[0], gpl[0], glist[0], swj, SCR, Sp, Tp);
                else if (gL == 1) apply_left<3>(first, stride, tl[1], gcnt[1], gpl[1], glist[1], swj, SCR, Sp, Tp);
                else apply_left<4>(first, stride, tl[2], gcnt[2], gpl[2], glist[2], swj, SCR, Sp, Tp);
            }
            __syncthreads();
            const int gR = warp < br[1] ? 0 : (warp < br[2] ? 1 : 2);
            if (warp < br[3]) {
                const int first = (warp - br[gR]) * 32 + lane, stride = (br[gR + 1] - br[gR]) * 32;
                if (gR == 0)
                    apply_right<2>(first, stride, tr[0], gcnt[0], gps[0], glist[0], swj, SCR, Sp, Tp);
                else if (gR == 1)
                    apply_right<3>(first, stride, tr[1], gcnt[1], gps[1], glist[1], swj, SCR, Sp, Tp);
                else
                    apply_right<4>(first, stride, tr[2], gcnt[2], gps[2], glist[2], swj, SCR, Sp, Tp);
            }
        }
        __syncthreads();
        // this step's UQ, UZ rows are pending now
        if (tid == 0) {
            pu_par = par;
            pu_next = 0;
        }
        // move the selection flags with the blocks
        for (int sw = tid; sw < ns; sw += nth) {
            const int j = swj[sw], k = swk[sw];
            if (k == 0) {
                sel[swp[sw]] = SEL_STUCK;
                continue;
            }
            // left (S, T) + right (S, T) + UQ, UZ rows [lo, hi]: k x k
            // applied to 2 (w - j - k) + 2 j + 2 (hi - lo + 1) vectors
            wflops += 2ull * k * k *
                      (unsigned long long)(2 * (w - j - k) + 2 * j + 2 * (shi[sw] - slo[sw] + 1));
            for (int c = 0; c < k; ++c) {
                urlo[j + c] = slo[sw];
                urhi[j + c] = shi[sw];
            }
            const int p = swp[sw], q = k - p;
            for (int i = 0; i < q; ++i) sel[j + i] = SEL_YES;
            for (int i = q; i < k; ++i) sel[j + i] = SEL_NO;
        }
        __syncthreads();
        for (int t = tid; t + 1 < w; t += nth)
            if (sel[t] == SEL_STUCK && Sp[gpoff(t) + t + 1] != 0.0) sel[t + 1] = SEL_STUCK;
    }
    // the last step's UQ, UZ rows
    __syncthreads();
    if (pu_par >= 0) pending_uqz(pu_par);
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
