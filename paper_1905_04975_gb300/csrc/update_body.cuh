// Off-diagonal updates of one window (Section 3.2: the accumulated
// transformation U applied to "the relevant sections of the matrix" as
// level-3 operations -- the left and right update tasks):
//
//   left   S[s:e, e:n] <- U^T S[s:e, e:n]
//   right  S[0:s, s:e] <- S[0:s, s:e] U
//   Q      Q[:,  s:e]  <- Q[:,  s:e]  U
//
// All three are the same product Y <- Y U on a tall panel Y (R x w): for the
// right and Q updates Y is the column-major panel itself; for the left update
// Y is its transpose, i.e. the panel read row-major (row c of Y = column c of
// S[s:e, e:n], contiguous in memory).  A tile is BM whole rows of Y, so the
// product is done in place.  The contraction runs on the FP64 tensor path
// (DMMA, mma.sync m8n8k4 f64).
//
// Included by the per-window launch (update.cu) and by the persistent
// scheduler (sched.cu); global loads go through L2 (ld.global.cg).
#pragma once

#include "common.cuh"
#include "window_body.cuh"

#include <cuda_bf16.h>

namespace gbr {
namespace upd {

constexpr int BM = UPD_BM;        // panel rows per tile
constexpr int UPD_THREADS = 256;  // 8 warps, each owning 16 output columns
constexpr int LDY = WMAX + 4;     // padded row pitch of the Y tile in shared memory
constexpr int LDU = WMAX + 8;     // padded row pitch of U (row k holds U[k, :])
constexpr size_t kUpdateSmem = sizeof(double) * ((size_t)WMAX * LDU +
                                                  (size_t)(BM * LDY > WMAX * (BM + 2)
                                                               ? BM * LDY
                                                               : WMAX * (BM + 2)));
// Wide windows (WMAX < w <= WMAX_WIDE): U stays in global memory (read via
// L2; the FP64 work per U element read hides its latency) and only the Y
// tile is staged.
constexpr int LDY_WIDE = WMAX_WIDE + 4;
constexpr size_t kUpdateSmemWide = sizeof(double) * (size_t)(BM * LDY_WIDE > WMAX_WIDE * (BM + 2)
                                                                 ? BM * LDY_WIDE
                                                                 : WMAX_WIDE * (BM + 2));

enum Panel { PANEL_L = 0, PANEL_R = 1, PANEL_Q = 2 };

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// Panel geometry: element (r, k) of Y at base + r*rs + k*ks, R rows.
__device__ __forceinline__ void panel_geom(int panel, int n, int s, int e, double* S, int ldS,
                                           double* Q, int ldQ, double** base, long long* rs,
                                           long long* ks, int* R) {
    if (panel == PANEL_L) {
        *base = S + cm(s, e, ldS);  // Y(r, k) = S[s + k, e + r]
        *rs = ldS; *ks = 1; *R = n - e;
    } else if (panel == PANEL_R) {
        *base = S + cm(0, s, ldS);  // Y(r, k) = S[r, s + k]
        *rs = 1; *ks = ldS; *R = s;
    } else {
        *base = Q + cm(0, s, ldQ);  // Y(r, k) = Q[r, s + k]
        *rs = 1; *ks = ldQ; *R = n;
    }
}

// Y rows [r0, r0 + rows) <- (Y U) rows, rows <= BM; nthreads >= UPD_THREADS
// (warps beyond the first 8 only help loading).  If load_u is false, Us
// already holds U (a previous tile of the same window in this CTA).
//
// U is a product of adjacent-block swaps, so the nonzeros of each of its
// columns form one contiguous run of rows (a staircase: about a quarter of
// U is zero for a window whose chain enters at the bottom, more for a
// chain's first window).  When U is loaded, each warp finds, for each of its
// two groups of 8 output columns, the rows [klo, khi) where they have
// nonzeros, and the products of a group run over those rows only.  If
// issued is not null, the flops issued by the tile are added to it.
//
// WIDE (w up to WMAX_WIDE, 16 column warps: nthreads >= 512): U is read from
// global memory where the window task formed it, instead of a shared copy.
template <bool WIDE = false>
__device__ __forceinline__ void update_tile(double* base, long long rs, long long ks, int r0,
                                            int rows, int w, const double* __restrict__ Ug,
                                            bool load_u, unsigned char* smem_raw,
                                            unsigned long long* issued = nullptr) {
    constexpr int LY = WIDE ? LDY_WIDE : LDY;
    constexpr int NWC = WIDE ? WMAX_WIDE / 16 : UPD_THREADS / 32;  // warps of 16 output columns
    double* Us = reinterpret_cast<double*>(smem_raw);  // WMAX x LDU (not with WIDE)
    double* Ys = WIDE ? Us : Us + WMAX * LDU;          // BM x LY
    __shared__ int k_lo[NWC][2], k_hi[NWC][2];
    const int wp = (w + 15) & ~15;  // padded to the warp column width
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    // U(k, c), zero outside w x w
    auto uat = [&](int k, int c) -> double {
        if constexpr (WIDE)
            return (k < w && c < w) ? __ldcg(&Ug[(size_t)c * w + k]) : 0.0;
        else
            return Us[k * LDU + c];
    };
    if (load_u) {
        if constexpr (!WIDE) {
            for (int i = tid; i < wp * wp; i += nth) {
                int k = i / wp, c = i % wp;
                Us[k * LDU + c] = (k < w && c < w) ? __ldcg(&Ug[(size_t)c * w + k]) : 0.0;
            }
            __syncthreads();
        }
        if (warp < NWC) {
            const int c0 = warp * 16;
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) {
                int lo = wp, hi = 0;
                if (c0 < wp)
                    for (int k = lane; k < wp; k += 32) {
                        bool nz = false;
#pragma unroll
                        for (int c = 0; c < 8; ++c) nz |= uat(k, c0 + 8 * ct + c) != 0.0;
                        if (nz) {
                            lo = min(lo, k);
                            hi = max(hi, k + 1);
                        }
                    }
                for (int o = 16; o; o >>= 1) {
                    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                }
                if (lane == 0) {
                    k_lo[warp][ct] = lo < hi ? (lo & ~3) : 0;
                    k_hi[warp][ct] = lo < hi ? min(wp, (hi + 3) & ~3) : 0;
                }
            }
        }
    }
    if (rs == 1) {
        for (int i = tid; i < BM * wp; i += nth) {
            int r = i % BM, k = i / BM;
            Ys[r * LY + k] = (r < rows && k < w) ? __ldcg(&base[(r0 + r) + (long long)k * ks]) : 0.0;
        }
    } else {
        for (int i = tid; i < BM * wp; i += nth) {
            int k = i % wp, r = i / wp;
            Ys[r * LY + k] = (r < rows && k < w) ? __ldcg(&base[(long long)(r0 + r) * rs + k]) : 0.0;
        }
    }
    __syncthreads();
    const int gid = lane >> 2, tig = lane & 3;
    const int c0 = warp * 16;
    if (issued && tid == 0) {
        unsigned long long f = 0;
        for (int v = 0; v < NWC && v * 16 < w; ++v)
            for (int ct = 0; ct < 2 && v * 16 + 8 * ct < w; ++ct)
                f += 2ull * rows * (unsigned long long)min(8, w - v * 16 - 8 * ct) *
                     (k_hi[v][ct] - k_lo[v][ct]);
        atomicAdd(issued, f);
    }
    if (warp < NWC && c0 < wp) {
        const int lo0 = k_lo[warp][0], hi0 = k_hi[warp][0];
        const int lo1 = k_lo[warp][1], hi1 = k_hi[warp][1];
        double acc[8][2][2];
#pragma unroll
        for (int rt = 0; rt < 8; ++rt)
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) acc[rt][ct][0] = acc[rt][ct][1] = 0.0;
        // rows where both groups have nonzeros, then the rows of one group
        // only (the ranges are contiguous, so at most one such run per side)
        const int blo = max(lo0, lo1), bhi = min(hi0, hi1);
        for (int kk = blo; kk < bhi; kk += 4) {
            double a[8], bb[2];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt) a[rt] = Ys[(rt * 8 + gid) * LY + kk + tig];
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) bb[ct] = uat(kk + tig, c0 + ct * 8 + gid);
#pragma unroll
            for (int rt = 0; rt < 8; ++rt)
#pragma unroll
                for (int ct = 0; ct < 2; ++ct) dmma(acc[rt][ct][0], acc[rt][ct][1], a[rt], bb[ct]);
        }
#pragma unroll
        for (int ct = 0; ct < 2; ++ct) {
            const int lo = ct ? lo1 : lo0, hi = ct ? hi1 : hi0;
            // rows of group ct outside [blo, bhi): below and above the common run
            for (int side = 0; side < 2; ++side) {
                const int a0 = side ? max(lo, max(bhi, blo)) : lo;
                const int a1 = side ? hi : min(hi, blo);
                for (int kk = a0; kk < a1; kk += 4) {
                    double a[8];
#pragma unroll
                    for (int rt = 0; rt < 8; ++rt) a[rt] = Ys[(rt * 8 + gid) * LY + kk + tig];
                    const double bv = uat(kk + tig, c0 + ct * 8 + gid);
#pragma unroll
                    for (int rt = 0; rt < 8; ++rt) dmma(acc[rt][ct][0], acc[rt][ct][1], a[rt], bv);
                }
            }
        }
        // write back (in place: this CTA read all of its rows before any write)
#pragma unroll
        for (int rt = 0; rt < 8; ++rt) {
            int r = rt * 8 + gid;
            if (r >= rows) continue;
#pragma unroll
            for (int ct = 0; ct < 2; ++ct)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    int k = c0 + ct * 8 + tig * 2 + v;
                    if (k < w) __stcg(&base[(long long)(r0 + r) * rs + (long long)k * ks], acc[rt][ct][v]);
                }
        }
    }
    __syncthreads();
}

// The same product Y <- Y U on the FP64 FMA pipe (DFMA) instead of the FP64
// tensor path.  On this GPU both share one FP64 pipe, and plain FMAs reach
// a higher rate than m8n8k4 DMMA (measured: 1.195 against 1.047 TFLOP/s for
// the whole GPU), so this tile trades the MMA fragments for a register tile.
//
// Shared memory: U as in update_tile (row k holds U[k, :]), the Y tile
// k-major (Yk[k * LDK + r]), so that a lane reads its two rows as one
// 16-byte load and its eight columns of U as four broadcast 16-byte loads.
// The output columns are cut into groups of 8; warp v computes groups v,
// v + nwarps, ...: lane l owns rows 2l, 2l + 1 of the 64-row tile and the 8
// columns of the group (16 FP64 accumulators).  Each group runs over the
// rows [klo, khi) of U where its 8 columns have nonzeros (the staircase of
// a product of adjacent swaps).  Every output is one FMA chain over k in
// increasing order, starting from 0.
constexpr int LDK = BM + 2;   // padded pitch of the k-major Y tile (16-byte rows)

// WIDE: w up to WMAX_WIDE, U read from global memory (see update_tile).
template <bool WIDE = false>
__device__ __forceinline__ void update_tile_fma(double* base, long long rs, long long ks, int r0,
                                                int rows, int w, const double* __restrict__ Ug,
                                                bool load_u, unsigned char* smem_raw,
                                                unsigned long long* issued = nullptr) {
    static_assert(BM == 64, "one lane owns two rows of the 64-row tile");
    constexpr int NG = (WIDE ? WMAX_WIDE : WMAX) / 8;  // groups of 8 output columns
    double* Us = reinterpret_cast<double*>(smem_raw);  // WMAX x LDU (not with WIDE)
    double* Yk = WIDE ? Us : Us + WMAX * LDU;          // wp x LDK (k-major)
    __shared__ int g_lo[NG], g_hi[NG];
    const int wp = (w + 7) & ~7;  // padded to the group width
    const int ng = wp >> 3;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
    if (load_u) {
        if constexpr (!WIDE) {
            for (int i = tid; i < wp * wp; i += nth) {
                int k = i / wp, c = i % wp;
                Us[k * LDU + c] = (k < w && c < w) ? __ldcg(&Ug[(size_t)c * w + k]) : 0.0;
            }
            __syncthreads();
        }
        // rows of U where each group of 8 columns has nonzeros
        for (int g = warp; g < ng; g += nw) {
            int lo = wp, hi = 0;
            for (int k = lane; k < wp; k += 32) {
                bool nz = false;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if constexpr (WIDE)
                        nz |= (k < w && 8 * g + c < w) &&
                              __ldcg(&Ug[(size_t)(8 * g + c) * w + k]) != 0.0;
                    else
                        nz |= Us[k * LDU + 8 * g + c] != 0.0;
                }
                if (nz) {
                    lo = min(lo, k);
                    hi = max(hi, k + 1);
                }
            }
            for (int o = 16; o; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0) {
                g_lo[g] = lo < hi ? lo : 0;
                g_hi[g] = lo < hi ? hi : 0;
            }
        }
    }
    if (rs == 1) {
        for (int i = tid; i < BM * wp; i += nth) {
            int r = i % BM, k = i / BM;
            Yk[k * LDK + r] = (r < rows && k < w) ? __ldcg(&base[(r0 + r) + (long long)k * ks]) : 0.0;
        }
    } else {
        for (int i = tid; i < BM * wp; i += nth) {
            int k = i % wp, r = i / wp;
            Yk[k * LDK + r] = (r < rows && k < w) ? __ldcg(&base[(long long)(r0 + r) * rs + k]) : 0.0;
        }
    }
    __syncthreads();
    // A short tile (the last rows of a task) packs q column groups into a
    // warp, 32 / q lanes each, so that its FMA instructions carry as many
    // active lanes as a full tile's.  The q groups of a warp run over the
    // union of their row ranges; outside its own range a group's entries of
    // U are zero, and adding their products (+-0) leaves each sum unchanged.
    const int q = rows > 32 ? 1 : (rows > 16 ? 2 : 4);
    const int lpg = 32 / q, sub = lane / lpg;
    const int nunits = (ng + q - 1) / q;
    auto unit_range = [&](int gu, int* lo, int* hi) {
        int a = wp, b = 0;
        for (int t = 0; t < q; ++t) {
            const int gg = gu * q + t;
            if (gg < ng && g_lo[gg] < g_hi[gg]) {
                a = min(a, g_lo[gg]);
                b = max(b, g_hi[gg]);
            }
        }
        *lo = a < b ? a : 0;
        *hi = a < b ? b : 0;
    };
    if (issued && tid == 0) {
        unsigned long long f = 0;
        for (int gu = 0; gu < nunits; ++gu) {
            int lo, hi;
            unit_range(gu, &lo, &hi);
            for (int t = 0; t < q; ++t) {
                const int gg = gu * q + t;
                if (gg < ng) f += 2ull * rows * (unsigned long long)min(8, w - 8 * gg) * (hi - lo);
            }
        }
        atomicAdd(issued, f);
    }
    const int ra = 2 * (lane % lpg);
    for (int gu = warp; gu < nunits; gu += nw) {
        int lo, hi;
        unit_range(gu, &lo, &hi);
        const int g = gu * q + sub;
        const bool gv = g < ng;
        const int gl = gv ? g : 0;  // lanes past the last group read a valid one
        double acc[2][8];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
#pragma unroll 2
        for (int k = lo; k < hi; ++k) {
            const double2 y = *reinterpret_cast<const double2*>(&Yk[k * LDK + ra]);
            double u[8];
            if constexpr (WIDE) {
                // k < hi <= w: the rows beyond w of U are zero, never in [lo, hi)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    u[j] = (8 * gl + j < w) ? __ldcg(&Ug[(size_t)(8 * gl + j) * w + k]) : 0.0;
            } else {
                const double2* u2 = reinterpret_cast<const double2*>(Us + 8 * gl + k * LDU);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double2 t = u2[j];
                    u[2 * j] = t.x;
                    u[2 * j + 1] = t.y;
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                acc[0][j] = fma(y.x, u[j], acc[0][j]);
                acc[1][j] = fma(y.y, u[j], acc[1][j]);
            }
        }
        // write back (in place: the tile's rows were all read before)
        if (gv) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = ra + i;
                if (r >= rows) continue;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = 8 * g + j;
                    if (k < w) __stcg(&base[(long long)(r0 + r) * rs + (long long)k * ks], acc[i][j]);
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace upd
}  // namespace gbr
