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
constexpr size_t kUpdateSmem = sizeof(double) * ((size_t)WMAX * LDU + (size_t)BM * LDY);

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
// chain's first window).  When U is loaded, each warp finds the rows
// [klo, khi) where its 16 output columns have nonzeros and the products run
// over those rows only.  If issued is not null, the flops issued by the
// tile are added to it.
__device__ __forceinline__ void update_tile(double* base, long long rs, long long ks, int r0,
                                            int rows, int w, const double* __restrict__ Ug,
                                            bool load_u, unsigned char* smem_raw,
                                            unsigned long long* issued = nullptr) {
    double* Us = reinterpret_cast<double*>(smem_raw);  // WMAX x LDU
    double* Ys = Us + WMAX * LDU;                        // BM x LDY
    __shared__ int k_lo[UPD_THREADS / 32], k_hi[UPD_THREADS / 32];
    const int wp = (w + 15) & ~15;  // padded to the warp column width
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (load_u) {
        for (int i = tid; i < wp * wp; i += nth) {
            int k = i / wp, c = i % wp;
            Us[k * LDU + c] = (k < w && c < w) ? __ldcg(&Ug[(size_t)c * w + k]) : 0.0;
        }
        __syncthreads();
        if (warp < UPD_THREADS / 32) {
            const int c0 = warp * 16;
            int lo = wp, hi = 0;
            if (c0 < wp)
                for (int k = lane; k < wp; k += 32) {
                    bool nz = false;
#pragma unroll
                    for (int c = 0; c < 16; ++c) nz |= Us[k * LDU + c0 + c] != 0.0;
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
                k_lo[warp] = lo < hi ? (lo & ~3) : 0;
                k_hi[warp] = lo < hi ? min(wp, (hi + 3) & ~3) : 0;
            }
        }
    }
    if (rs == 1) {
        for (int i = tid; i < BM * wp; i += nth) {
            int r = i % BM, k = i / BM;
            Ys[r * LDY + k] = (r < rows && k < w) ? __ldcg(&base[(r0 + r) + (long long)k * ks]) : 0.0;
        }
    } else {
        for (int i = tid; i < BM * wp; i += nth) {
            int k = i % wp, r = i / wp;
            Ys[r * LDY + k] = (r < rows && k < w) ? __ldcg(&base[(long long)(r0 + r) * rs + k]) : 0.0;
        }
    }
    __syncthreads();
    const int gid = lane >> 2, tig = lane & 3;
    const int c0 = warp * 16;
    if (issued && tid == 0) {
        unsigned long long f = 0;
        for (int v = 0; v < UPD_THREADS / 32 && v * 16 < w; ++v)
            f += 2ull * rows * (unsigned long long)min(16, w - v * 16) * (k_hi[v] - k_lo[v]);
        atomicAdd(issued, f);
    }
    if (warp < UPD_THREADS / 32 && c0 < wp) {
        const int klo = k_lo[warp], khi = k_hi[warp];
        double acc[8][2][2];
#pragma unroll
        for (int rt = 0; rt < 8; ++rt)
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) acc[rt][ct][0] = acc[rt][ct][1] = 0.0;
        for (int kk = klo; kk < khi; kk += 4) {
            double a[8], bb[2];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt) a[rt] = Ys[(rt * 8 + gid) * LDY + kk + tig];
#pragma unroll
            for (int ct = 0; ct < 2; ++ct) bb[ct] = Us[(kk + tig) * LDU + c0 + ct * 8 + gid];
#pragma unroll
            for (int rt = 0; rt < 8; ++rt)
#pragma unroll
                for (int ct = 0; ct < 2; ++ct) dmma(acc[rt][ct][0], acc[rt][ct][1], a[rt], bb[ct]);
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

}  // namespace upd
}  // namespace gbr

// ---------------------------------------------------------------------------
// Split-precision (Ozaki) update tile: the same Y <- Y U in emulated FP64.
//
// Each FP64 operand is written as OZ_SLICES = 7 signed 8-bit digits relative
// to the largest exponent of its row (Y) or column (U): 56 bits, truncated.
// Digit matrices are exact in bf16, and a product of two digit matrices over
// K <= 128 stays below 255^2 * 128 < 2^23, so the bf16 tensor cores with FP32
// accumulation compute it exactly.  The 28 products with p + q <= 8 (slices
// counted from 1) are summed exactly per diagonal d = p + q in int32, the
// diagonals are combined in a 128-bit integer by Horner's rule, and the
// result is rounded once to the nearest double; dropped terms and the
// truncation of the operands are below 2^-49 of |y|max |u|max per product
// sum, under the FP64 rounding of a K = 128 dot product.  No FP64 arithmetic.
//
// U's digits (per window, from the window task) are used one half of the
// output columns at a time, resident in shared memory while every row of the
// task streams through; the task first copies its rows of Y to a per-CTA
// scratch so that the outputs can be written in place.
// ---------------------------------------------------------------------------
namespace gbr {
namespace oz {

constexpr int BR = 32;                // rows per pass
constexpr int NH = 64;                // output columns per half
constexpr int LDK = WMAX + 8;         // bf16 pitch along K (conflict-free fragment loads)
constexpr size_t kSmem = (size_t)OZ_SLICES * NH * LDK * 2 + (size_t)OZ_SLICES * BR * LDK * 2 +
                         (size_t)(BR + NH) * 4;

__device__ __forceinline__ unsigned ld_u32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const unsigned*>(p);
}

__device__ __forceinline__ void mma_bf16(float* c, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Signed 128-bit integer (hi, lo) times 2^(xe) rounded to the nearest double.
__device__ __forceinline__ double i128_to_double(long long hi, unsigned long long lo, int xe) {
    const bool neg = hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1 : 0);
    }
    const unsigned long long uh = (unsigned long long)hi;
    if (uh == 0ull && lo == 0ull) return 0.0;
    const int L = uh ? 64 + 63 - __clzll((long long)uh) : 63 - __clzll((long long)lo);
    unsigned long long m;
    const int sh = L - 52;
    if (sh > 0) {
        // sh <= 64 + 63 - 52: the value has at most 75 bits here, so sh < 64
        m = (uh << (64 - sh)) | (lo >> sh);
        const unsigned long long rem = lo & ((1ull << sh) - 1ull);
        const unsigned long long half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) ++m;
    } else {
        m = lo << (-sh);
    }
    int L2 = L;
    if (m >> 53) {  // rounding carried into a new bit
        m >>= 1;
        ++L2;
    }
    const int biased = L2 + xe + 1023;
    if (biased <= 0) return neg ? -0.0 : 0.0;
    if (biased >= 2047) return neg ? -__longlong_as_double(0x7ff0000000000000ll)
                                   : __longlong_as_double(0x7ff0000000000000ll);
    const unsigned long long bits = ((unsigned long long)neg << 63) |
                                    ((unsigned long long)biased << 52) | (m & 0xfffffffffffffull);
    return __longlong_as_double((long long)bits);
}

}  // namespace oz
}  // namespace gbr

namespace gbr {
namespace upd {

// Rows [y0, y0 + rows) of Y (rows <= UPD_FAR) <- (Y U) rows in emulated FP64.
// uslices: the window's U digits and column exponents (window task);
// scratch: UPD_FAR x WMAX doubles owned by this CTA.  blockDim.x = 512.
__device__ __forceinline__ void update_tile_ozaki(double* base, long long rs, long long ks, int y0,
                                                  int rows, int w,
                                                  const unsigned char* __restrict__ uslices,
                                                  double* __restrict__ scratch,
                                                  unsigned char* smem_raw) {
    using namespace oz;
    __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(smem_raw);       // [slice][NH][LDK]
    __nv_bfloat16* As = Bs + (size_t)OZ_SLICES * NH * LDK;                 // [slice][BR][LDK]
    int* rexp = reinterpret_cast<int*>(As + (size_t)OZ_SLICES * BR * LDK); // [BR]
    int* cexp = rexp + BR;                                                 // [NH]
    const __nv_bfloat16* udig = reinterpret_cast<const __nv_bfloat16*>(uslices);
    const int* ucexp = reinterpret_cast<const int*>(uslices + OZ_UDIG_ELEMS * 2);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;

    // 1. this task's rows of Y, row-major, to the CTA's scratch
    if (rs == 1) {
        for (int i = tid; i < rows * w; i += nth) {
            const int r = i % rows, k = i / rows;
            __stcg(&scratch[r * WMAX + k], __ldcg(&base[(y0 + r) + (long long)k * ks]));
        }
    } else {
        for (int i = tid; i < rows * w; i += nth) {
            const int k = i % w, r = i / w;
            __stcg(&scratch[r * WMAX + k], __ldcg(&base[(long long)(y0 + r) * rs + k]));
        }
    }
    __threadfence_block();
    __syncthreads();

    const int halves = (w + NH - 1) / NH;
    for (int h = 0; h < halves; ++h) {
        // 2. U digits of output columns [h NH, h NH + NH), all K, and their exponents
        for (int i = tid; i < OZ_SLICES * NH * (WMAX / 8); i += nth) {
            const int kv = i % (WMAX / 8), rest = i / (WMAX / 8);
            const int nl = rest % NH, q = rest / NH;
            const uint4 v = __ldcg(reinterpret_cast<const uint4*>(
                udig + ((size_t)q * WMAX + h * NH + nl) * WMAX + kv * 8));
            *reinterpret_cast<uint4*>(Bs + ((size_t)q * NH + nl) * LDK + kv * 8) = v;
        }
        for (int i = tid; i < NH; i += nth) cexp[i] = __ldcg(&ucexp[h * NH + i]);
        for (int p0 = 0; p0 < rows; p0 += BR) {
            const int pr = min(BR, rows - p0);
            __syncthreads();
            // 3. row exponents of this pass: one warp per row
            for (int r = warp; r < BR; r += nth / 32) {
                int em = 0;
                if (r < pr)
                    for (int k = lane; k < w; k += 32) {
                        const int e = (int)((((unsigned long long)__double_as_longlong(
                                                 __ldcg(&scratch[(p0 + r) * WMAX + k]))) >> 52) & 0x7ff);
                        em = e > em ? e : em;
                    }
                for (int o = 16; o; o >>= 1) {
                    const int v = __shfl_xor_sync(0xffffffffu, em, o);
                    em = v > em ? v : em;
                }
                if (lane == 0) rexp[r] = em;
            }
            __syncthreads();
            // 4. Y digits of this pass (zero beyond the rows and beyond w)
            for (int i = tid; i < BR * WMAX; i += nth) {
                const int r = i / WMAX, k = i % WMAX;
                bool neg = false;
                unsigned long long F = 0ull;
                if (r < pr && k < w)
                    F = win::oz_fixed(__ldcg(&scratch[(p0 + r) * WMAX + k]), rexp[r], &neg);
#pragma unroll
                for (int p = 0; p < OZ_SLICES; ++p) {
                    const int d = (int)((F >> (48 - 8 * p)) & 255ull);
                    As[((size_t)p * BR + r) * LDK + k] = __int2bfloat16_rn(neg ? -d : d);
                }
            }
            __syncthreads();
            // 5. products: warp -> output tile rows 16 (warp & 1) .., columns 8 (warp >> 1) ..
            {
                const int mt = warp & 1, nt = warp >> 1;
                const int ra = mt * 16 + g, nb = nt * 8 + g;
                // R[q - 1][i]: exact int32 sum of the products on diagonal p + q
                // (at most 7 terms below 2^23).  Diagonal p + 1 is complete once
                // slice p is done; T takes it by Horner's rule, highest weight first.
                int R[OZ_SLICES][4];
#pragma unroll
                for (int q = 0; q < OZ_SLICES; ++q)
#pragma unroll
                    for (int i = 0; i < 4; ++i) R[q][i] = 0;
                long long thi[4] = {0, 0, 0, 0};
                unsigned long long tlo[4] = {0, 0, 0, 0};
#pragma unroll 1
                for (int p = 1; p <= OZ_SLICES; ++p) {
                    // A fragments of digit slice p for this warp's 16 rows, all of K
                    const __nv_bfloat16* A = As + (size_t)(p - 1) * BR * LDK;
                    unsigned af[WMAX / 16][4];
#pragma unroll
                    for (int kk = 0; kk < WMAX / 16; ++kk) {
                        af[kk][0] = ld_u32(A + (size_t)ra * LDK + kk * 16 + 2 * t4);
                        af[kk][1] = ld_u32(A + (size_t)(ra + 8) * LDK + kk * 16 + 2 * t4);
                        af[kk][2] = ld_u32(A + (size_t)ra * LDK + kk * 16 + 2 * t4 + 8);
                        af[kk][3] = ld_u32(A + (size_t)(ra + 8) * LDK + kk * 16 + 2 * t4 + 8);
                    }
#pragma unroll
                    for (int q = 1; q <= OZ_SLICES; ++q) {
                        if (q > OZ_SLICES + 1 - p) break;
                        const __nv_bfloat16* B = Bs + (size_t)(q - 1) * NH * LDK + (size_t)nb * LDK;
                        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int kk = 0; kk < WMAX / 16; ++kk)
                            mma_bf16(c, af[kk][0], af[kk][1], af[kk][2], af[kk][3],
                                     ld_u32(B + kk * 16 + 2 * t4), ld_u32(B + kk * 16 + 2 * t4 + 8));
#pragma unroll
                        for (int i = 0; i < 4; ++i) R[q - 1][i] += __float2int_rn(c[i]);  // exact
                    }
                    // T <- T 2^8 + (diagonal p + 1); the other sums move down one slot
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        thi[i] = (long long)(((unsigned long long)thi[i] << 8) | (tlo[i] >> 56));
                        const unsigned long long sh = tlo[i] << 8;
                        const unsigned long long add = (unsigned long long)(long long)R[0][i];
                        tlo[i] = sh + add;
                        thi[i] += (tlo[i] < sh ? 1 : 0) - (R[0][i] < 0 ? 1 : 0);
                    }
#pragma unroll
                    for (int q = 0; q + 1 < OZ_SLICES; ++q)
#pragma unroll
                        for (int i = 0; i < 4; ++i) R[q][i] = R[q + 1][i];
#pragma unroll
                    for (int i = 0; i < 4; ++i) R[OZ_SLICES - 1][i] = 0;
                }
                // value = T 2^-64 2^(er - 1022) 2^(en - 1022); c layout: (g, 2t), (g, 2t+1),
                // (g + 8, 2t), (g + 8, 2t + 1)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = mt * 16 + g + (i >= 2 ? 8 : 0);
                    const int nl = nt * 8 + 2 * t4 + (i & 1);
                    const int n = h * NH + nl;
                    if (r >= pr || n >= w) continue;
                    const int xe = -64 + (rexp[r] - 1022) + (cexp[nl] - 1022);
                    const double v = (rexp[r] == 0 || cexp[nl] == 0) ? 0.0
                                                                     : oz::i128_to_double(thi[i], tlo[i], xe);
                    __stcg(&base[(long long)(y0 + p0 + r) * rs + (long long)n * ks], v);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace upd
}  // namespace gbr
