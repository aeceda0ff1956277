// Split-precision (Ozaki) off-diagonal update Y <- Y U on the fifth-generation
// tensor cores (tcgen05 + tensor memory).  The windows, the swaps and the
// stability test stay in FP64; only the level-3 updates of Section 3.2 (the
// accumulated U applied to the left, right and Q panels) are emulated.
//
// Representation.  Every FP64 entry x of a row of Y (or a column of U) is
// scaled by the largest binary exponent field emax of its row (column) and
// written as a 55-bit fixed-point integer V = +-F, F = m 2^(2 + e - emax)
// truncated (m the 53-bit significand, e the exponent field of x), so that
// x = V 2^(emax - 1077).  V is split into 7 balanced base-256 digits,
//
//     V = d1 2^48 + d2 2^40 + ... + d7,   d2..d7 in [-128, 127], d1 in [-128, 128],
//
// computed from G = V + 0x808080808080: d1 = G >> 48 (arithmetic), dp =
// byte (7 - p) of G minus 128.  Digits are exact in bf16.
//
// Products.  For a K <= 128 contraction every slice product A_p B_q has
// integer entries of magnitude <= 128^2 * 128 = 2^21; the products on one
// diagonal d = p + q (at most 7 of them) sum to < 2^24, so they accumulate
// exactly in one FP32 accumulator in tensor memory.  The 28 products with
// p + q <= 8 fill 7 accumulators (d = 2..8) of 64 columns each, stored in
// order of d, so that the products of one Y slice p with the U slices
// q = 1..8-p hit consecutive accumulators and run as one or two MMAs of N up
// to 256 (the U slices are stacked along N).  The epilogue converts the
// accumulators to integers, combines them by Horner's rule in 128-bit
// integers,
//
//     T = sum_d D_d 256^(8 - d),   y u = T 2^-64 2^(er - 1021) 2^(ec - 1021),
//
// and rounds T once to the nearest double.  Per product term, the dropped
// digit products (p + q >= 9) and the truncation of both operands are below
// 2^-50 |y|max |u|max.  No FP64 arithmetic.
//
// Layout in shared memory (what the MMA reads): K-major, 128-byte swizzle:
// rows of 64 bf16 (128 B) whose 16-byte chunks are permuted by XOR with the
// row index mod 8, 8-row atoms of 1024 B; the two 64-wide halves of K are
// stored one after the other.  The window task writes U's digits in exactly
// this layout ([output half][K half][slice][column][128 B]), so one bulk
// asynchronous copy brings one half of U's slices into shared memory; Y's
// digits are generated by the CTA's threads.
#pragma once

#include <string.h>

#include "common.cuh"

namespace gbr {
namespace oz {

constexpr long long OZ_BIAS = 0x808080808080ll;  // 128 in each of the six low digit positions

// G = V + OZ_BIAS for the entry x of a row (column) with exponent field emax.
// Entries below the normal range count as zero.  Integer work only.
__host__ __device__ __forceinline__ long long oz_balanced(double x, int emax) {
#ifdef __CUDA_ARCH__
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, 8);
#endif
    const int e = (int)((b >> 52) & 0x7ff);
    const int sh = emax - e;
    if (e == 0 || sh >= 64) return OZ_BIAS;
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    long long F = (long long)((m << 2) >> sh);
    if (b >> 63) F = -F;
    return F + OZ_BIAS;
}

// Digit p (1..7) of G = (hi:lo) as an exact float.  For p >= 2 the byte is
// placed in the significand of 1.5 * 2^23 by a byte permute.
template <int P>
__device__ __forceinline__ float oz_digit(unsigned lo, unsigned hi) {
    if (P == 1) return __int_as_float(0x4B400000 + ((int)hi >> 16)) - 12582912.0f;
    const unsigned src = P <= 3 ? hi : lo;
    constexpr unsigned sel = 0x7640u | (unsigned)(P <= 3 ? 3 - P : 7 - P);
    return __uint_as_float(__byte_perm(src, 0x4B400000u, sel)) - 12583040.0f;
}

// Two floats holding small integers -> one bf16x2 word (exact: at most 8
// significant bits, so the low 16 bits of each float are zero).
__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi) {
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Byte offset of the 16-byte chunk c (0..7) of row r in a 128-byte-swizzled
// K-major block of 128-byte rows.
__host__ __device__ constexpr int sw128(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }

// The seven accumulators (FP32 bit patterns, diagonals 2..8) of one output ->
// y u, given the exponent fields of its row (er) and column (ec).  The
// accumulators hold exact integers; T = sum_d D_d 256^(8 - d) (|T| < 2^74) is
// formed in 128-bit integers and rounded once to the nearest double: |T| is
// shifted right by 0, 7 or 11 bits so that it fits 63 bits with at least 56
// significant bits whenever bits are dropped, the dropped bits are kept as a
// sticky bit in bit 0, and the 64-bit integer is converted with
// round-to-nearest-even.  Results below the normal range flush to zero.
__device__ __forceinline__ double oz_combine(const unsigned (&a)[7], int er, int ec) {
    if (er == 0 || ec == 0) return 0.0;
    int D[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) D[j] = __float2int_rn(__uint_as_float(a[j]));  // exact
    // D2..D6 by Horner in 64 bits (|.| < 2^57), then T = th 2^16 + D7 256 + D8
    long long th = D[0];
#pragma unroll
    for (int j = 1; j <= 4; ++j) th = th * 256 + D[j];
    const long long lowp = (long long)D[5] * 256 + (long long)D[6];
    const unsigned long long lo0 = (unsigned long long)th << 16;
    unsigned long long lo = lo0 + (unsigned long long)lowp;
    long long hi = (th >> 48) + (lo < lo0 ? 1 : 0) - (lowp < 0 ? 1 : 0);
    const bool neg = hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1 : 0);
    }
    const unsigned long long uh = (unsigned long long)hi;  // |T| = uh 2^64 + lo
    const int sh = uh >= 64ull ? 11 : ((uh != 0ull || (long long)lo < 0) ? 7 : 0);
    unsigned long long t = lo;
    if (sh) t = (uh << (64 - sh)) | (lo >> sh) | ((lo & ((1ull << sh) - 1ull)) != 0ull ? 1ull : 0ull);
    if (t == 0ull) return 0.0;
    long long bits = __double_as_longlong(__ull2double_rn(t));
    const int xe = sh - 64 + (er - 1021) + (ec - 1021);
    const int ef = (int)((bits >> 52) & 0x7ff) + xe;
    if (ef <= 0) return neg ? -0.0 : 0.0;
    if (ef >= 2047) bits = 0x7ff0000000000000ll;
    else bits += (long long)xe << 52;
    if (neg) bits |= (long long)(1ull << 63);
    return __longlong_as_double(bits);
}

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier / bulk-copy wrappers (inline PTX, sm_103a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Waits until the phase of the given parity has completed.  Bounded: about
// 2^26 polls (a second or more with the back-off); false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    for (int i = 0; i < (1 << 26); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (i >= 64) __nanosleep(32);
    }
    return false;
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One-dimensional bulk asynchronous copy global -> shared, completing on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {  // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // one whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 B apart (the leading byte offset is unused for this layout).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}
// Instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N given.
constexpr uint32_t TC_M = 128, TC_N = 64;
__host__ __device__ constexpr uint32_t idesc(uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((TC_M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, unsigned (&v)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                 : "=r"(v[0]), "=r"(v[1])
                 : "r"(taddr)
                 : "memory");
}
// Prefetch of one line of global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Tensor memory held by a CTA that runs split-precision tiles.
constexpr uint32_t TMEM_COLS = 512;

// Shared memory of the tile (offsets from a 1024-byte-aligned base).
constexpr int NACC = 7;                                    // accumulators: diagonals 2..8
constexpr size_t KH_ROW = 128;                             // bytes per row of one K half
constexpr size_t B_SLICE = (size_t)TC_N * KH_ROW;          // one K half of one U slice: 8 KB
constexpr size_t B_KH = (size_t)OZ_SLICES * B_SLICE;       // one K half of all slices: 56 KB
constexpr size_t B_BYTES = 2 * B_KH;                       // one output half of U: 112 KB
constexpr size_t A_KH = (size_t)TC_M * KH_ROW;             // one K half of a Y slice: 16 KB
constexpr size_t A_BYTES = 2 * A_KH;                       // one Y slice: 32 KB
constexpr size_t OFF_A = B_BYTES;
constexpr size_t OFF_RED = OFF_A + 2 * A_BYTES;            // int [4][128]: row exponents
constexpr size_t OFF_CEXP = OFF_RED + 4 * 128 * 4;         // int [2][64]: column exponents
constexpr size_t OFF_BAR = OFF_CEXP + 2 * TC_N * 4;        // 3 mbarriers
constexpr size_t kSmem = OFF_BAR + 3 * 8 + 1024;           // + alignment slack
constexpr int TILE_THREADS = 512;
static_assert(OZ_UDIG_ELEMS * 2 == 2 * B_BYTES, "U digit image = two output halves");

// Issues the products of Y digit slice p (shared memory, a_addr) with the U
// digit slices q = 1..8-p (b_addr): accumulators p-1..6, at most 4 per MMA.
__device__ __forceinline__ void issue_slice(int p, uint32_t a_addr, uint32_t b_addr, uint32_t tmem,
                                            int ksteps) {
    const int nq = 8 - p;
    for (int q0 = 1; q0 <= nq; q0 += 4) {
        const int cnt = min(4, nq - q0 + 1);
        const uint32_t id = idesc(64u * cnt);
        const uint32_t d = tmem + 64u * (uint32_t)(p + q0 - 2);
        const uint32_t bq = b_addr + (uint32_t)(q0 - 1) * (uint32_t)B_SLICE;
        for (int s = 0; s < ksteps; ++s) {
            const uint32_t off = (uint32_t)(s & 3) * 32u;  // K step of 16 within the 128 B row
            const uint32_t ka = a_addr + (uint32_t)(s >> 2) * (uint32_t)A_KH + off;
            const uint32_t kb = bq + (uint32_t)(s >> 2) * (uint32_t)B_KH + off;
            mma_bf16(d, sdesc(ka), sdesc(kb), id, (p == 1 && s == 0) ? 0u : 1u);
        }
    }
}

// Writes digit slice P of the thread's 4 chunks (row m, 16-byte chunks
// c16 = cq + 4 i of K, i.e. K columns 8 c16 .. 8 c16 + 7) into As.
template <int P>
__device__ __forceinline__ void put_slice(const long long (&G)[4][8], unsigned char* As, int m,
                                          int cq) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned wv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const long long g0 = G[i][2 * t], g1 = G[i][2 * t + 1];
            wv[t] = pack_bf16x2(oz_digit<P>((unsigned)g0, (unsigned)(g0 >> 32)),
                                oz_digit<P>((unsigned)g1, (unsigned)(g1 >> 32)));
        }
        const int c16 = cq + 4 * i;
        *reinterpret_cast<uint4*>(As + (c16 >> 3) * A_KH + sw128(m, c16 & 7)) =
            make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
}

template <int P>
__device__ __forceinline__ bool slice_step(const long long (&G)[4][8], unsigned char* sm,
                                           uint64_t* bar, uint32_t (&ph)[2], uint32_t tmem,
                                           int ksteps, int m, int cq) {
    constexpr int b = P & 1;
    unsigned char* As = sm + OFF_A + b * A_BYTES;
    bool ok = true;
    if (P >= 3) {  // the products of slice P - 2 read this buffer
        ok = mbar_wait(&bar[b], ph[b]);
        ph[b] ^= 1u;
    }
    put_slice<P>(G, As, m, cq);
    fence_async_smem();
    if (__syncthreads_or(!ok)) return false;
    if (threadIdx.x == 0) {
        tc_fence_after();
        issue_slice(P, smem_u32(As), smem_u32(sm), tmem, ksteps);
        mma_commit(&bar[b]);
    }
    return true;
}

// Staging of 128 rows x 64 columns of Y in shared memory for panels whose
// rows are contiguous in memory (ks == 1): element (r, c) at r * 64 +
// (c ^ (r & 15)), so that a half-warp touches 16 different bank pairs both
// when its lanes run along a row (global side) and down a column (one lane
// per row: digit generation and the accumulator read-out).
static_assert(2 * A_BYTES == (size_t)TC_M * 64 * sizeof(double), "staging = both slice buffers");
__device__ __forceinline__ int stg_idx(int r, int c) { return r * 64 + (c ^ (r & 15)); }

// Columns [k0, k0 + 64) of rows [row0, row0 + pr) into the staging area
// (zeros beyond w and beyond pr), coalesced along each row.
// Eight loads per thread are issued before the first store, so that their
// latencies overlap.
__device__ __forceinline__ void stage_rows_in(const double* base, long long rs, int row0, int pr,
                                              int k0, int w, double* stg) {
    constexpr int PER = (int)TC_M * 64 / TILE_THREADS;  // elements per thread
    static_assert(PER % 8 == 0, "whole batches of eight");
#pragma unroll 1
    for (int u0 = 0; u0 < PER; u0 += 8) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = threadIdx.x + (u0 + u) * TILE_THREADS;
            const int r = i >> 6, k = k0 + (i & 63);
            x[u] = (r < pr && k < w) ? __ldcg(&base[(long long)(row0 + r) * rs + k]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = threadIdx.x + (u0 + u) * TILE_THREADS;
            stg[stg_idx(i >> 6, i & 63)] = x[u];
        }
    }
}

// The staged outputs (columns [n0, n0 + 64) of rows [row0, row0 + pr)) back
// to Y, coalesced along each row.
__device__ __forceinline__ void stage_rows_out(double* base, long long rs, int row0, int pr, int n0,
                                               int w, const double* stg) {
    for (int i = threadIdx.x; i < pr * 64; i += TILE_THREADS) {
        const int r = i >> 6, c = i & 63, n = n0 + c;
        if (n < w) __stcg(&base[(long long)(row0 + r) * rs + n], stg[stg_idx(r, c)]);
    }
}

// Rows [y0, y0 + rows) of Y <- (Y U) rows, emulated FP64, in place.
// uslices: the window's U digits (written by its window task) and column
// exponents; tmem: the CTA's TMEM_COLS columns of tensor memory; smem_raw:
// at least kSmem bytes.  blockDim.x == TILE_THREADS.  Rows are read once per
// block of 128 into registers before any output of that block is written.
// Returns false (on every thread) if a wait for the tensor cores or the
// copy engine ran out.
static __device__ __noinline__ bool update_tile_tc(double* base, long long rs, long long ks, int y0,
                                            int rows, int w,
                                            const unsigned char* __restrict__ uslices,
                                            unsigned char* smem_raw, uint32_t tmem) {
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    int* red = reinterpret_cast<int*>(sm + OFF_RED);
    int* cexp = reinterpret_cast<int*>(sm + OFF_CEXP);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);  // A0, A1, B
    // left-panel staging (rows of Y contiguous): both slice buffers, free
    // while rows are read and after a block's products have completed
    double* stg = reinterpret_cast<double*>(sm + OFF_A);
    const int* ucexp = reinterpret_cast<const int*>(uslices + OZ_UDIG_ELEMS * 2);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ksteps = (w + 15) >> 4;
    const int halves = (w + (int)TC_N - 1) / (int)TC_N;
    const int passes = (rows + (int)TC_M - 1) / (int)TC_M;
    const int m = tid & 127, cq = tid >> 7;   // digit generation: row m, K chunks cq + 4 i
    const int lq = warp & 3, cc = warp >> 2;  // epilogue: TMEM lanes 32 lq.., columns 16 cc..
    uint32_t ph[2] = {0u, 0u}, phb = 0u;

    // U digits of output half h (all slices) by one bulk copy, and the
    // column exponents into cexp[h]
    auto load_u = [&](int h) {
        if (tid == 0) {
            mbar_expect_tx(&bar[2], (uint32_t)B_BYTES);
            bulk_g2s(sm, uslices + (size_t)h * B_BYTES, (uint32_t)B_BYTES, &bar[2]);
        }
        if (tid < (int)TC_N) cexp[h * TC_N + tid] = __ldcg(&ucexp[h * TC_N + tid]);
    };
    // the generic writes of earlier tasks are ordered before the copy
    fence_async_smem();
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_fence_init();
    }
    __syncthreads();
    load_u(0);
    bool loaded = true;  // a copy of U half 0 is in flight
    for (int pass = 0; pass < passes; ++pass) {
        const int p0 = pass * (int)TC_M, pr = min((int)TC_M, rows - p0);
        // 1. the thread's 32 entries (row m, 4 chunks of 8 K) and the row's
        // largest exponent field (4 threads per row, combined in shared memory)
        long long G[4][8];
        if (ks == 1) {
            // rows of Y are contiguous (left panel): read them coalesced into
            // the free slice buffers, 64 columns at a time, then take the
            // thread's entries from there
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
#pragma unroll
                for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                    for (int j = 0; j < 8; ++j) G[2 * kh + ii][j] = 0;
                if (kh * 64 < w) {
                    stage_rows_in(base, rs, y0 + p0, pr, kh * 64, w, stg);
                    __syncthreads();
#pragma unroll
                    for (int ii = 0; ii < 2; ++ii) {
                        const int c0 = 8 * cq + 32 * ii;   // K columns 64 kh + c0 .. + 7
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            G[2 * kh + ii][j] = __double_as_longlong(stg[stg_idx(m, c0 + j)]);
                    }
                    __syncthreads();
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k0 = 8 * (cq + 4 * i);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    double x = 0.0;
                    if (m < pr && k0 + j < w)
                        x = __ldcg(&base[(long long)(y0 + p0 + m) * rs + (long long)(k0 + j) * ks]);
                    G[i][j] = __double_as_longlong(x);
                }
            }
        }
        int em = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int e = (int)(((unsigned long long)G[i][j] >> 52) & 0x7ff);
                em = e > em ? e : em;
            }
        red[cq * 128 + m] = em;
        __syncthreads();
        const int er_gen = max(max(red[m], red[128 + m]), max(red[256 + m], red[384 + m]));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) G[i][j] = oz_balanced(__longlong_as_double(G[i][j]), er_gen);
        const int r_out = 32 * lq + lane;  // epilogue row (TMEM lane)
        const int er = (r_out < pr) ? max(max(red[r_out], red[128 + r_out]),
                                          max(red[256 + r_out], red[384 + r_out]))
                                    : 0;
        for (int h = 0; h < halves; ++h) {
            if (!loaded) load_u(h);
            loaded = false;
            bool ok = mbar_wait(&bar[2], phb);
            phb ^= 1u;
            if (__syncthreads_or(!ok)) return false;
            // 2. slices 1..7: digits into a double-buffered slice, products
            // issued by one thread while the next slice is generated
            if (!slice_step<1>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            if (!slice_step<2>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            if (!slice_step<3>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            if (!slice_step<4>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            if (!slice_step<5>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            if (!slice_step<6>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            if (!slice_step<7>(G, sm, bar, ph, tmem, ksteps, m, cq)) return false;
            ok = mbar_wait(&bar[0], ph[0]);
            ph[0] ^= 1u;
            ok = mbar_wait(&bar[1], ph[1]) && ok;
            ph[1] ^= 1u;
            tc_fence_after();
            // 3. the tensor cores are done with U: start the next half's copy
            // (two halves alternate; with one half U stays resident)
            if (halves == 2 && (h == 0 || pass + 1 < passes)) {
                fence_async_smem();
                if (__syncthreads_or(!ok)) return false;
                load_u(h ^ 1);
                loaded = true;
            } else if (halves == 1) {
                loaded = true;
                if (tid == 0) mbar_arrive(&bar[2]);  // U stays: an empty phase for the next wait
            }
            // the next block's rows into L2 while this block's last epilogue runs
            if (h == halves - 1 && pass + 1 < passes) {
                const int q0 = p0 + (int)TC_M, qn = min((int)TC_M, rows - q0);
                if (rs == 1) {
                    for (int i = tid; i < w * 8; i += TILE_THREADS) {
                        const int k = i >> 3, seg = i & 7;
                        if (seg * 16 < qn)
                            prefetch_l2(&base[(long long)(y0 + q0 + seg * 16) + (long long)k * ks]);
                    }
                } else {
                    for (int i = tid; i < qn * 8; i += TILE_THREADS) {
                        const int r = i >> 3, seg = i & 7;
                        if (seg * 16 < w) prefetch_l2(&base[(long long)(y0 + q0 + r) * rs + seg * 16]);
                    }
                }
            }
            // 4. epilogue: each thread one row (TMEM lane), 2 columns at a time
            const int hc = (halves == 2) ? h : 0;
#pragma unroll 1
            for (int c2 = 0; c2 < 8; ++c2) {
                const int col0 = 16 * cc + 2 * c2;
                unsigned v[NACC][2];
#pragma unroll
                for (int j = 0; j < NACC; ++j)
                    tmem_ld2(tmem + ((uint32_t)(32 * lq) << 16) + 64u * j + (uint32_t)col0, v[j]);
                tmem_wait_ld();
                if (ok && r_out < pr) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int n = h * (int)TC_N + col0 + c;
                        if (n < w) {
                            unsigned a[NACC];
#pragma unroll
                            for (int j = 0; j < NACC; ++j) a[j] = v[j][c];
                            const double y = oz_combine(a, er, cexp[hc * TC_N + col0 + c]);
                            if (ks == 1)
                                stg[stg_idx(r_out, col0 + c)] = y;
                            else
                                __stcg(&base[(long long)(y0 + p0 + r_out) * rs + (long long)n * ks],
                                       y);
                        }
                    }
                }
            }
            if (ks == 1) {
                // left panel: the staged outputs go out as contiguous row segments
                if (__syncthreads_or(!ok)) return false;
                stage_rows_out(base, rs, y0 + p0, pr, h * (int)TC_N, w, stg);
            }
            tc_fence_before();
            if (__syncthreads_or(!ok)) return false;
        }
    }
    // every copy started was waited for (the last half issues none), and the
    // empty phase armed with one half has completed: nothing is in flight
    if (tid == 0) {
        mbar_inval(&bar[0]);
        mbar_inval(&bar[1]);
        mbar_inval(&bar[2]);
    }
    __syncthreads();
    return true;
}

}  // namespace oz
}  // namespace gbr
