// Generalized reordering of a matrix pair (S, T) with Q and Z (Section 2,
// Eq. 7, second form): structure scans of the pair, the per-window launches
// (window task + off-diagonal updates of S, T, Q, Z), and the C-ABI entry
// points gbr_reorder_gen / gbr_reorder_gen_host.
//
// The planner, the window chains and the update tiles are those of the
// standard form (the block structure lives in S alone); the window task
// accumulates two factors, UQ (rows, applied from the left to S and T and
// to Q's columns) and UZ (columns: S, T and Z), and every update tile is the
// FP64 tensor-core product Y <- Y U of update_body.cuh.
#include "gen_body.cuh"
#include "host.h"
#include "update_body.cuh"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <vector>

namespace gbr {

namespace {

// One warp per column j: S is zero two or more below the diagonal, T below
// the diagonal; a 2x2 block of S does not overlap the next one and the 2x2
// pencil (S_b, T_b) has a complex-conjugate pair: b^2 < 4ac for
// det(S_b - lambda T_b) = a lambda^2 - b lambda + c.
__global__ void validate_gen_kernel(int n, const double* __restrict__ S, int ldS,
                                    const double* __restrict__ T, int ldT,
                                    DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nwarps) {
        bool bad = false;
        const double* cs = S + cm(0, j, ldS);
        const double* ct = T + cm(0, j, ldT);
        for (int i = j + 1 + lane; i < n; i += 32) bad |= (ct[i] != 0.0) || (i >= j + 2 && cs[i] != 0.0);
        if (lane == 0 && j + 1 < n && cs[j + 1] != 0.0) {
            if (j + 2 < n && S[cm(j + 2, j + 1, ldS)] != 0.0) bad = true;
            const double s11 = cs[j], s21 = cs[j + 1];
            const double s12 = S[cm(j, j + 1, ldS)], s22 = S[cm(j + 1, j + 1, ldS)];
            const double t11 = ct[j], t12 = T[cm(j, j + 1, ldT)], t22 = T[cm(j + 1, j + 1, ldT)];
            const double a = t11 * t22, b = s11 * t22 + s22 * t11 - s21 * t12, c = s11 * s22 - s12 * s21;
            if (!(b * b < 4.0 * a * c)) bad = true;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMin(&ctr->bad_column, j);
    }
}

// Generalized eigenvalue at diagonal position i: s/t for a 1x1 block; for
// the 2x2 block the roots of a lambda^2 - b lambda + c, positive imaginary
// part on the block's first row (a real pair, possible only after rounding,
// gives its larger root first).
__global__ void eigs_gen_kernel(int n, const double* __restrict__ S, int ldS,
                                const double* __restrict__ T, int ldT, double* __restrict__ wr,
                                double* __restrict__ wi) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int j = -1, row = 0;
        if (i + 1 < n && S[cm(i + 1, i, ldS)] != 0.0) j = i;
        else if (i > 0 && S[cm(i, i - 1, ldS)] != 0.0) { j = i - 1; row = 1; }
        if (j < 0) {
            wr[i] = S[cm(i, i, ldS)] / T[cm(i, i, ldT)];
            wi[i] = 0.0;
            continue;
        }
        const double s11 = S[cm(j, j, ldS)], s21 = S[cm(j + 1, j, ldS)];
        const double s12 = S[cm(j, j + 1, ldS)], s22 = S[cm(j + 1, j + 1, ldS)];
        const double t11 = T[cm(j, j, ldT)], t12 = T[cm(j, j + 1, ldT)], t22 = T[cm(j + 1, j + 1, ldT)];
        const double a = t11 * t22, b = s11 * t22 + s22 * t11 - s21 * t12, c = s11 * s22 - s12 * s21;
        const double d = 4.0 * a * c - b * b;
        const double mid = b / (2.0 * a);
        if (d > 0.0) {
            const double im = sqrt(d) / (2.0 * fabs(a));
            wr[i] = mid;
            wi[i] = row ? -im : im;
        } else {
            const double r = sqrt(-d) / (2.0 * fabs(a));
            wr[i] = row ? mid - r : mid + r;
            wi[i] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(gen::GEN_THREADS, 1)
window_gen_kernel(int n, double* __restrict__ S, int ldS, double* __restrict__ T, int ldT, int s0,
                  int w, uint8_t* __restrict__ gsel, double* __restrict__ UQg,
                  double* __restrict__ UZg, int strong, DevCounters* __restrict__ ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    gen::window_gen_body(n, S, ldS, T, ldT, s0, w, gsel, UQg, UZg, strong, ctr, smem_raw);
}

// Off-diagonal updates of one window of the pair: one CTA per BM-row tile
// of the panels, in this order:
//   0 S left  (UQ^T)   1 T left  (UQ^T)   2 S right (UZ)   3 T right (UZ)
//   4 Q       (UQ)     5 Z       (UZ)
struct GenPanels {
    int cnt[6];
};

__global__ void __launch_bounds__(upd::UPD_THREADS, 1)
update_gen_kernel(int n, int s, int e, double* __restrict__ S, int ldS, double* __restrict__ T,
                  int ldT, double* __restrict__ Q, int ldQ, double* __restrict__ Z, int ldZ,
                  const double* __restrict__ UQg, const double* __restrict__ UZg, GenPanels pc,
                  DevCounters* ctr, int fma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int b = blockIdx.x, k = 0;
    while (k < 5 && b >= pc.cnt[k]) b -= pc.cnt[k++];
    double* base;
    long long rs, ks;
    int R;
    const bool onT = (k == 1 || k == 3 || k == 5);
    const int panel = k < 2 ? upd::PANEL_L : (k < 4 ? upd::PANEL_R : upd::PANEL_Q);
    upd::panel_geom(panel, n, s, e, onT ? T : S, onT ? ldT : ldS, onT ? Z : Q, onT ? ldZ : ldQ,
                    &base, &rs, &ks, &R);
    const double* U = (k == 0 || k == 1 || k == 4) ? UQg : UZg;
    const int r0 = b * upd::BM;
    if (fma)
        upd::update_tile_fma(base, rs, ks, r0, min(upd::BM, R - r0), e - s, U, true, smem_raw,
                             ctr ? &ctr->upd_issued : nullptr);
    else
        upd::update_tile(base, rs, ks, r0, min(upd::BM, R - r0), e - s, U, true, smem_raw,
                         ctr ? &ctr->upd_issued : nullptr);
}

bool g_win_cfg[64], g_upd_cfg[64];

cudaError_t configure(const void* fn, size_t smem, bool* done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

}  // namespace

cudaError_t launch_validate_gen(int n, const double* S, int ldS, const double* T, int ldT,
                                DevCounters* ctr, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = 256, grid = std::min(1024, (n * 32 + threads - 1) / threads);
    validate_gen_kernel<<<grid, threads, 0, st>>>(n, S, ldS, T, ldT, ctr);
    return cudaGetLastError();
}

cudaError_t launch_eigs_gen(int n, const double* S, int ldS, const double* T, int ldT, double* wr,
                            double* wi, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = 256, grid = std::min(1024, (n + threads - 1) / threads);
    eigs_gen_kernel<<<grid, threads, 0, st>>>(n, S, ldS, T, ldT, wr, wi);
    return cudaGetLastError();
}

cudaError_t launch_window_gen(int n, const Window& wd, double* S, int ldS, double* T, int ldT,
                              uint8_t* sel, double* UQ, double* UZ, int strong, DevCounters* ctr,
                              cudaStream_t st) {
    cudaError_t e = configure((const void*)window_gen_kernel, gen::kGenWindowSmem, g_win_cfg);
    if (e != cudaSuccess) return e;
    window_gen_kernel<<<1, gen::GEN_THREADS, gen::kGenWindowSmem, st>>>(
        n, S, ldS, T, ldT, wd.s, wd.e - wd.s, sel, UQ, UZ, strong, ctr);
    return cudaGetLastError();
}

cudaError_t launch_update_gen(int n, const Window& wd, double* S, int ldS, double* T, int ldT,
                              double* Q, int ldQ, double* Z, int ldZ, const double* UQ,
                              const double* UZ, DevCounters* ctr, cudaStream_t st, bool fma) {
    cudaError_t e = configure((const void*)update_gen_kernel, upd::kUpdateSmem, g_upd_cfg);
    if (e != cudaSuccess) return e;
    const int BM = upd::BM;
    GenPanels pc;
    pc.cnt[0] = pc.cnt[1] = (n - wd.e + BM - 1) / BM;
    pc.cnt[2] = pc.cnt[3] = (wd.s + BM - 1) / BM;
    pc.cnt[4] = Q ? (n + BM - 1) / BM : 0;
    pc.cnt[5] = Z ? (n + BM - 1) / BM : 0;
    int grid = 0;
    for (int k = 0; k < 6; ++k) grid += pc.cnt[k];
    if (grid == 0) return cudaSuccess;
    update_gen_kernel<<<grid, upd::UPD_THREADS, upd::kUpdateSmem, st>>>(
        n, wd.s, wd.e, S, ldS, T, ldT, Q, ldQ, Z, ldZ, UQ, UZ, pc, ctr, fma ? 1 : 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reorder of a device-resident pair.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Duration model of the queue order: a pair window task at w = 128
// equivalent (the model scales it as w^2), in microseconds.
constexpr double kGenWinUs128 = 4.0 * 2000.0;

// Window and chain of a generalized call: the window is capped at gen::GW
// (the factors UQ and UZ both live in shared memory), and with the cap the
// chain at half of it.
void gen_window(const gbr_opts& o, int* w, int* m) {
    *w = o.window;
    *m = o.chain;
    if (*w > gen::GW) {
        *w = gen::GW;
        *m = std::min(*m, gen::GW / 2);
    }
}

// One planned pass through the persistent scheduler: the generalized
// instance's window tasks run window_gen_body, its tiles update S and T
// (left by UQ, right by UZ), Q (UQ) and Z (UZ).  A large pass runs as
// chunked launches like a pass of a standard form.
int run_persistent_gen(int n, const std::vector<Window>& wins, double* S, int ldS, double* T,
                       int ldT, double* Q, int ldQ, double* Z, int ldZ, uint8_t* d_sel,
                       DevCounters* d_ctr, const gbr_opts& o, long long* ntasks_out,
                       double* ms_out, long long* launches_out, SchedInfo* info, cudaStream_t st) {
    PassLaunch pl{};
    pl.inst = Inst{S, Q, d_sel, d_ctr, n, ldS, ldQ, 0, T, Z, ldT, ldZ};
    pl.cm.lr_mats = 2.0;
    pl.cm.win_us_128 = kGenWinUs128;
    if (o.precision == GBR_PREC_OZAKI) pl.cm.tile_rate = 100000.0;
    if (o.precision == GBR_PREC_FMA) pl.cm.tile_rate = 7600.0;
    pl.slot[0] = POOL_GEN_SCHED;
    pl.slot[1] = POOL_GEN_SCHED_ALT;
    pl.mode = 1;
    pl.timeout_msg = "persistent scheduler (pair): a task waited longer than wait_limit_ms";
    return run_pass_persistent(wins, pl, o, ntasks_out, ms_out, launches_out, info, st);
}

int reorder_gen_device(int n, double* S, int ldS, double* T, int ldT, double* Q, int ldQ, double* Z,
                       int ldZ, const int* select, double* eig_re, double* eig_im, int* m_out,
                       const gbr_opts& o, gbr_stats* stats, cudaStream_t st) {
    const size_t off_sub = 256, off_sel = off_sub + al256(n), off_eig = off_sel + al256(n),
                 off_u = off_eig + al256(2 * (size_t)n * sizeof(double)),
                 total = off_u + 2 * (size_t)gen::GW * gen::GW * sizeof(double);
    char* b = nullptr;
    int rc = pool_get(POOL_GEN_SCRATCH, total, (void**)&b);
    if (rc) return rc;
    DevCounters* d_ctr = (DevCounters*)b;
    uint8_t* d_sub = (uint8_t*)(b + off_sub);
    uint8_t* d_sel = (uint8_t*)(b + off_sel);
    double* d_eig = (double*)(b + off_eig);
    double* d_uq = (double*)(b + off_u);
    double* d_uz = d_uq + gen::GW * gen::GW;

    DevCounters h_ctr{0, 0, INT_MAX, 0, 0, 0};
    GBR_CK(cudaMemcpyAsync(d_ctr, &h_ctr, sizeof h_ctr, cudaMemcpyHostToDevice, st), "H2D counters");
    if (o.validate) GBR_CK(launch_validate_gen(n, S, ldS, T, ldT, d_ctr, st), "validate kernel");
    GBR_CK(launch_subdiag(n, S, ldS, d_sub, st), "subdiag kernel");
    std::vector<uint8_t> sub(n), sel(n);
    GBR_CK(cudaMemcpyAsync(sub.data(), d_sub, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
    GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (h_ctr.bad_column != INT_MAX) return -2;
    const int msel = selection_positions(n, sub.data(), select, sel.data());
    GBR_CK(cudaMemcpyAsync(d_sel, sel.data(), n, cudaMemcpyHostToDevice, st), "H2D selection");

    int w, m;
    gen_window(o, &w, &m);
    std::vector<cudaEvent_t> evw, evu;
    struct Cleanup {
        std::vector<cudaEvent_t>* a;
        std::vector<cudaEvent_t>* b;
        ~Cleanup() {
            for (cudaEvent_t e : *a) cudaEventDestroy(e);
            for (cudaEvent_t e : *b) cudaEventDestroy(e);
        }
    } cleanup{&evw, &evu};
    auto mark = [&](std::vector<cudaEvent_t>& v) -> cudaError_t {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        v.push_back(ev);
        return cudaEventRecord(ev, st);
    };
    long long launches = o.validate ? 2 : 1, nwin = 0;
    int nchains = 0;
    double flops = 0.0;
    unsigned long long seen_rej = 0;
    long long ntasks = 0;
    double ms_sched = 0.0;
    SchedInfo info_all;
    PlanState ps;
    init_state(ps, n, sub.data(), sel.data());
    for (int pass = 0; pass < 1 + 2 * n; ++pass) {
        std::vector<Window> win;
        plan_pass(ps, w, m, win, nchains);
        if (win.empty()) break;
        // S, T left and right, Q and Z: 2 w^2 flops per panel row each
        for (const Window& wd : win) {
            const double ww = (double)(wd.e - wd.s) * (wd.e - wd.s);
            flops += 2.0 * ww * (2.0 * (n - wd.e) + 2.0 * wd.s + (Q ? n : 0) + (Z ? n : 0));
        }
        if (o.sched == GBR_SCHED_PERSISTENT) {
            SchedInfo inf;
            rc = run_persistent_gen(n, win, S, ldS, T, ldT, Q, ldQ, Z, ldZ, d_sel, d_ctr, o, &ntasks,
                                    &ms_sched, &launches, &inf, st);
            if (rc) return rc;
            info_all.cp_us = inf.cp_us;
            info_all.sim_us = inf.sim_us;
            info_all.graph_ms += inf.graph_ms;
            info_all.order_ms += inf.order_ms;
        } else
        for (const Window& wd : win) {
            if (o.timing) GBR_CK(mark(evw), "event");
            GBR_CK(launch_window_gen(n, wd, S, ldS, T, ldT, d_sel, d_uq, d_uz, o.strong_test, d_ctr, st),
                   "window kernel (pair)");
            if (o.timing) { GBR_CK(mark(evw), "event"); GBR_CK(mark(evu), "event"); }
            GBR_CK(launch_update_gen(n, wd, S, ldS, T, ldT, Q, ldQ, Z, ldZ, d_uq, d_uz, d_ctr, st,
                                     o.precision == GBR_PREC_FMA),
                   "update kernel (pair)");
            if (o.timing) GBR_CK(mark(evu), "event");
            launches += 2;
        }
        nwin += (long long)win.size();
        GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        if (h_ctr.rejected == seen_rej) break;
        seen_rej = h_ctr.rejected;
        GBR_CK(launch_subdiag(n, S, ldS, d_sub, st), "subdiag kernel");
        GBR_CK(cudaMemcpyAsync(sub.data(), d_sub, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
        GBR_CK(cudaMemcpyAsync(sel.data(), d_sel, n, cudaMemcpyDeviceToHost, st), "D2H selection");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        init_state(ps, n, sub.data(), sel.data());
        launches += 1;
    }
    if (eig_re || eig_im) {
        GBR_CK(launch_eigs_gen(n, S, ldS, T, ldT, d_eig, d_eig + n, st), "eigenvalue kernel (pair)");
        if (eig_re)
            GBR_CK(cudaMemcpyAsync(eig_re, d_eig, n * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "D2H eig_re");
        if (eig_im)
            GBR_CK(cudaMemcpyAsync(eig_im, d_eig + n, n * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "D2H eig_im");
        launches += 1;
    }
    GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    double msw = 0.0, msu = 0.0;
    for (size_t i = 0; i + 1 < evw.size(); i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, evw[i], evw[i + 1]) == cudaSuccess) msw += t;
    }
    for (size_t i = 0; i + 1 < evu.size(); i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, evu[i], evu[i + 1]) == cudaSuccess) msu += t;
    }
    if (h_ctr.step_overflow) {
        set_last_error("window kernel (pair) exceeded its step bound");
        return GBR_ERR_CUDA;
    }
    if (m_out) *m_out = msel;
    if (stats) {
        stats->swaps = (long long)h_ctr.swaps;
        stats->rejected = (long long)h_ctr.rejected;
        stats->windows = nwin;
        stats->chains = nchains;
        stats->launches = launches;
        stats->upd_flops = flops;
        stats->ms_window = msw;
        stats->ms_update = msu;
        stats->win_flops = (double)h_ctr.win_flops;
        stats->upd_flops_issued = (double)h_ctr.upd_issued;
        stats->ms_sched = ms_sched;
        stats->tasks = ntasks;
        stats->sched_cp_ms = ntasks ? info_all.cp_us / 1e3 : 0.0;
        stats->sched_sim_ms = ntasks ? info_all.sim_us / 1e3 : 0.0;
        stats->ms_graph = info_all.graph_ms;
        stats->ms_order = info_all.order_ms;
    }
    const long long rej = (long long)h_ctr.rejected;
    return rej > INT_MAX ? INT_MAX : (int)rej;
}

int gen_args(int n, const void* S, int ldS, const void* T, int ldT, const void* Q, int ldQ,
             const void* Z, int ldZ, const int* select, const gbr_opts& o) {
    const int ld1 = n > 1 ? n : 1;
    if (n < 0) return -1;
    if (n > 0 && (!S || !T)) return -2;
    if (ldS < ld1 || ldT < ld1) return -3;
    if ((Q && ldQ < ld1) || (Z && ldZ < ld1)) return -5;
    if (n > 0 && !select) return -6;
    if (o.window < 4 || o.window > WMAX || o.chain < 1 || o.chain > o.window - 2) return -10;
    if (o.sched != GBR_SCHED_PERSISTENT && o.sched != GBR_SCHED_SEQUENTIAL) return -10;
    if (o.precision != GBR_PREC_DMMA && o.precision != GBR_PREC_OZAKI &&
        o.precision != GBR_PREC_FMA)
        return GBR_ERR_UNSUPPORTED;
    // split precision runs on the persistent scheduler only
    if (o.precision == GBR_PREC_OZAKI &&
        (o.sched != GBR_SCHED_PERSISTENT || (o.slices != 0 && o.slices != OZ_SLICES)))
        return GBR_ERR_UNSUPPORTED;
    if (o.wait_limit_ms < 0) return -10;
    if (o.on_reject != GBR_ON_REJECT_CONTINUE) return GBR_ERR_UNSUPPORTED;
    return 0;
}

}  // namespace

}  // namespace gbr

using namespace gbr;

extern "C" {

int gbr_reorder_gen(int n, double* S, int ldS, double* T, int ldT, double* Q, int ldQ, double* Z,
                    int ldZ, const int* select, double* eig_re, double* eig_im, int* m_out,
                    const gbr_opts* opts, gbr_stats* stats, void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    gbr_opts o;
    if (opts) o = *opts; else gbr_default_opts(&o);
    int rc = gen_args(n, S, ldS, T, ldT, Q, ldQ, Z, ldZ, select, o);
    if (rc) return rc;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) {
        if (m_out) *m_out = 0;
        return 0;
    }
    rc = refuse_capture((cudaStream_t)cuda_stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(api_mutex());
    rc = reorder_gen_device(n, S, ldS, T, ldT, Q, ldQ, Z, ldZ, select, eig_re, eig_im, m_out, o,
                            stats, (cudaStream_t)cuda_stream);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gbr_reorder_gen_host(int n, double* S, int ldS, double* T, int ldT, double* Q, int ldQ,
                         double* Z, int ldZ, const int* select, double* eig_re, double* eig_im,
                         int* m_out, const gbr_opts* opts, gbr_stats* stats, void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    gbr_opts o;
    if (opts) o = *opts; else gbr_default_opts(&o);
    int rc = gen_args(n, S, ldS, T, ldT, Q, ldQ, Z, ldZ, select, o);
    if (rc) return rc;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) {
        if (m_out) *m_out = 0;
        return 0;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    rc = refuse_capture(st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(api_mutex());
    const size_t mat = (size_t)n * n * sizeof(double);
    double* d = nullptr;
    const int nm = 2 + (Q ? 1 : 0) + (Z ? 1 : 0);
    rc = pool_get(POOL_GEN_HOST, mat * nm, (void**)&d);
    if (rc) return rc;
    double* hs[4] = {S, T, Q, Z};
    const int lds[4] = {ldS, ldT, ldQ, ldZ};
    double* dv[4] = {nullptr, nullptr, nullptr, nullptr};
    int used = 0;
    CopyTimer ct(o.timing != 0 && stats != nullptr);
    ct.mark(0, st);
    for (int i = 0; i < 4; ++i) {
        if (!hs[i]) continue;
        dv[i] = d + (size_t)used * n * n;
        ++used;
        GBR_CK(cudaMemcpy2DAsync(dv[i], n * sizeof(double), hs[i], (size_t)lds[i] * sizeof(double),
                                 n * sizeof(double), n, cudaMemcpyHostToDevice, st), "H2D pair");
    }
    ct.mark(1, st);
    rc = reorder_gen_device(n, dv[0], n, dv[1], n, dv[2], n, dv[3], n, select, eig_re, eig_im, m_out,
                            o, stats, st);
    if (rc < 0) return rc;
    ct.mark(2, st);
    for (int i = 0; i < 4; ++i) {
        if (!hs[i]) continue;
        GBR_CK(cudaMemcpy2DAsync(hs[i], (size_t)lds[i] * sizeof(double), dv[i], n * sizeof(double),
                                 n * sizeof(double), n, cudaMemcpyDeviceToHost, st), "D2H pair");
    }
    ct.mark(3, st);
    GBR_CK(cudaStreamSynchronize(st), "sync");
    ct.report(stats);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // extern "C"
