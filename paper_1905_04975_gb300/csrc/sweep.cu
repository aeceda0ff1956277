// One bulge-chasing sweep of the Schur reduction on an upper Hessenberg H
// (Section 3.2): the window planner for chains of bulges, the window kernel
// (sweep_body.cuh), the Hessenberg check, and the C-ABI entry point
// gbr_qr_sweep.  The off-diagonal updates are the reordering's tiles
// (left: H[s:e, e:n] <- U^T ..., right: H[0:s, s:e] <- ... U, Q <- Q U).
#include "host.h"
#include "sweep_body.cuh"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <vector>

namespace gbr {

namespace {

// One warp per column j: entries two or more below the diagonal are zero.
__global__ void validate_hess_kernel(int n, const double* __restrict__ H, int ldH,
                                     DevCounters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = warp; j < n; j += nwarps) {
        bool bad = false;
        const double* col = H + cm(0, j, ldH);
        for (int i = j + 2 + lane; i < n; i += 32) bad |= (col[i] != 0.0);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMin(&ctr->bad_column, j);
    }
}

__global__ void __launch_bounds__(swp::SWEEP_THREADS, 1)
sweep_window_kernel(int n, double* __restrict__ H, int ldH, int s0, int w, int t0, int t1, int nb,
                    const double* __restrict__ sp, double* __restrict__ Ug,
                    DevCounters* __restrict__ ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    swp::sweep_body(n, H, ldH, s0, w, t0, t1, nb, sp, Ug, ctr, smem_raw);
}

bool g_sw_cfg[64];

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

cudaError_t launch_validate_hess(int n, const double* H, int ldH, DevCounters* ctr, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = 256, grid = std::min(1024, (n * 32 + threads - 1) / threads);
    validate_hess_kernel<<<grid, threads, 0, st>>>(n, H, ldH, ctr);
    return cudaGetLastError();
}

cudaError_t launch_sweep_window(int n, const SweepWin& sw, double* H, int ldH, const double* sp,
                                double* U, DevCounters* ctr, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !g_sw_cfg[dev]) {
        e = cudaFuncSetAttribute(sweep_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)swp::kSweepSmem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) g_sw_cfg[dev] = true;
    }
    sweep_window_kernel<<<1, swp::SWEEP_THREADS, swp::kSweepSmem, st>>>(
        n, H, ldH, sw.s, sw.e - sw.s, sw.t0, sw.t1, sw.nb, sp + 2 * sw.b0, U, ctr);
    return cudaGetLastError();
}

namespace {

// Window and chain of a sweep: w capped at the kernel's window, the chain
// (shifts per chain) so that its introductions fit in the first window
// (at most w / 6 bulges).
void sweep_shape(const gbr_opts& o, int* w, int* nbc) {
    *w = std::min(o.window, swp::SW);
    *nbc = std::max(1, std::min(o.chain / 2, *w / 6));
}

// Duration model of the queue order: a sweep window task at w = 128
// equivalent (the model scales it as w^2), in microseconds.
constexpr double kSweepWinUs128 = 650.0;

// All windows of the sweep through one persistent-scheduler launch (mode 2):
// window tasks chase the bulges, the tiles are the reordering's.
int run_persistent_sweep(int n, const std::vector<SweepWin>& sw, double* H, int ldH, double* Q,
                         int ldQ, const double* d_sp, DevCounters* d_ctr, const gbr_opts& o,
                         long long* ntasks_out, double* ms_out, SchedInfo* info, cudaStream_t st) {
    std::vector<InstPlan> plans(1);
    plans[0].d = Inst{H, Q, nullptr, d_ctr, n, ldH, ldQ, 0, nullptr, nullptr, 0, 0, d_sp};
    plans[0].wins.reserve(sw.size());
    for (const SweepWin& x : sw)
        plans[0].wins.push_back(Window{x.s, x.e, x.b0, 0, 0, x.t0, x.t1, x.b0, x.nb});
    CostModel cm;
    cm.win_us_128 = kSweepWinUs128;
    SchedLaunch L;
    int rc = sched_prepare(
        plans, o, cm, num_sms(),
        [](size_t b) -> void* {
            void* p = nullptr;
            return pool_get(POOL_SWEEP_SCHED, b, &p) ? nullptr : p;
        },
        &L, info, st);
    if (rc) return rc;
    L.P.mode = 2;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (o.timing) {
        GBR_CK(cudaEventCreate(&e0), "event");
        GBR_CK(cudaEventCreate(&e1), "event");
        GBR_CK(cudaEventRecord(e0, st), "event");
    }
    rc = sched_enqueue(L, st);
    if (rc) return rc;
    if (o.timing) GBR_CK(cudaEventRecord(e1, st), "event");
    int h_err = 0;
    GBR_CK(cudaMemcpyAsync(&h_err, L.P.err, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H err");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (o.timing) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            ms = 0.f;
            (void)cudaGetLastError();
        }
        *ms_out += ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (L.trace_bytes) {
        const int rct = store_trace(L);
        if (rct) return rct;
    }
    *ntasks_out += L.P.ntasks;
    if (h_err) {
        set_last_error("persistent scheduler (sweep): a task waited longer than wait_limit_ms");
        return GBR_ERR_TIMEOUT;
    }
    return 0;
}

int sweep_device(int n, double* H, int ldH, double* Q, int ldQ, int nshifts, const double* sr,
                 const double* si, const gbr_opts& o, gbr_stats* stats, cudaStream_t st) {
    const int nb = nshifts / 2;
    const size_t off_sp = 256, off_u = off_sp + al256(sizeof(double) * 2 * std::max(1, nb)),
                 total = off_u + sizeof(double) * swp::SW * swp::SW;
    char* b = nullptr;
    int rc = pool_get(POOL_SWEEP, total, (void**)&b);
    if (rc) return rc;
    DevCounters* d_ctr = (DevCounters*)b;
    double* d_sp = (double*)(b + off_sp);
    double* d_u = (double*)(b + off_u);
    DevCounters h_ctr{0, 0, INT_MAX, 0, 0, 0};
    // shift parameters per bulge: s = sigma1 + sigma2, p = sigma1 sigma2
    std::vector<double> sp(2 * std::max(1, nb));
    for (int j = 0; j < nb; ++j) {
        sp[2 * j] = sr[2 * j] + sr[2 * j + 1];
        sp[2 * j + 1] = sr[2 * j] * sr[2 * j + 1] - si[2 * j] * si[2 * j + 1];
    }
    GBR_CK(cudaMemcpyAsync(d_ctr, &h_ctr, sizeof h_ctr, cudaMemcpyHostToDevice, st), "H2D counters");
    GBR_CK(cudaMemcpyAsync(d_sp, sp.data(), sizeof(double) * sp.size(), cudaMemcpyHostToDevice, st),
           "H2D shifts");
    long long launches = 0;
    if (o.validate) {
        GBR_CK(launch_validate_hess(n, H, ldH, d_ctr, st), "validate kernel (Hessenberg)");
        GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        launches += 1;
        if (h_ctr.bad_column != INT_MAX) return -2;
    }
    int w, nbc;
    sweep_shape(o, &w, &nbc);
    std::vector<SweepWin> wins;
    if (plan_sweep(n, nb, w, nbc, wins)) return -10;
    double flops = 0.0;
    std::vector<cudaEvent_t> ev;
    struct Cleanup {
        std::vector<cudaEvent_t>* v;
        ~Cleanup() {
            for (cudaEvent_t e : *v) cudaEventDestroy(e);
        }
    } cleanup{&ev};
    auto mark = [&]() -> cudaError_t {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
        return cudaEventRecord(e, st);
    };
    double msw = 0.0, msu = 0.0, ms_sched = 0.0;
    long long ntasks = 0;
    SchedInfo inf;
    for (const SweepWin& sw : wins) {
        const double ww = (double)(sw.e - sw.s) * (sw.e - sw.s);
        flops += 2.0 * ww * ((n - sw.e) + sw.s + (Q ? n : 0));
    }
    if (o.sched == GBR_SCHED_PERSISTENT && !wins.empty()) {
        rc = run_persistent_sweep(n, wins, H, ldH, Q, ldQ, d_sp, d_ctr, o, &ntasks, &ms_sched, &inf, st);
        if (rc) return rc;
        launches += 1;
    } else
    for (const SweepWin& sw : wins) {
        if (o.timing) GBR_CK(mark(), "event");
        GBR_CK(launch_sweep_window(n, sw, H, ldH, d_sp, d_u, d_ctr, st), "sweep window kernel");
        if (o.timing) GBR_CK(mark(), "event");
        Window wd{sw.s, sw.e, 0, 0, 0};
        GBR_CK(launch_update(n, wd, H, ldH, Q, ldQ, d_u, d_ctr, st, o.precision == GBR_PREC_FMA),
               "update kernel (sweep)");
        if (o.timing) GBR_CK(mark(), "event");
        launches += 2;
    }
    GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    for (size_t i = 0; i + 2 < ev.size(); i += 3) {
        float a = 0.f, c = 0.f;
        if (cudaEventElapsedTime(&a, ev[i], ev[i + 1]) == cudaSuccess) msw += a;
        if (cudaEventElapsedTime(&c, ev[i + 1], ev[i + 2]) == cudaSuccess) msu += c;
    }
    if (stats) {
        stats->windows = (long long)wins.size();
        stats->chains = (nb + nbc - 1) / nbc;
        stats->launches = launches;
        stats->upd_flops = flops;
        stats->ms_window = msw;
        stats->ms_update = msu;
        stats->win_flops = (double)h_ctr.win_flops;
        stats->upd_flops_issued = (double)h_ctr.upd_issued;
        stats->ms_sched = ms_sched;
        stats->tasks = ntasks;
        stats->sched_cp_ms = ntasks ? inf.cp_us / 1e3 : 0.0;
        stats->sched_sim_ms = ntasks ? inf.sim_us / 1e3 : 0.0;
        stats->ms_graph = inf.graph_ms;
        stats->ms_order = inf.order_ms;
    }
    if (h_ctr.step_overflow) {
        set_last_error("sweep window exceeded its step bound");
        return GBR_ERR_CUDA;
    }
    return 0;
}

}  // namespace

}  // namespace gbr

using namespace gbr;

extern "C" {

int gbr_plan_sweep(int n, int nshifts, int window, int chain, int* out, int max_windows) {
    if (n < 0 || nshifts < 0 || (nshifts & 1)) return -1;
    if (window < 8 || window > WMAX || chain < 1) return -10;
    gbr_opts o;
    gbr_default_opts(&o);
    o.window = window;
    o.chain = chain;
    int w, nbc;
    sweep_shape(o, &w, &nbc);
    std::vector<SweepWin> wins;
    if (window < 8 || plan_sweep(n, nshifts / 2, w, nbc, wins)) return -10;
    if (out)
        for (int i = 0; i < (int)wins.size() && i < max_windows; ++i) {
            const SweepWin& x = wins[i];
            int* r = out + 6 * i;
            r[0] = x.s; r[1] = x.e; r[2] = x.t0; r[3] = x.t1; r[4] = x.b0; r[5] = x.nb;
        }
    return (int)wins.size();
}

int gbr_qr_sweep(int n, double* H, int ldH, double* Q, int ldQ, int nshifts, const double* shift_re,
                 const double* shift_im, const gbr_opts* opts, gbr_stats* stats,
                 void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    gbr_opts o;
    if (opts) {
        o = *opts;
    } else {
        // the measured best shape of a sweep (window 64, 16 shifts per chain)
        gbr_default_opts(&o);
        o.window = 64;
        o.chain = 16;
    }
    const int ld1 = n > 1 ? n : 1;
    if (n < 0) return -1;
    if (n > 0 && !H) return -2;
    if (ldH < ld1) return -3;
    if (Q && ldQ < ld1) return -5;
    if (nshifts < 0 || (nshifts & 1) || (nshifts > 0 && (!shift_re || !shift_im))) return -6;
    for (int j = 0; j + 1 < nshifts; j += 2) {
        const double a1 = shift_re[j], b1 = shift_im[j], a2 = shift_re[j + 1], b2 = shift_im[j + 1];
        if (!((b1 == 0.0 && b2 == 0.0) || (a1 == a2 && b1 == -b2))) return -6;
    }
    // a sweep window holds at least one bulge with room to move (w >= 8)
    if (o.window < 8 || o.window > WMAX || o.chain < 1) return -10;
    if (o.precision != GBR_PREC_DMMA && o.precision != GBR_PREC_FMA) return GBR_ERR_UNSUPPORTED;
    if (o.sched != GBR_SCHED_PERSISTENT && o.sched != GBR_SCHED_SEQUENTIAL) return -10;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n < 3 || nshifts == 0) return 0;
    int rc = refuse_capture((cudaStream_t)cuda_stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(api_mutex());
    rc = sweep_device(n, H, ldH, Q, ldQ, nshifts, shift_re, shift_im, o, stats,
                          (cudaStream_t)cuda_stream);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

}  // extern "C"
