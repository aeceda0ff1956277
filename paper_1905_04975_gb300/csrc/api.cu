// C-ABI entry points for one reordering, the device scratch pool and the
// pass loop: plan (host), run the windows and updates (persistent scheduler
// or one window/update launch pair per window), re-plan after rejected swaps.
#include "host.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace gbr {

static std::vector<long long> g_trace;  // last traced persistent launch, 8 words per task

// ---------------------------------------------------------------------------
// Device scratch pool: one grow-only allocation per device and purpose.
// ---------------------------------------------------------------------------
enum PoolSlot { POOL_SCRATCH = 0, POOL_HOST_S = 1, POOL_HOST_Q = 2, POOL_SCHED = 3, POOL_PANEL = 4,
                POOL_EIGVEC = 5 };
static_assert(POOL_GEN_SCRATCH == 6 && POOL_GEN_HOST == 7 && POOL_GEN_SCHED == 8 &&
                  POOL_SWEEP == 9 && POOL_SWEEP_SCHED == 10 && POOL_SCHED_ALT == 11 &&
                  POOL_GEN_SCHED_ALT == 12 && POOL_NSLOTS == 13,
              "pool slots of the generalized entry points");
struct DevPool {
    void* ptr[POOL_NSLOTS] = {};
    size_t bytes[POOL_NSLOTS] = {};
};
static std::mutex g_mu;  // serializes calls: the pool is shared per device
static DevPool g_pool[64];

std::mutex& api_mutex() { return g_mu; }

int store_trace(const SchedLaunch& L) {
    const int nt = L.P.ntasks;
    std::vector<unsigned long long> raw((size_t)4 * nt);
    GBR_CK(cudaMemcpy(raw.data(), L.P.trace, sizeof(unsigned long long) * 4 * nt,
                      cudaMemcpyDeviceToHost), "D2H trace");
    g_trace.assign((size_t)8 * nt, 0);
    for (int q = 0; q < nt; ++q) {
        const SchedTask& k = L.tq[q];
        long long* r = &g_trace[(size_t)8 * q];
        r[0] = k.kind; r[1] = k.win; r[2] = k.y0; r[3] = k.rows;
        for (int j = 0; j < 4; ++j) r[4 + j] = (long long)raw[4 * q + j];
    }
    return 0;
}

int pool_get(int slot, size_t bytes, void** out) {
    int dev = 0;
    GBR_CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return GBR_ERR_CUDA;
    DevPool& p = g_pool[dev];
    if (p.bytes[slot] < bytes) {
        if (p.ptr[slot]) {
            GBR_CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
            cudaFree(p.ptr[slot]);
            p.ptr[slot] = nullptr;
            p.bytes[slot] = 0;
        }
        size_t grow = bytes + bytes / 4;
        GBR_CK(cudaMalloc(&p.ptr[slot], grow), "cudaMalloc(pool)");
        p.bytes[slot] = grow;
    }
    *out = p.ptr[slot];
    return 0;
}

// ---------------------------------------------------------------------------
// One planned pass through the persistent scheduler (one instance).
// ---------------------------------------------------------------------------
static SchedInfo g_last_sched;  // last persistent launch: task count, model, host times

static CostModel cost_model(const gbr_opts& o) {
    CostModel c;
    // one SM on an update tile: DMMA ~7.0 GFLOP/s; split precision ~33 GFLOP/s
    // FP64-equivalent (both measured on a panel of 256-row tiles)
    c.tile_rate = (o.precision == GBR_PREC_OZAKI) ? 100000.0
                : (o.precision == GBR_PREC_FMA)  ? 7600.0
                                                 : 6900.0;
    return c;
}

// A non-blocking stream per device for uploading the launch images of later
// chunks while an earlier chunk runs (created on first use, destroyed by
// gbr_release).
static cudaStream_t g_side[64];

static int side_stream(cudaStream_t* out) {
    int dev = 0;
    GBR_CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return GBR_ERR_CUDA;
    if (!g_side[dev])
        GBR_CK(cudaStreamCreateWithFlags(&g_side[dev], cudaStreamNonBlocking), "side stream");
    *out = g_side[dev];
    return 0;
}

// Cuts of one pass's window list (in pipeline order) into chunks that run as
// consecutive persistent launches.  Ordering the task graph of a large pass
// takes the host tens of milliseconds, during which the device would idle;
// with chunks, the first launch starts after the host has ordered only its
// first sixteenth, and each later chunk is planned, ordered and uploaded
// while the previous one runs.  Small passes, traced launches (one timeline)
// and ABORT (one abort word per launch) take one launch.
static std::vector<size_t> chunk_cuts(size_t nw, const gbr_opts& o) {
    std::vector<size_t> cuts{0};
    if (nw >= 1024 && o.timing < 2 && o.on_reject != GBR_ON_REJECT_ABORT) {
        cuts.push_back(nw / 16);
        cuts.push_back(nw / 4);
    }
    cuts.push_back(nw);
    return cuts;
}

static int read_err(const SchedLaunch& L, cudaStream_t s, int* acc) {
    int h = 0;
    GBR_CK(cudaMemcpyAsync(&h, L.P.err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H err");
    GBR_CK(cudaStreamSynchronize(s), "sync");
    *acc |= h;
    return 0;
}

// One planned pass through the persistent scheduler.  The windows are put in
// pipeline order and cut into chunks (chunk_cuts); a chunk is a prefix-closed
// part of that order (every window that overlaps one of its windows and
// comes earlier is in it or in an earlier chunk), so running the chunks one
// after another on the stream keeps every dependence.  Two launch images
// alternate between the pool slots pl.slot[0] and pl.slot[1].
int run_pass_persistent(const std::vector<Window>& wins, const PassLaunch& pl, const gbr_opts& o,
                        long long* ntasks_out, double* ms_out, long long* launches_out,
                        SchedInfo* info, cudaStream_t st) {
    std::vector<Window> all = wins;
    pipeline_order(pl.inst.n, all);
    const std::vector<size_t> cuts = chunk_cuts(all.size(), o);
    const int nch = (int)cuts.size() - 1;
    cudaStream_t up = st;
    if (nch > 1) {
        int rcs = side_stream(&up);
        if (rcs) return rcs;
    }
    // events: timing (e0, e1) and the end of the last chunk of each image
    struct Events {
        cudaEvent_t e[4] = {};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    if (o.timing) {
        GBR_CK(cudaEventCreate(&ev.e[0]), "event");
        GBR_CK(cudaEventCreate(&ev.e[1]), "event");
    }
    if (nch > 1) {
        GBR_CK(cudaEventCreateWithFlags(&ev.e[2], cudaEventDisableTiming), "event");
        GBR_CK(cudaEventCreateWithFlags(&ev.e[3], cudaEventDisableTiming), "event");
    }
    SchedLaunch L[2];
    SchedInfo tot;
    int h_err = 0;
    // On an error, launches of earlier chunks may still be running on the
    // stream with images from the pool: the stream is drained before the
    // error returns, so that no later call reuses an image in flight.
    const int rc_loop = [&]() -> int {
        for (int c = 0; c < nch; ++c) {
            const int b = c & 1;
            if (c >= 2) {
                // image b held chunk c - 2: wait until it has run, then reuse it
                GBR_CK(cudaEventSynchronize(ev.e[2 + b]), "sync chunk");
                int rce = read_err(L[b], up, &h_err);
                if (rce) return rce;
            }
            NvtxRange nv_chunk("gbr task graph, order and launch of a chunk");
            std::vector<InstPlan> plans(1);
            plans[0].d = pl.inst;
            plans[0].wins.assign(all.begin() + (long)cuts[c], all.begin() + (long)cuts[c + 1]);
            // the global pipeline order, so that the chunks together make the
            // same program order (and the same result) as one launch
            plans[0].in_pipeline_order = true;
            const int slot = pl.slot[b];
            SchedInfo inf;
            int rc = sched_prepare(
                plans, o, pl.cm, num_sms(),
                [slot](size_t bytes) -> void* {
                    void* p = nullptr;
                    return pool_get(slot, bytes, &p) ? nullptr : p;
                },
                &L[b], &inf, up);
            if (rc) return rc;
            if (pl.mode >= 0) L[b].P.mode = pl.mode;
            tot.tasks += inf.tasks;
            tot.cp_us += inf.cp_us;
            tot.sim_us += inf.sim_us;
            tot.graph_ms += inf.graph_ms;
            tot.order_ms += inf.order_ms;
            if (c == 0 && o.timing) GBR_CK(cudaEventRecord(ev.e[0], st), "event");
            rc = sched_enqueue(L[b], st);
            if (rc) return rc;
            if (nch > 1) GBR_CK(cudaEventRecord(ev.e[2 + b], st), "event");
            *ntasks_out += L[b].P.ntasks;
            if (L[b].P.ntasks > 0) *launches_out += 1;
        }
        return 0;
    }();
    if (rc_loop) {
        (void)cudaStreamSynchronize(st);
        return rc_loop;
    }
    if (o.timing) GBR_CK(cudaEventRecord(ev.e[1], st), "event");
    for (int c = std::max(0, nch - 2); c < nch; ++c) {
        int rce = read_err(L[c & 1], st, &h_err);
        if (rce) return rce;
    }
    if (o.timing) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]) != cudaSuccess) {
            ms = 0.f;
            (void)cudaGetLastError();
        }
        *ms_out += ms;
    }
    if (info) *info = tot;
    if (nch == 1 && L[0].trace_bytes) {
        int rct = store_trace(L[0]);
        if (rct) return rct;
    }
    if (h_err) {
        set_last_error(pl.timeout_msg);
        return GBR_ERR_TIMEOUT;
    }
    return 0;
}

// A pass of a standard form (S, Q).
static int run_persistent(int n, const std::vector<Window>& wins, double* S, int ldS, double* Q,
                          int ldQ, uint8_t* d_sel, DevCounters* d_ctr, const gbr_opts& o,
                          long long* ntasks_out, double* ms_out, long long* launches_out,
                          cudaStream_t st) {
    PassLaunch pl{};
    pl.inst = Inst{S, Q, d_sel, d_ctr, n, ldS, ldQ, 0};
    pl.cm = cost_model(o);
    pl.slot[0] = POOL_SCHED;
    pl.slot[1] = POOL_SCHED_ALT;
    pl.timeout_msg = "persistent scheduler: a task waited longer than wait_limit_ms";
    return run_pass_persistent(wins, pl, o, ntasks_out, ms_out, launches_out, &g_last_sched, st);
}

// ---------------------------------------------------------------------------
// Reorder on device-resident S, Q.
// ---------------------------------------------------------------------------
static int check_opts(const gbr_opts* o) {
    if (o->window < 4 || o->window > WMAX_WIDE) return -10;
    if (o->chain < 1 || o->chain > o->window - 2) return -10;
    if (o->precision != GBR_PREC_DMMA && o->precision != GBR_PREC_OZAKI &&
        o->precision != GBR_PREC_FMA)
        return GBR_ERR_UNSUPPORTED;
    if (o->precision == GBR_PREC_OZAKI &&
        (o->sched != GBR_SCHED_PERSISTENT || (o->slices != 0 && o->slices != OZ_SLICES)))
        return GBR_ERR_UNSUPPORTED;
    if (o->on_reject != GBR_ON_REJECT_CONTINUE && o->on_reject != GBR_ON_REJECT_ABORT)
        return GBR_ERR_UNSUPPORTED;
    if (o->sched != GBR_SCHED_PERSISTENT && o->sched != GBR_SCHED_SEQUENTIAL) return -10;
    if (o->wait_limit_ms < 0) return -10;
    // windows wider than WMAX: the persistent schedule with FP64 updates
    if (o->window > WMAX && (o->sched != GBR_SCHED_PERSISTENT || o->precision == GBR_PREC_OZAKI))
        return GBR_ERR_UNSUPPORTED;
    return 0;
}

// Scratch layout of one reorder call of order n (bytes from a 256-aligned base):
// counters | subdiagonal flags | selection flags | eigenvalues | U.
struct ScratchLayout {
    size_t off_ctr, off_sub, off_sel, off_eig, off_u, total;
};
static constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static constexpr ScratchLayout scratch_layout(size_t n) {
    return ScratchLayout{0,
                         256,
                         256 + align256(n),
                         256 + 2 * align256(n),
                         256 + 2 * align256(n) + align256(2 * n * sizeof(double)),
                         256 + 2 * align256(n) + align256(2 * n * sizeof(double)) +
                             (size_t)WMAX * WMAX * sizeof(double)};
}

static int reorder_device_at(char* b, int n, double* S, int ldS, double* Q, int ldQ,
                             const int* select, double* eig_re, double* eig_im, int* m_out,
                             const gbr_opts& o, gbr_stats* stats, cudaStream_t st);

static int reorder_device(int n, double* S, int ldS, double* Q, int ldQ, const int* select,
                          double* eig_re, double* eig_im, int* m_out, const gbr_opts& o,
                          gbr_stats* stats, cudaStream_t st) {
    void* base = nullptr;
    int rc = pool_get(POOL_SCRATCH, scratch_layout(n).total, &base);
    if (rc) return rc;
    return reorder_device_at((char*)base, n, S, ldS, Q, ldQ, select, eig_re, eig_im, m_out, o,
                             stats, st);
}

static int reorder_device_at(char* b, int n, double* S, int ldS, double* Q, int ldQ,
                             const int* select, double* eig_re, double* eig_im, int* m_out,
                             const gbr_opts& o, gbr_stats* stats, cudaStream_t st) {
    const ScratchLayout L = scratch_layout(n);
    const size_t off_ctr = L.off_ctr, off_sub = L.off_sub, off_sel = L.off_sel,
                 off_eig = L.off_eig, off_u = L.off_u;
    DevCounters* d_ctr = (DevCounters*)(b + off_ctr);
    uint8_t* d_sub = (uint8_t*)(b + off_sub);
    uint8_t* d_sel = (uint8_t*)(b + off_sel);
    double* d_eig = (double*)(b + off_eig);
    double* d_u = (double*)(b + off_u);

    DevCounters h_ctr{0, 0, INT_MAX, 0, 0};
    GBR_CK(cudaMemcpyAsync(d_ctr, &h_ctr, sizeof h_ctr, cudaMemcpyHostToDevice, st), "H2D counters");
    NvtxRange nv_call("gbr_reorder");
    if (o.validate) GBR_CK(launch_validate(n, S, ldS, d_ctr, st), "validate kernel");
    GBR_CK(launch_subdiag(n, S, ldS, d_sub, st), "subdiag kernel");
    std::vector<uint8_t> sub(n), sel(n);
    GBR_CK(cudaMemcpyAsync(sub.data(), d_sub, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
    GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (h_ctr.bad_column != INT_MAX) return -2;

    // selection per position; a 2x2 block is selected if either row is
    const int msel = selection_positions(n, sub.data(), select, sel.data());
    GBR_CK(cudaMemcpyAsync(d_sel, sel.data(), n, cudaMemcpyHostToDevice, st), "H2D selection");

    // optional per-kernel event timing: one event pair per launch, read at the end
    struct Events {
        std::vector<cudaEvent_t> w, u;
        ~Events() {
            for (cudaEvent_t e : w) cudaEventDestroy(e);
            for (cudaEvent_t e : u) cudaEventDestroy(e);
        }
    } evs;
    std::vector<cudaEvent_t>& evw = evs.w;
    std::vector<cudaEvent_t>& evu = evs.u;
    auto mark = [&](std::vector<cudaEvent_t>& v) -> cudaError_t {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        v.push_back(ev);
        return cudaEventRecord(ev, st);
    };
    long long launches = o.validate ? 2 : 1;

    PlanState ps;
    init_state(ps, n, sub.data(), sel.data());
    long long nwin = 0;
    int nchains = 0;
    double flops = 0.0;
    unsigned long long seen_rej = 0;
    double ms_sched = 0.0;
    long long ntasks = 0;
    for (int pass = 0; pass < 1 + 2 * n; ++pass) {
        std::vector<Window> win;
        {
            NvtxRange nv_plan("gbr window plan");
            plan_pass(ps, o.window, o.chain, win, nchains);
        }
        if (win.empty()) break;
        if (o.sched == GBR_SCHED_PERSISTENT) {
            int rcs = run_persistent(n, win, S, ldS, Q, ldQ, d_sel, d_ctr, o, &ntasks, &ms_sched,
                                     &launches, st);
            if (rcs) return rcs;
            flops += update_flops(n, win, Q != nullptr);
        } else
        {
          flops += update_flops(n, win, Q != nullptr);
          for (const Window& wdw : win) {
            if (o.timing) GBR_CK(mark(evw), "event");
            GBR_CK(launch_window(n, wdw, S, ldS, d_sel, d_u, o.strong_test, d_ctr, st,
                                 o.on_reject == GBR_ON_REJECT_ABORT),
                   "window kernel");
            if (o.timing) { GBR_CK(mark(evw), "event"); GBR_CK(mark(evu), "event"); }
            GBR_CK(launch_update(n, wdw, S, ldS, Q, ldQ, d_u, d_ctr, st,
                                 o.precision == GBR_PREC_FMA),
                   "update kernel");
            if (o.timing) GBR_CK(mark(evu), "event");
            launches += 2;
          }
        }
        nwin += (long long)win.size();
        GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        if (h_ctr.rejected == seen_rej) break;  // the simulated plan was exact
        if (o.on_reject == GBR_ON_REJECT_ABORT) break;  // stopped at the first rejection
        seen_rej = h_ctr.rejected;
        // re-plan from the device state: stuck blocks are barriers now
        GBR_CK(launch_subdiag(n, S, ldS, d_sub, st), "subdiag kernel");
        GBR_CK(cudaMemcpyAsync(sub.data(), d_sub, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
        GBR_CK(cudaMemcpyAsync(sel.data(), d_sel, n, cudaMemcpyDeviceToHost, st), "D2H selection");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        init_state(ps, n, sub.data(), sel.data());
        launches += 1;
    }

    if (eig_re || eig_im) {
        GBR_CK(launch_eigs(n, S, ldS, d_eig, d_eig + n, st), "eigenvalue kernel");
        if (eig_re)
            GBR_CK(cudaMemcpyAsync(eig_re, d_eig, n * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "D2H eig_re");
        if (eig_im)
            GBR_CK(cudaMemcpyAsync(eig_im, d_eig + n, n * sizeof(double), cudaMemcpyDeviceToHost, st),
                   "D2H eig_im");
    }
    if (eig_re || eig_im) launches += 1;
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
        set_last_error("window kernel exceeded its step bound");
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
        stats->ms_sched = ms_sched;
        stats->win_flops = (double)h_ctr.win_flops;
        stats->upd_flops_issued = (double)h_ctr.upd_issued;
        stats->tasks = ntasks;
        stats->sched_cp_ms = ntasks ? g_last_sched.cp_us / 1e3 : 0.0;
        stats->sched_sim_ms = ntasks ? g_last_sched.sim_us / 1e3 : 0.0;
        stats->ms_graph = ntasks ? g_last_sched.graph_ms : 0.0;
        stats->ms_order = ntasks ? g_last_sched.order_ms : 0.0;
    }
    long long rej = (long long)h_ctr.rejected;
    return rej > INT_MAX ? INT_MAX : (int)rej;
}

}  // namespace gbr

using namespace gbr;

extern "C" {

void gbr_default_opts(gbr_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->window = 128;
    o->chain = 64;
    o->precision = GBR_PREC_FMA;
    o->slices = 0;
    o->strong_test = 1;
    o->on_reject = GBR_ON_REJECT_CONTINUE;
    o->validate = 1;
    o->timing = 0;
    o->sched = GBR_SCHED_PERSISTENT;
    o->inject = 0;
    o->wait_limit_ms = 0;
}

static int common_args(int n, const void* S, int ldS, const void* Q, int ldQ, const int* select) {
    if (n < 0) return -1;
    if (n > 0 && !S) return -2;
    if (ldS < (n > 1 ? n : 1)) return -3;
    if (Q && ldQ < (n > 1 ? n : 1)) return -5;
    if (n > 0 && !select) return -6;
    return 0;
}

int gbr_reorder(int n, double* S, int ldS, double* Q, int ldQ, const int* select, double* eig_re,
                double* eig_im, int* m_out, const gbr_opts* opts, gbr_stats* stats,
                void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = common_args(n, S, ldS, Q, ldQ, select);
    if (rc) return rc;
    gbr_opts o;
    if (opts) o = *opts; else gbr_default_opts(&o);
    rc = check_opts(&o);
    if (rc) return rc;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) {
        if (m_out) *m_out = 0;
        return 0;
    }
    rc = refuse_capture((cudaStream_t)cuda_stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    rc = reorder_device(n, S, ldS, Q, ldQ, select, eig_re, eig_im, m_out, o, stats,
                        (cudaStream_t)cuda_stream);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gbr_reorder_host(int n, double* S, int ldS, double* Q, int ldQ, const int* select,
                     double* eig_re, double* eig_im, int* m_out, const gbr_opts* opts,
                     gbr_stats* stats, void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = common_args(n, S, ldS, Q, ldQ, select);
    if (rc) return rc;
    gbr_opts o;
    if (opts) o = *opts; else gbr_default_opts(&o);
    rc = check_opts(&o);
    if (rc) return rc;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) {
        if (m_out) *m_out = 0;
        return 0;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    rc = refuse_capture(st);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    size_t mat = (size_t)n * n * sizeof(double);
    void *dS = nullptr, *dQ = nullptr;
    rc = pool_get(POOL_HOST_S, mat, &dS);
    if (rc) return rc;
    if (Q) {
        rc = pool_get(POOL_HOST_Q, mat, &dQ);
        if (rc) return rc;
    }
    NvtxRange nv_host("gbr_reorder_host");
    CopyTimer ct(o.timing != 0 && stats != nullptr);
    ct.mark(0, st);
    GBR_CK(cudaMemcpy2DAsync(dS, n * sizeof(double), S, (size_t)ldS * sizeof(double),
                             n * sizeof(double), n, cudaMemcpyHostToDevice, st), "H2D S");
    if (Q)
        GBR_CK(cudaMemcpy2DAsync(dQ, n * sizeof(double), Q, (size_t)ldQ * sizeof(double),
                                 n * sizeof(double), n, cudaMemcpyHostToDevice, st), "H2D Q");
    ct.mark(1, st);
    rc = reorder_device(n, (double*)dS, n, (double*)dQ, n, select, eig_re, eig_im, m_out, o, stats, st);
    if (rc < 0) return rc;
    ct.mark(2, st);
    GBR_CK(cudaMemcpy2DAsync(S, (size_t)ldS * sizeof(double), dS, n * sizeof(double),
                             n * sizeof(double), n, cudaMemcpyDeviceToHost, st), "D2H S");
    if (Q)
        GBR_CK(cudaMemcpy2DAsync(Q, (size_t)ldQ * sizeof(double), dQ, n * sizeof(double),
                                 n * sizeof(double), n, cudaMemcpyDeviceToHost, st), "D2H Q");
    ct.mark(3, st);
    GBR_CK(cudaStreamSynchronize(st), "sync");
    ct.report(stats);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gbr_plan(int n, const unsigned char* sub, const int* select, int window, int chain,
             int with_q, int* windows, int max_windows, int* chains, double* upd_flops) {
    if (n < 0) return -1;
    if (n > 0 && (!sub || !select)) return -2;
    if (window < 4 || window > WMAX_WIDE) return -4;
    if (chain < 1 || chain > window - 2) return -5;
    std::vector<uint8_t> sb(n), sl(n);
    for (int p = 0; p < n;) {
        int sz = (p + 1 < n && sub[p]) ? 2 : 1;
        uint8_t v = select[p] != 0;
        if (sz == 2) v |= select[p + 1] != 0;
        for (int t = 0; t < sz; ++t) {
            sl[p + t] = v;
            sb[p + t] = (t == 0 && sz == 2) ? 1 : 0;
        }
        p += sz;
    }
    PlanState ps;
    init_state(ps, n, sb.data(), sl.data());
    std::vector<Window> win;
    int nch = 0;
    plan_pass(ps, window, chain, win, nch);
    double fl = 0.0;
    for (size_t i = 0; i < win.size(); ++i) {
        double ww = (double)(win[i].e - win[i].s);
        fl += 2.0 * ww * ww * ((double)(n - win[i].e) + win[i].s + (with_q ? n : 0));
        if (windows && (int)i < max_windows) {
            windows[2 * i] = win[i].s;
            windows[2 * i + 1] = win[i].e;
        }
    }
    if (chains) *chains = nch;
    if (upd_flops) *upd_flops = fl;
    return (int)win.size();
}

// ---------------------------------------------------------------------------
// Reordering without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// reorder: programs whose device memory is all handed out by their own
// arena or allocator, and processes where a cudaMalloc (which may
// synchronize the device) must not happen in the middle of their work.  For
// them this entry point takes its scratch (counters, block flags, selection
// flags, eigenvalue staging and one window accumulator) from a fixed array
// in device global memory that is part of the library image instead of the
// library's pool.  Every GPU that loads the library holds this array
// (GBR_NOALLOC_SCRATCH_BYTES) until the process exits; each process (each
// CUDA context) has its own copy.
// ---------------------------------------------------------------------------
static constexpr size_t kNoallocBytes = scratch_layout(GBR_NOALLOC_MAX_N).total;
static_assert(kNoallocBytes == GBR_NOALLOC_SCRATCH_BYTES, "header and layout disagree");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch in the current context.  In host code
// the symbol is only a host-side stand-in, so the address is looked up with
// the device current, on every call: a cached address would outlive a
// cudaDeviceReset or belong to another context.  The lookup allocates
// nothing once the library's module is loaded.
static int noalloc_scratch(char** out) {
    void* p = nullptr;
    GBR_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
    *out = (char*)p;
    return 0;
}

int gbr_reorder_noalloc(int n, double* S, int ldS, double* Q, int ldQ, const int* select,
                        double* eig_re, double* eig_im, int* m_out, const gbr_opts* opts,
                        gbr_stats* stats, void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = common_args(n, S, ldS, Q, ldQ, select);
    if (rc) return rc;
    if (n > GBR_NOALLOC_MAX_N) return GBR_ERR_NOALLOC_LIMIT;
    gbr_opts o;
    if (opts) o = *opts; else gbr_default_opts(&o);
    rc = check_opts(&o);
    if (rc) return rc;
    o.timing = 0;  // event timing would create events; this path creates nothing
    o.sched = GBR_SCHED_SEQUENTIAL;  // the persistent schedule needs scratch sized per plan
    if (o.precision == GBR_PREC_OZAKI || o.window > WMAX) return GBR_ERR_UNSUPPORTED;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) {
        if (m_out) *m_out = 0;
        return 0;
    }
    rc = refuse_capture((cudaStream_t)cuda_stream);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    char* base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc) return rc;
    rc = reorder_device_at(base, n, S, ldS, Q, ldQ, select, eig_re, eig_im, m_out, o, stats,
                           (cudaStream_t)cuda_stream);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gbr_update_panel(int rows, int w, double* Y, long long rs, long long ks, const double* U,
                     int ldU, int precision, void* cuda_stream) {
    if (rows < 0) return -1;
    if (w < 1 || w > WMAX) return -2;
    if (rows > 0 && !Y) return -3;
    if (rs < 1 || ks < 1 || (rs != 1 && ks != 1)) return -4;
    if (!U) return -6;
    if (ldU < w) return -7;
    if (precision != GBR_PREC_DMMA && precision != GBR_PREC_OZAKI && precision != GBR_PREC_FMA)
        return -8;
    if (rows == 0) return 0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int rcc = refuse_capture(st);
    if (rcc) return rcc;
    std::lock_guard<std::mutex> lock(g_mu);
    // scratch: U contiguous (w x w), then the digit slices, then an error word
    const size_t b_u = align256((size_t)w * w * sizeof(double));
    const size_t b_us = align256(OZ_USLICE_BYTES);
    char* b = nullptr;
    int rc = pool_get(POOL_PANEL, b_u + b_us + 256, (void**)&b);
    if (rc) return rc;
    double* dU = (double*)b;
    unsigned char* dUS = (unsigned char*)(b + b_u);
    int* derr = (int*)(b + b_u + b_us);
    GBR_CK(cudaMemcpy2DAsync(dU, (size_t)w * sizeof(double), U, (size_t)ldU * sizeof(double),
                             (size_t)w * sizeof(double), (size_t)w, cudaMemcpyDeviceToDevice, st),
           "D2D U");
    if (precision != GBR_PREC_OZAKI) {
        GBR_CK(launch_panel_dmma(rows, w, Y, rs, ks, dU, st, precision == GBR_PREC_FMA),
               "panel kernel");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        return 0;
    }
    GBR_CK(cudaMemsetAsync(derr, 0, sizeof(int), st), "memset");
    GBR_CK(launch_panel_ozaki(rows, w, Y, rs, ks, dU, dUS, derr, num_sms(), st), "panel kernel");
    int h_err = 0;
    GBR_CK(cudaMemcpyAsync(&h_err, derr, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H err");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (h_err) {
        set_last_error("gbr_update_panel: a tensor-core tile waited longer than its limit");
        return GBR_ERR_TIMEOUT;
    }
    return 0;
}

int gbr_eigenvectors(int n, const double* S, int ldS, const double* Q, int ldQ,
                     const int* select, double* X, int ldX, int* m_out, int* nscale,
                     gbr_ev_stats* stats, void* cuda_stream) {
    if (stats) memset(stats, 0, sizeof *stats);
    if (n < 0) return -1;
    if (n > 0 && !S) return -2;
    if (ldS < (n > 1 ? n : 1)) return -3;
    if (Q && ldQ < (n > 1 ? n : 1)) return -5;
    if (X && ldX < (n > 1 ? n : 1)) return -8;
    if (m_out) *m_out = 0;
    if (n == 0) return 0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int rcc = refuse_capture(st);
    if (rcc) return rcc;
    std::lock_guard<std::mutex> lock(g_mu);
    // structure: validation and the 2x2 pattern
    char* b = nullptr;
    const size_t b_ctr = 256, b_sub = align256((size_t)n);
    int rc = pool_get(POOL_SCRATCH, b_ctr + b_sub, (void**)&b);
    if (rc) return rc;
    DevCounters* d_ctr = (DevCounters*)b;
    uint8_t* d_sub = (uint8_t*)(b + b_ctr);
    DevCounters h_ctr{0, 0, INT_MAX, 0, 0};
    GBR_CK(cudaMemcpyAsync(d_ctr, &h_ctr, sizeof h_ctr, cudaMemcpyHostToDevice, st), "H2D counters");
    GBR_CK(launch_validate(n, S, ldS, d_ctr, st), "validate kernel");
    GBR_CK(launch_subdiag(n, S, ldS, d_sub, st), "subdiag kernel");
    std::vector<uint8_t> sub(n);
    GBR_CK(cudaMemcpyAsync(sub.data(), d_sub, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
    GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (h_ctr.bad_column != INT_MAX) return -2;
    // selected blocks in diagonal order: output columns; 1x1 blocks first in the launch list
    std::vector<int4> real, cplx;
    std::vector<int> col_top;  // per output column: rows [0, top) may be nonzero
    int m = 0;
    for (int j = 0; j < n;) {
        const int nb = (j + 1 < n && sub[j]) ? 2 : 1;
        const bool on = !select || select[j] != 0 || (nb == 2 && select[j + 1] != 0);
        if (on) {
            (nb == 1 ? real : cplx).push_back(make_int4(j, nb, m, 0));
            for (int t = 0; t < nb; ++t) col_top.push_back(j + nb);
            m += nb;
        }
        j += nb;
    }
    if (m_out) *m_out = m;
    if (!X || m == 0) return 0;  // query of m only
    const int nreal = (int)real.size(), nblk = nreal + (int)cplx.size();
    std::vector<int4> blocks(real);
    blocks.insert(blocks.end(), cplx.begin(), cplx.end());
    const int GN = evgemm_col_block();
    const int ncb = (m + GN - 1) / GN;
    std::vector<int> kmax(ncb);
    for (int cb = 0; cb < ncb; ++cb) kmax[cb] = col_top[std::min(m, (cb + 1) * GN) - 1];
    // scratch: blocks, kmax, column bounds, scalings, Y (when back-transformed),
    // and the right-hand sides of one wave of CTAs when they do not fit shared memory
    const bool rsm = eigvec_rhs_smem(n) != 0;
    const int wave = rsm ? nblk : std::min(nblk, 8 * num_sms());
    const size_t b_blk = align256(sizeof(int4) * nblk), b_km = align256(sizeof(int) * ncb);
    const size_t b_cm = align256(sizeof(double) * 2 * n), b_ns = align256(sizeof(int) * m);
    const size_t b_y = Q ? align256(sizeof(double) * (size_t)n * m) : 0;
    const size_t b_r = rsm ? 0 : align256(sizeof(double) * 3 * (size_t)n * wave);
    char* e = nullptr;
    rc = pool_get(POOL_EIGVEC, b_blk + b_km + b_cm + b_ns + b_y + b_r, (void**)&e);
    if (rc) return rc;
    int4* d_blk = (int4*)e;
    int* d_km = (int*)(e + b_blk);
    double* d_cm = (double*)(e + b_blk + b_km);
    int* d_ns = (int*)(e + b_blk + b_km + b_cm);
    double* d_y = Q ? (double*)(e + b_blk + b_km + b_cm + b_ns) : X;
    const int ldY = Q ? n : ldX;
    double* d_r = rsm ? nullptr : (double*)(e + b_blk + b_km + b_cm + b_ns + b_y);
    GBR_CK(cudaMemcpyAsync(d_blk, blocks.data(), sizeof(int4) * nblk, cudaMemcpyHostToDevice, st), "H2D blocks");
    GBR_CK(cudaMemcpyAsync(d_km, kmax.data(), sizeof(int) * ncb, cudaMemcpyHostToDevice, st), "H2D kmax");
    if (stats) {
        // algorithmic flops: the right-hand-side updates of the back
        // substitution (2 per real multiply-add, twice for a complex vector)
        // and the products of the back-transformation
        std::vector<double> cum(n + 1, 0.0);  // cum[p]: sum of b0 k over blocks ending at or before p
        for (int p = 0; p < n;) {
            const int nb = (p + 1 < n && sub[p]) ? 2 : 1;
            cum[p + nb] = cum[p] + (double)p * nb;
            if (nb == 2) cum[p + 1] = cum[p];
            p += nb;
        }
        double fs = 0.0;
        for (const int4& bk : blocks) fs += 2.0 * (bk.y == 2 ? 2.0 : 1.0) * cum[bk.x];
        stats->solve_flops = fs;
        double fg = 0.0;
        if (Q)
            for (int cb = 0; cb < ncb; ++cb)
                fg += 2.0 * n * kmax[cb] * (double)(std::min(m, (cb + 1) * GN) - cb * GN);
        stats->backtransform_flops = fg;
    }
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (stats)
        for (int i = 0; i < 4; ++i) {
            GBR_CK(cudaEventCreate(&ev[i]), "event");
        }
    if (stats) GBR_CK(cudaEventRecord(ev[0], st), "event");
    GBR_CK(launch_colmax(n, S, ldS, d_cm, d_cm + n, st), "column bounds kernel");
    // back substitution, in waves when the right-hand sides live in global memory
    for (int b0 = 0; b0 < nblk; b0 += wave) {
        const int cnt = std::min(wave, nblk - b0);
        const int nr = std::max(0, std::min(nreal - b0, cnt));
        GBR_CK(launch_eigvec(n, S, ldS, d_blk + b0, cnt, nr, d_y, ldY, d_cm, d_cm + n, d_r, d_ns, st),
               "eigenvector kernel");
    }
    if (stats) GBR_CK(cudaEventRecord(ev[1], st), "event");
    if (Q) GBR_CK(launch_evgemm(n, m, Q, ldQ, d_y, ldY, X, ldX, d_km, st), "back-transform kernel");
    if (stats) GBR_CK(cudaEventRecord(ev[2], st), "event");
    GBR_CK(launch_evnorm(n, d_blk, nblk, X, ldX, st), "normalization kernel");
    if (stats) GBR_CK(cudaEventRecord(ev[3], st), "event");
    if (nscale)
        GBR_CK(cudaMemcpyAsync(nscale, d_ns, sizeof(int) * m, cudaMemcpyDeviceToHost, st), "D2H scalings");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (stats) {
        float a = 0.f, b2 = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b2, ev[1], ev[2]);
        cudaEventElapsedTime(&c, ev[2], ev[3]);
        stats->ms_solve = a;
        stats->ms_backtransform = b2;
        stats->ms_normalize = c;
        for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    }
    return 0;
}

int gbr_last_trace(long long* out, int max_tasks) {
    std::lock_guard<std::mutex> lock(g_mu);
    const int nt = (int)(g_trace.size() / 8);
    if (out) {
        const int k = std::min(nt, std::max(0, max_tasks));
        memcpy(out, g_trace.data(), sizeof(long long) * 8 * (size_t)k);
    }
    return nt;
}

const char* gbr_status_string(int s) {
    if (s == 0) return "success";
    if (s > 0) return "partial reorder: some block swaps were rejected by the stability test";
    switch (s) {
        case -1: return "invalid argument 1: n < 0";
        case -2: return "invalid argument 2: S is NULL or not in standard real Schur form";
        case -3: return "invalid argument 3: ldS < max(1, n)";
        case -5: return "invalid argument 5: ldQ < max(1, n)";
        case -6: return "invalid argument 6: select is NULL";
        case -10: return "invalid argument 10: window must be 4..256 and chain 1..window-2";
        case GBR_ERR_CUDA: return "CUDA error (see gbr_last_error)";
        case GBR_ERR_NOMEM: return "out of device memory";
        case GBR_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case GBR_ERR_UNSUPPORTED: return "unsupported option value";
        case GBR_ERR_NOALLOC_LIMIT:
            return "n exceeds GBR_NOALLOC_MAX_N, the size the no-allocation entry point supports";
        case GBR_ERR_PLAN_MISMATCH:
            return "the block structure of an S differs from the one its batch was planned for";
        case GBR_ERR_CAPTURING:
            return "the stream is being captured into a CUDA graph; the call synchronizes it";
        default: return "invalid argument";
    }
}

const char* gbr_last_error(void) { return last_error_cstr(); }

long long gbr_pool_bytes(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    long long b = 0;
    for (int s = 0; s < POOL_NSLOTS; ++s) b += (long long)g_pool[dev].bytes[s];
    return b;
}

void gbr_release(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    for (int s = 0; s < POOL_NSLOTS; ++s) {
        if (g_pool[dev].ptr[s]) cudaFree(g_pool[dev].ptr[s]);
        g_pool[dev].ptr[s] = nullptr;
        g_pool[dev].bytes[s] = 0;
    }
    if (g_side[dev]) {
        cudaStreamDestroy(g_side[dev]);
        g_side[dev] = nullptr;
    }
}

int gbr_version(void) { return 100; }

}  // extern "C"
