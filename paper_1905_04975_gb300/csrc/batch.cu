// Batched reordering: many independent problems in one persistent-scheduler
// launch, replayed from a CUDA graph, with window, chain and update-tile
// sizes chosen per instance by an autotuner.
//
// Every instance is the reordering of Eq. 7 with the windows, chains and
// update tasks of Section 3.2; the batch only merges their task graphs (no
// edges between instances) and orders the union for the device's SMs, so
// small problems fill the GPU together instead of one after another.
#include "host.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <random>
#include <string>

struct gbr_batch {
    int count = 0;
    int dev = 0;
    gbr_opts o{};
    std::vector<int> n, ldS, ldQ, valid, msel;
    std::vector<double*> S, Q;
    std::vector<long long> off;
    long long ntot = 0;
    // device: inst | ctr | ctr_init | off | sub_init | sel_init | sel | wr | wi
    void* dmem = nullptr;
    void* smem = nullptr;  // scheduler image
    gbr::Inst* d_inst = nullptr;
    gbr::DevCounters* d_ctr = nullptr;
    gbr::DevCounters* d_ctr0 = nullptr;
    long long* d_off = nullptr;
    uint8_t* d_sub0 = nullptr;
    uint8_t* d_sel0 = nullptr;
    uint8_t* d_sel = nullptr;
    double* d_wr = nullptr;
    double* d_wi = nullptr;
    // pinned host staging: ctr | err | wr | wi
    void* hmem = nullptr;
    gbr::DevCounters* h_ctr = nullptr;
    int* h_err = nullptr;
    double* h_wr = nullptr;
    double* h_wi = nullptr;
    gbr::SchedLaunch L;
    gbr::SchedInfo info;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double upd_flops = 0.0;
    long long windows = 0, chains = 0;
};

namespace gbr {

// ---------------------------------------------------------------------------
// Autotuner table: size class -> (window, chain, far tile rows), per device.
// Class c holds n in (2^(c-1), 2^c]; n <= 16 shares the class of 32.
// ---------------------------------------------------------------------------
struct TuneChoice {
    int w, m, far;
};
static std::mutex g_tmu;
static std::map<int, TuneChoice> g_tune[64];

static int size_class(int n) {
    int c = 5;
    while ((1 << c) < n) ++c;
    return c;
}

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return dev;
}

static TuneChoice tune_lookup(int n, bool* tuned) {
    std::lock_guard<std::mutex> lk(g_tmu);
    auto& t = g_tune[current_device()];
    auto it = t.find(size_class(n));
    if (it != t.end()) {
        if (tuned) *tuned = true;
        return it->second;
    }
    if (tuned) *tuned = false;
    return TuneChoice{WMAX, WMAX / 2, 0};
}

static CostModel batch_cost_model(const gbr_opts& o) {
    CostModel c;
    c.tile_rate = (o.precision == GBR_PREC_OZAKI) ? 100000.0
                : (o.precision == GBR_PREC_FMA)  ? 7600.0
                                                 : 6900.0;
    return c;
}

static int check_batch_opts(const gbr_opts& o) {
    const bool auto_w = (o.window == GBR_AUTO);
    if (!auto_w && (o.window < 4 || o.window > WMAX)) return -8;
    if (o.chain != GBR_AUTO && (o.chain < 1 || (!auto_w && o.chain > o.window - 2))) return -8;
    if (o.precision != GBR_PREC_DMMA && o.precision != GBR_PREC_OZAKI &&
        o.precision != GBR_PREC_FMA)
        return GBR_ERR_UNSUPPORTED;
    if (o.precision == GBR_PREC_OZAKI && o.slices != 0 && o.slices != OZ_SLICES)
        return GBR_ERR_UNSUPPORTED;
    if (o.sched != GBR_SCHED_PERSISTENT) return GBR_ERR_UNSUPPORTED;
    if (o.on_reject != GBR_ON_REJECT_CONTINUE) return GBR_ERR_UNSUPPORTED;
    if (o.wait_limit_ms < 0) return -8;
    return 0;
}

// Window, chain and far tile rows for one instance under the options.
static TuneChoice choose(const gbr_opts& o, int n, int far_override) {
    TuneChoice c = tune_lookup(n, nullptr);
    if (o.window != GBR_AUTO) {
        c.w = o.window;
        c.m = (o.chain != GBR_AUTO) ? o.chain : std::max(1, o.window / 2);
        c.far = 0;
    } else if (o.chain != GBR_AUTO) {
        c.m = std::min(o.chain, c.w - 2);
    }
    if (far_override) c.far = far_override;
    return c;
}

static void free_batch(gbr_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->dmem) cudaFree(b->dmem);
    if (b->smem) cudaFree(b->smem);
    if (b->hmem) cudaFreeHost(b->hmem);
    delete b;
}

static int batch_args(int count, const int* n, double* const* S, const int* ldS,
                      double* const* Q, const int* ldQ, const int* select) {
    if (count < 0) return -1;
    if (count == 0) return 0;
    if (!n) return -2;
    if (!S) return -3;
    if (!ldS) return -4;
    if (Q && !ldQ) return -6;
    long long tot = 0;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 0) return -2;
        if (n[i] > 0 && !S[i]) return -3;
        if (ldS[i] < std::max(1, n[i])) return -4;
        if (Q && Q[i] && ldQ[i] < std::max(1, n[i])) return -6;
        tot += n[i];
    }
    if (tot > 0 && !select) return -7;
    return 0;
}

// Plans the batch and captures its graph.  far_override (autotuner only)
// forces the far tile rows of every instance.
static int batch_create(int count, const int* n, double* const* S, const int* ldS,
                        double* const* Q, const int* ldQ, const int* select, const gbr_opts& o,
                        int far_override, int* status, gbr_batch** out, cudaStream_t st) {
    gbr_batch* b = new (std::nothrow) gbr_batch;
    if (!b) return GBR_ERR_NOMEM;
    struct Guard {
        gbr_batch*& p;
        ~Guard() { free_batch(p); }
    } guard{b};
    b->count = count;
    b->dev = current_device();
    b->o = o;
    b->n.assign(n, n + count);
    b->ldS.assign(ldS, ldS + count);
    b->S.assign(S, S + count);
    b->Q.assign(count, nullptr);
    b->ldQ.assign(count, 1);
    if (Q)
        for (int i = 0; i < count; ++i) {
            b->Q[i] = Q[i];
            b->ldQ[i] = Q[i] ? ldQ[i] : 1;
        }
    b->off.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) b->off[i + 1] = b->off[i] + n[i];
    b->ntot = b->off[count];
    const long long ntot = b->ntot;
    const int cnt1 = std::max(1, count);

    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_inst = al(sizeof(Inst) * cnt1), b_ctr = al(sizeof(DevCounters) * cnt1);
    const size_t b_off = al(sizeof(long long) * (count + 1)), b_pos = al((size_t)std::max(1LL, ntot));
    const size_t b_eig = al(sizeof(double) * std::max(1LL, ntot));
    GBR_CK(cudaMalloc(&b->dmem, b_inst + 2 * b_ctr + b_off + 3 * b_pos + 2 * b_eig), "cudaMalloc(batch)");
    char* p = (char*)b->dmem;
    b->d_inst = (Inst*)p; p += b_inst;
    b->d_ctr = (DevCounters*)p; p += b_ctr;
    b->d_ctr0 = (DevCounters*)p; p += b_ctr;
    b->d_off = (long long*)p; p += b_off;
    b->d_sub0 = (uint8_t*)p; p += b_pos;
    b->d_sel0 = (uint8_t*)p; p += b_pos;
    b->d_sel = (uint8_t*)p; p += b_pos;
    b->d_wr = (double*)p; p += b_eig;
    b->d_wi = (double*)p;
    const size_t h_ctr = al(sizeof(DevCounters) * cnt1);
    GBR_CK(cudaMallocHost(&b->hmem, h_ctr + 256 + 2 * b_eig), "cudaMallocHost(batch)");
    char* h = (char*)b->hmem;
    b->h_ctr = (DevCounters*)h; h += h_ctr;
    b->h_err = (int*)h; h += 256;
    b->h_wr = (double*)h; h += b_eig;
    b->h_wi = (double*)h;

    // instance table, counters, validation and block structure
    std::vector<Inst> itab(count);
    for (int i = 0; i < count; ++i)
        itab[i] = Inst{b->S[i], b->Q[i], b->d_sel + b->off[i], b->d_ctr + i, b->n[i], b->ldS[i], b->ldQ[i], 0};
    std::vector<DevCounters> c0(count, DevCounters{0, 0, INT_MAX, 0, 0});
    if (count) {
        GBR_CK(cudaMemcpyAsync(b->d_inst, itab.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, st), "H2D instances");
        GBR_CK(cudaMemcpyAsync(b->d_ctr, c0.data(), sizeof(DevCounters) * count, cudaMemcpyHostToDevice, st), "H2D counters");
        GBR_CK(cudaMemcpyAsync(b->d_ctr0, c0.data(), sizeof(DevCounters) * count, cudaMemcpyHostToDevice, st), "H2D counters");
        GBR_CK(cudaMemcpyAsync(b->d_off, b->off.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, st), "H2D offsets");
        if (o.validate) GBR_CK(launch_validate_batched(count, b->d_inst, st), "validate kernel");
        GBR_CK(launch_subdiag_batched(count, b->d_inst, b->d_off, b->d_sub0, nullptr, st), "subdiag kernel");
    }
    std::vector<uint8_t> sub((size_t)std::max(1LL, ntot)), sel((size_t)std::max(1LL, ntot), 0);
    std::vector<DevCounters> hc(cnt1);
    if (ntot) GBR_CK(cudaMemcpyAsync(sub.data(), b->d_sub0, ntot, cudaMemcpyDeviceToHost, st), "D2H subdiag");
    if (count) GBR_CK(cudaMemcpyAsync(hc.data(), b->d_ctr, sizeof(DevCounters) * count, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    b->valid.assign(count, 1);
    b->msel.assign(count, 0);
    bool any_invalid = false;
    for (int i = 0; i < count; ++i) {
        if (hc[i].bad_column != INT_MAX) {
            b->valid[i] = 0;
            itab[i].n = 0;  // left out of every batched kernel
            any_invalid = true;
        }
        if (status) status[i] = b->valid[i] ? 0 : -2;
        if (!b->valid[i] || b->n[i] == 0) continue;
        b->msel[i] = selection_positions(b->n[i], sub.data() + b->off[i], select + b->off[i],
                                         sel.data() + b->off[i]);
    }
    if (any_invalid)
        GBR_CK(cudaMemcpyAsync(b->d_inst, itab.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, st), "H2D instances");
    if (ntot) {
        GBR_CK(cudaMemcpyAsync(b->d_sel0, sel.data(), ntot, cudaMemcpyHostToDevice, st), "H2D selection");
        GBR_CK(cudaMemcpyAsync(b->d_sel, sel.data(), ntot, cudaMemcpyHostToDevice, st), "H2D selection");
    }

    // windows per instance, then one task graph over all of them
    std::vector<InstPlan> plans;
    plans.reserve(count);
    for (int i = 0; i < count; ++i) {
        if (!b->valid[i] || b->n[i] == 0) continue;
        const TuneChoice tc = choose(o, b->n[i], far_override);
        PlanState ps;
        init_state(ps, b->n[i], sub.data() + b->off[i], sel.data() + b->off[i]);
        InstPlan ip;
        ip.d = itab[i];
        int nch = 0;
        plan_pass(ps, tc.w, std::min(tc.m, tc.w - 2), ip.wins, nch);
        if (ip.wins.empty()) continue;
        ip.far = tc.far;
        b->chains += nch;
        b->windows += (long long)ip.wins.size();
        b->upd_flops += update_flops(b->n[i], ip.wins, b->Q[i] != nullptr);
        plans.push_back(std::move(ip));
    }
    int rc = sched_prepare(
        plans, o, batch_cost_model(o), num_sms(),
        [b](size_t bytes) -> void* {
            void* q = nullptr;
            if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
            b->smem = q;
            return q;
        },
        &b->L, &b->info, st);
    if (rc) return rc;
    GBR_CK(cudaMemcpyAsync(b->d_ctr0, b->d_ctr, sizeof(DevCounters) * cnt1, cudaMemcpyDeviceToDevice, st), "counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");

    // capture: restore selection and counters, check the structure, run the
    // scheduler, read eigenvalues, counters and the error word back
    GBR_CK(sched_configure(), "scheduler attributes");
    GBR_CK(cudaEventCreate(&b->e0), "event");
    GBR_CK(cudaEventCreate(&b->e1), "event");
    cudaStream_t cs = nullptr;
    GBR_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } sg{cs};
    GBR_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    auto body = [&]() -> int {
        if (ntot) GBR_CK(cudaMemcpyAsync(b->d_sel, b->d_sel0, ntot, cudaMemcpyDeviceToDevice, cs), "restore selection");
        if (count) GBR_CK(cudaMemcpyAsync(b->d_ctr, b->d_ctr0, sizeof(DevCounters) * count, cudaMemcpyDeviceToDevice, cs), "reset counters");
        int r = sched_enqueue(b->L, cs, [&](cudaStream_t s) -> int {
            if (count) GBR_CK(launch_subdiag_batched(count, b->d_inst, b->d_off, b->d_sub0, b->L.P.err, s), "structure check");
            // an external event node: a plain record inside a capture only orders streams
            GBR_CK(cudaEventRecordWithFlags(b->e0, s, cudaEventRecordExternal), "event");
            return 0;
        });
        if (r) return r;
        GBR_CK(cudaEventRecordWithFlags(b->e1, cs, cudaEventRecordExternal), "event");
        if (count) GBR_CK(launch_eigs_batched(count, b->d_inst, b->d_off, b->d_wr, b->d_wi, cs), "eigenvalue kernel");
        if (count) GBR_CK(cudaMemcpyAsync(b->h_ctr, b->d_ctr, sizeof(DevCounters) * count, cudaMemcpyDeviceToHost, cs), "D2H counters");
        GBR_CK(cudaMemcpyAsync(b->h_err, b->L.P.err, sizeof(int), cudaMemcpyDeviceToHost, cs), "D2H err");
        if (ntot) {
            GBR_CK(cudaMemcpyAsync(b->h_wr, b->d_wr, sizeof(double) * ntot, cudaMemcpyDeviceToHost, cs), "D2H eig_re");
            GBR_CK(cudaMemcpyAsync(b->h_wi, b->d_wi, sizeof(double) * ntot, cudaMemcpyDeviceToHost, cs), "D2H eig_im");
        }
        return 0;
    };
    int rb = body();
    cudaGraph_t g = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (rb) {
        if (g) cudaGraphDestroy(g);
        return rb;
    }
    GBR_CK(ec, "end capture");
    b->graph = g;
    GBR_CK(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
    *out = b;
    b = nullptr;  // ownership to the caller
    return 0;
}

// Further passes for instances whose swaps were rejected (the graph's plan
// assumed none): re-plan each from its device state, where stuck blocks are
// barriers, and run them together until no new rejection appears.
static int batch_fixup(gbr_batch* b, std::vector<unsigned long long>& seen, long long* tasks,
                       double* flops, long long* wins, cudaStream_t st) {
    std::vector<int> todo;
    for (int i = 0; i < b->count; ++i)
        if (b->valid[i] && b->h_ctr[i].rejected > seen[i]) todo.push_back(i);
    void* tmp = nullptr;
    struct Free {
        void*& p;
        ~Free() { if (p) cudaFree(p); }
    } fr{tmp};
    for (int pass = 0; !todo.empty() && pass < 64; ++pass) {
        std::vector<InstPlan> plans;
        for (int i : todo) {
            seen[i] = b->h_ctr[i].rejected;
            const int n = b->n[i];
            std::vector<uint8_t> sub(n), sel(n);
            uint8_t* d_tmp = nullptr;
            GBR_CK(cudaMallocAsync((void**)&d_tmp, n, st), "cudaMallocAsync");
            GBR_CK(launch_subdiag(n, b->S[i], b->ldS[i], d_tmp, st), "subdiag kernel");
            GBR_CK(cudaMemcpyAsync(sub.data(), d_tmp, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
            GBR_CK(cudaMemcpyAsync(sel.data(), b->d_sel + b->off[i], n, cudaMemcpyDeviceToHost, st), "D2H selection");
            GBR_CK(cudaFreeAsync(d_tmp, st), "cudaFreeAsync");
            GBR_CK(cudaStreamSynchronize(st), "sync");
            const TuneChoice tc = choose(b->o, n, 0);
            PlanState ps;
            init_state(ps, n, sub.data(), sel.data());
            InstPlan ip;
            ip.d = Inst{b->S[i], b->Q[i], b->d_sel + b->off[i], b->d_ctr + i, n, b->ldS[i], b->ldQ[i], 0};
            int nch = 0;
            plan_pass(ps, tc.w, std::min(tc.m, tc.w - 2), ip.wins, nch);
            if (ip.wins.empty()) continue;
            *flops += update_flops(n, ip.wins, b->Q[i] != nullptr);
            *wins += (long long)ip.wins.size();
            plans.push_back(std::move(ip));
        }
        if (plans.empty()) break;
        SchedLaunch L;
        SchedInfo inf;
        if (tmp) { cudaFree(tmp); tmp = nullptr; }
        int rc = sched_prepare(
            plans, b->o, batch_cost_model(b->o), num_sms(),
            [&tmp](size_t bytes) -> void* {
                return cudaMalloc(&tmp, bytes) == cudaSuccess ? tmp : nullptr;
            },
            &L, &inf, st);
        if (rc) return rc;
        *tasks += inf.tasks;
        rc = sched_enqueue(L, st);
        if (rc) return rc;
        int err = 0;
        GBR_CK(cudaMemcpyAsync(&err, L.P.err, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H err");
        GBR_CK(cudaMemcpyAsync(b->h_ctr, b->d_ctr, sizeof(DevCounters) * b->count, cudaMemcpyDeviceToHost, st), "D2H counters");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        if (err) {
            set_last_error("persistent scheduler: a task waited longer than wait_limit_ms");
            return GBR_ERR_TIMEOUT;
        }
        std::vector<int> next;
        for (int i : todo)
            if (b->h_ctr[i].rejected > seen[i]) next.push_back(i);
        todo.swap(next);
    }
    if (b->ntot) {
        GBR_CK(launch_eigs_batched(b->count, b->d_inst, b->d_off, b->d_wr, b->d_wi, st), "eigenvalue kernel");
        GBR_CK(cudaMemcpyAsync(b->h_wr, b->d_wr, sizeof(double) * b->ntot, cudaMemcpyDeviceToHost, st), "D2H eig_re");
        GBR_CK(cudaMemcpyAsync(b->h_wi, b->d_wi, sizeof(double) * b->ntot, cudaMemcpyDeviceToHost, st), "D2H eig_im");
        GBR_CK(cudaStreamSynchronize(st), "sync");
    }
    return 0;
}

static int batch_run(gbr_batch* b, double* eig_re, double* eig_im, int* m_out, int* status,
                     gbr_stats* stats, cudaStream_t st) {
    auto t0 = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof *stats);
    if (current_device() != b->dev) {
        set_last_error("gbr_batch_run: the current device is not the batch's device");
        return GBR_ERR_CUDA;
    }
    GBR_CK(cudaGraphLaunch(b->exec, st), "graph launch");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (*b->h_err == 2) {
        set_last_error("gbr_batch_run: block structure differs from the planned one");
        return GBR_ERR_PLAN_MISMATCH;
    }
    if (*b->h_err) {
        set_last_error("persistent scheduler: a task waited longer than wait_limit_ms");
        return GBR_ERR_TIMEOUT;
    }
    if (b->L.trace_bytes) {
        // opts.timing = 2: the graph's scheduler launch recorded its timeline
        int rct = store_trace(b->L);
        if (rct) return rct;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->e0, b->e1) != cudaSuccess) {
        ms = 0.f;
        (void)cudaGetLastError();  // not a failure of the run; leave no stale error
    }
    long long tasks = b->L.P.ntasks, wins = b->windows;
    double flops = b->upd_flops;
    std::vector<unsigned long long> seen(b->count, 0);
    bool rej = false;
    for (int i = 0; i < b->count; ++i) rej |= b->h_ctr[i].rejected > 0;
    if (rej) {
        int rc = batch_fixup(b, seen, &tasks, &flops, &wins, st);
        if (rc) return rc;
    }
    int with_rej = 0;
    long long swaps = 0, rejected = 0;
    double wfl = 0.0, iss = 0.0;
    for (int i = 0; i < b->count; ++i) {
        const DevCounters& c = b->h_ctr[i];
        if (c.step_overflow) {
            set_last_error("window kernel exceeded its step bound");
            return GBR_ERR_CUDA;
        }
        const long long r = b->valid[i] ? (long long)c.rejected : 0;
        if (status) status[i] = b->valid[i] ? (int)std::min<long long>(r, INT_MAX) : -2;
        if (m_out) m_out[i] = b->msel[i];
        with_rej += r > 0;
        swaps += b->valid[i] ? (long long)c.swaps : 0;
        rejected += r;
        wfl += b->valid[i] ? (double)c.win_flops : 0.0;
        iss += b->valid[i] ? (double)c.upd_issued : 0.0;
    }
    if (b->ntot) {
        if (eig_re) memcpy(eig_re, b->h_wr, sizeof(double) * b->ntot);
        if (eig_im) memcpy(eig_im, b->h_wi, sizeof(double) * b->ntot);
    }
    if (stats) {
        stats->swaps = swaps;
        stats->rejected = rejected;
        stats->windows = wins;
        stats->chains = b->chains;
        stats->launches = 5 + (rej ? 1 : 0);
        stats->upd_flops = flops;
        stats->ms_sched = ms;
        stats->win_flops = wfl;
        stats->upd_flops_issued = iss;
        stats->tasks = tasks;
        stats->sched_cp_ms = b->info.cp_us / 1e3;
        stats->sched_sim_ms = b->info.sim_us / 1e3;
        stats->ms_graph = b->info.graph_ms;
        stats->ms_order = b->info.order_ms;
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return with_rej;
}

// ---------------------------------------------------------------------------
// Autotuner: synthetic standard Schur forms (seeded, as the test inputs:
// 60% of positions in 1x1 blocks N(0,1), the rest in standardized 2x2 blocks
// [[a, b], [c, a]] with a ~ N(0,1), |b|, |c| ~ U(0.1, 2), bc < 0; strict upper
// part N(0,1)), Q = I, 20-60% of the eigenvalues selected.
// ---------------------------------------------------------------------------
static void synth_schur(int n, std::mt19937_64& rng, double* S, int* sel) {
    std::normal_distribution<double> nd;
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) S[(size_t)j * n + i] = (i < j) ? nd(rng) : 0.0;
    const double frac = 0.2 + 0.4 * u01(rng);
    for (int p = 0; p < n;) {
        const bool two = (p + 1 < n) && u01(rng) < 0.25;  // about 40% of positions
        if (two) {
            const double a = nd(rng);
            double bb = 0.1 + 1.9 * u01(rng), c = 0.1 + 1.9 * u01(rng);
            if (u01(rng) < 0.5) bb = -bb; else c = -c;
            S[(size_t)p * n + p] = a;
            S[(size_t)(p + 1) * n + p + 1] = a;
            S[(size_t)(p + 1) * n + p] = bb;
            S[(size_t)p * n + p + 1] = c;
            const int v = u01(rng) < frac;
            sel[p] = sel[p + 1] = v;
            p += 2;
        } else {
            S[(size_t)p * n + p] = nd(rng);
            sel[p] = u01(rng) < frac;
            p += 1;
        }
    }
}

static int autotune(int n_max, int per_class, cudaStream_t st) {
    if (n_max < 1) return -1;
    if (per_class < 1) return -2;
    const int rcc = refuse_capture(st);
    if (rcc) return rcc;
    const int dev = current_device();
    int tuned = 0;
    for (int cls = 5; (1 << (cls - 1)) < n_max; ++cls) {
        const int hi = std::min(1 << cls, std::max(n_max, 1 << (cls - 1)));
        const int lo = std::max(1, (1 << (cls - 1)) + 1);
        std::mt19937_64 rng(0x5eed0000ull + cls);
        std::uniform_int_distribution<int> un(std::min(lo, hi), hi);
        std::vector<int> ns(per_class), lds(per_class);
        size_t elems = 0;
        for (int i = 0; i < per_class; ++i) {
            ns[i] = un(rng);
            lds[i] = ns[i];
            elems += (size_t)ns[i] * ns[i];
        }
        std::vector<double> hS(elems), hQ(elems, 0.0);
        std::vector<int> sel;
        size_t o2 = 0;
        for (int i = 0; i < per_class; ++i) {
            std::vector<int> si(ns[i]);
            synth_schur(ns[i], rng, hS.data() + o2, si.data());
            for (int k = 0; k < ns[i]; ++k) hQ[o2 + (size_t)k * ns[i] + k] = 1.0;
            sel.insert(sel.end(), si.begin(), si.end());
            o2 += (size_t)ns[i] * ns[i];
        }
        double* d = nullptr;  // S | Q | pristine S | pristine Q
        GBR_CK(cudaMalloc(&d, 4 * elems * sizeof(double)), "cudaMalloc(autotune)");
        struct Free {
            double* p;
            ~Free() { cudaFree(p); }
        } fr{d};
        GBR_CK(cudaMemcpy(d + 2 * elems, hS.data(), elems * 8, cudaMemcpyHostToDevice), "H2D");
        GBR_CK(cudaMemcpy(d + 3 * elems, hQ.data(), elems * 8, cudaMemcpyHostToDevice), "H2D");
        std::vector<double*> Sp(per_class), Qp(per_class);
        o2 = 0;
        for (int i = 0; i < per_class; ++i) {
            Sp[i] = d + o2;
            Qp[i] = d + elems + o2;
            o2 += (size_t)ns[i] * ns[i];
        }
        TuneChoice best{WMAX, WMAX / 2, 0};
        float best_ms = 1e30f;
        for (int w : {32, 64, 96, 128}) {
            if (w > std::max(32, hi)) continue;
            for (int mq = 1; mq <= 3; ++mq) {
                const int m = std::max(1, std::min(w - 2, w * mq / 4));
                for (int far : {UPD_BM, UPD_FAR}) {
                    gbr_opts o;
                    gbr_default_opts(&o);
                    o.window = w;
                    o.chain = m;
                    o.validate = 0;
                    gbr_batch* b = nullptr;
                    // plan on the pristine forms (the previous candidate reordered them)
                    GBR_CK(cudaMemcpyAsync(d, d + 2 * elems, 2 * elems * 8, cudaMemcpyDeviceToDevice, st), "restore");
                    int rc = batch_create(per_class, ns.data(), Sp.data(), lds.data(), Qp.data(),
                                          lds.data(), sel.data(), o, far, nullptr, &b, st);
                    if (rc) return rc;
                    float tms = 1e30f;
                    for (int rep = 0; rep < 2 && rc >= 0; ++rep) {
                        GBR_CK(cudaMemcpyAsync(d, d + 2 * elems, 2 * elems * 8, cudaMemcpyDeviceToDevice, st), "restore");
                        gbr_stats s;
                        rc = batch_run(b, nullptr, nullptr, nullptr, nullptr, &s, st);
                        if (rc >= 0 && rep > 0) tms = (float)s.ms_sched;
                    }
                    free_batch(b);
                    if (rc < 0) return rc;
                    if (tms < best_ms) {
                        best_ms = tms;
                        best = TuneChoice{w, m, far};
                    }
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(g_tmu);
            g_tune[dev][cls] = best;
        }
        ++tuned;
    }
    return tuned;
}

}  // namespace gbr

using namespace gbr;

extern "C" {

int gbr_batch_create(int count, const int* n, double* const* S, const int* ldS, double* const* Q,
                     const int* ldQ, const int* select, const gbr_opts* opts, int* status,
                     gbr_batch** out, void* cuda_stream) {
    if (!out) return -10;
    *out = nullptr;
    int rc = batch_args(count, n, S, ldS, Q, ldQ, select);
    if (rc) return rc;
    gbr_opts o;
    if (opts) o = *opts; else gbr_default_opts(&o);
    rc = check_batch_opts(o);
    if (rc) return rc;
    o.timing = o.timing >= 2 ? 2 : (o.timing ? 1 : 0);  // 2: per-task timeline of each run
    rc = refuse_capture((cudaStream_t)cuda_stream);
    if (rc) return rc;
    return batch_create(count, n, S, ldS, Q, ldQ, select, o, 0, status, out,
                        (cudaStream_t)cuda_stream);
}

int gbr_batch_run(gbr_batch* batch, double* eig_re, double* eig_im, int* m_out, int* status,
                  gbr_stats* stats, void* cuda_stream) {
    if (!batch) return -1;
    const int rc = refuse_capture((cudaStream_t)cuda_stream);
    if (rc) return rc;
    return batch_run(batch, eig_re, eig_im, m_out, status, stats, (cudaStream_t)cuda_stream);
}

void gbr_batch_destroy(gbr_batch* batch) { free_batch(batch); }

int gbr_reorder_batched(int count, const int* n, double* const* S, const int* ldS,
                        double* const* Q, const int* ldQ, const int* select, double* eig_re,
                        double* eig_im, int* m_out, int* status, const gbr_opts* opts,
                        gbr_stats* stats, void* cuda_stream) {
    auto t0 = std::chrono::steady_clock::now();
    gbr_batch* b = nullptr;
    int rc = gbr_batch_create(count, n, S, ldS, Q, ldQ, select, opts, status, &b, cuda_stream);
    if (rc) return rc;
    rc = batch_run(b, eig_re, eig_im, m_out, status, stats, (cudaStream_t)cuda_stream);
    free_batch(b);
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gbr_autotune(int n_max, int per_class, void* cuda_stream) {
    return autotune(n_max, per_class, (cudaStream_t)cuda_stream);
}

int gbr_tune_get(int n, int* window, int* chain, int* tile) {
    bool tuned = false;
    const TuneChoice c = tune_lookup(std::max(1, n), &tuned);
    if (window) *window = c.w;
    if (chain) *chain = c.m;
    if (tile) *tile = c.far ? c.far : far_rows(std::max(1, n));
    return tuned ? 1 : 0;
}

int gbr_tune_save(const char* path) {
    if (!path) return -1;
    std::map<int, TuneChoice> t;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        t = g_tune[current_device()];
    }
    FILE* f = fopen(path, "w");
    if (!f) return -2;
    int k = 0;
    fprintf(f, "{\"tune\": [");
    for (const auto& kv : t) {
        fprintf(f, "%s\n  {\"n_max\": %d, \"window\": %d, \"chain\": %d, \"tile\": %d}",
                k ? "," : "", 1 << kv.first, kv.second.w, kv.second.m, kv.second.far);
        ++k;
    }
    fprintf(f, "%s]}\n", k ? "\n" : "");
    if (fclose(f) != 0) return -2;
    return k;
}

// Reads the integer after "key": in [p, end); false if absent or malformed.
static bool json_int(const char* p, const char* end, const char* key, long* out) {
    const size_t kl = strlen(key);
    for (const char* q = p; q + kl + 2 <= end; ++q) {
        if (q[0] != '"' || strncmp(q + 1, key, kl) != 0 || q[kl + 1] != '"') continue;
        const char* r = q + kl + 2;
        while (r < end && (*r == ' ' || *r == '\t' || *r == '\n' || *r == '\r')) ++r;
        if (r >= end || *r != ':') return false;
        ++r;
        char* e = nullptr;
        const long v = strtol(r, &e, 10);
        if (e == r || e > end) return false;
        *out = v;
        return true;
    }
    return false;
}

int gbr_tune_load(const char* path) {
    if (!path) return -1;
    FILE* f = fopen(path, "r");
    if (!f) return -2;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) {
        text.append(buf, got);
        if (text.size() > (1u << 20)) break;  // a table is a few hundred bytes
    }
    fclose(f);
    if (text.size() > (1u << 20)) return -3;
    // every {...} object holds one class; all are checked before any is kept
    std::map<int, TuneChoice> in;
    const char* s0 = text.c_str();
    const char* endp = s0 + text.size();
    const char* arr = strstr(s0, "\"tune\"");
    if (!arr) return -3;
    for (const char* p = strchr(arr, '{'); p && p < endp; p = strchr(p + 1, '{')) {
        const char* q = strchr(p, '}');
        if (!q) return -3;
        long nm, w, m, far;
        if (!json_int(p, q, "n_max", &nm) || !json_int(p, q, "window", &w) ||
            !json_int(p, q, "chain", &m) || !json_int(p, q, "tile", &far))
            return -3;
        if (nm < 32 || nm > (1L << 30) || (nm & (nm - 1)) != 0) return -3;
        if (w < 4 || w > WMAX || m < 1 || m > w - 2) return -3;
        if (far != 0 && far != UPD_BM && far != UPD_FAR) return -3;
        in[size_class((int)nm)] = TuneChoice{(int)w, (int)m, (int)far};
        p = q;
    }
    std::lock_guard<std::mutex> lk(g_tmu);
    auto& t = g_tune[current_device()];
    for (const auto& kv : in) t[kv.first] = kv.second;
    return (int)in.size();
}

}  // extern "C"
