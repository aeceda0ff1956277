// Reordering server: continuous batching of requests on one GPU.
//
// One long-lived server kernel (sched.cu) runs every task of every request.
// The host feeds it through a ring of (request, task) entries in device
// memory: each admitted request's tasks (window tasks and update tiles of
// Section 3.2 in its own queue order, then its eigenvalue task) are appended
// a chunk at a time, round-robin over the requests in flight, so a request
// that arrives while others are on the GPU starts within one chunk of
// their tasks instead of after them, and the SMs never wait for a launch.
//
// Requests are validated and planned on the submitting thread (the block
// structure is read from the caller's S), admitted in arrival order while
// their device footprint fits under the memory cap, copied to server-owned
// device memory where they stay until they complete, and copied back to the
// caller's buffers at the end.  Per request, every output element is
// computed by the same operations in the same order as when it runs alone
// (tasks only partition rows), so the result does not depend on the mix.
#include "host.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace gbr {
namespace {

using Clock = std::chrono::steady_clock;

// Host image of one planned pass of a request: its task graph in queue
// order plus the final eigenvalue task.
struct PassImage {
    std::vector<SchedTask> tasks;  // last: TASK_E
    std::vector<Window> wins;
    std::vector<int> deps, soff, succ;
    long long u_doubles = 0;
};

enum ReqState { Q_WAIT = 0, UPLOADING, FEEDING, RUNNING, COPYING, FINISHED };

struct Req {
    long long ticket = 0;
    int n = 0, ldS = 0, ldQ = 0;
    double* S = nullptr;
    double* Q = nullptr;
    double* er = nullptr;
    double* ei = nullptr;
    std::vector<uint8_t> sel;
    int w = WMAX, m = WMAX / 2;
    int msel = 0;
    size_t footprint = 0;
    Clock::time_point t_submit, t_done;
    PassImage img;                 // the pass being uploaded or run
    int state = Q_WAIT;
    int status = 0;
    // device
    char* dmat = nullptr;          // S | Q | counters | selection | eigenvalues
    char* dpass = nullptr;         // tasks | windows | deps | succ_off | succ | U | U slices
    double* dS = nullptr;
    double* dQ = nullptr;
    DevCounters* d_ctr = nullptr;
    uint8_t* d_sel = nullptr;
    double* d_eig = nullptr;
    int slot = -1;
    int id = 0;
    long long fed = 0;             // tasks of the current pass appended to the ring
    long long first_pos = -1;      // ring position of its first entry of this pass
    unsigned long long seen_rej = 0;
    cudaEvent_t ev = nullptr;      // upload or result copy
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t mat_bytes(int n, bool withQ) {
    const size_t m = al256((size_t)n * n * sizeof(double));
    return m * (withQ ? 2 : 1) + al256(sizeof(DevCounters)) + al256((size_t)std::max(1, n)) +
           al256(sizeof(double) * 2 * std::max(1, n));
}

size_t pass_bytes(const PassImage& p, bool ozaki) {
    return al256(sizeof(SchedTask) * p.tasks.size()) + al256(sizeof(Window) * std::max<size_t>(1, p.wins.size())) +
           al256(sizeof(int) * p.tasks.size()) + al256(sizeof(int) * (p.tasks.size() + 1)) +
           al256(sizeof(int) * std::max<size_t>(1, p.succ.size())) +
           al256(sizeof(double) * std::max<long long>(1, p.u_doubles)) +
           (ozaki ? al256(OZ_USLICE_BYTES * p.wins.size()) : 0);
}

// Task graph of one pass of one request, in list-scheduling order for P
// SMs, followed by the eigenvalue task.
void make_pass(int n, bool withQ, std::vector<Window> wins, int P, const CostModel& cm,
               PassImage& out) {
    out = PassImage{};
    TaskGraph G;
    if (!wins.empty()) {
        pipeline_order(n, wins);
        build_graph(n, wins, withQ, cm, G);
    }
    std::vector<int> order;
    queue_order(G, P, order);
    const int nt = (int)G.t.size();
    std::vector<int> pos(nt);
    for (int q = 0; q < nt; ++q) pos[order[q]] = q;
    out.tasks.resize(nt + 1);
    out.deps.resize(nt + 1);
    out.soff.assign(nt + 2, 0);
    out.succ.resize(G.succ.size());
    for (int q = 0; q < nt; ++q) {
        const HostTask& h = G.t[order[q]];
        out.tasks[q] = SchedTask{h.kind, h.win, h.y0, h.rows};
        out.deps[q] = G.ndeps[order[q]];
        out.soff[q + 1] = out.soff[q] + (G.soff[order[q] + 1] - G.soff[order[q]]);
    }
    for (int q = 0; q < nt; ++q) {
        int t = order[q], o2 = out.soff[q];
        for (int i = G.soff[t]; i < G.soff[t + 1]; ++i) out.succ[o2++] = pos[G.succ[i]];
    }
    out.soff[nt + 1] = out.soff[nt];
    out.tasks[nt] = SchedTask{TASK_E, 0, 0, 0};
    out.deps[nt] = nt;  // every other task of the request
    long long u = 0;
    for (Window& w : wins) {
        w.u_off = u;
        u += (long long)(w.e - w.s) * (w.e - w.s);
    }
    out.wins = std::move(wins);
    out.u_doubles = u;
}

// Standard real Schur form check on the host (Eq. 4): zeros below the
// subdiagonal, no two adjacent subdiagonal entries, standardized 2x2 blocks.
bool host_standard(int n, const double* S, int ldS) {
    for (int j = 0; j < n; ++j) {
        const double* col = S + (size_t)j * ldS;
        for (int i = j + 2; i < n; ++i)
            if (col[i] != 0.0) return false;
        if (j + 1 < n && col[j + 1] != 0.0) {
            if (j + 2 < n && S[(size_t)(j + 1) * ldS + j + 2] != 0.0) return false;
            const double a = col[j], c = col[j + 1];
            const double b = S[(size_t)(j + 1) * ldS + j], d = S[(size_t)(j + 1) * ldS + j + 1];
            if (a != d || !(b * c < 0.0)) return false;
        }
    }
    return true;
}

CostModel server_cost(const gbr_opts& o) {
    CostModel c;
    c.tile_rate = (o.precision == GBR_PREC_OZAKI) ? 100000.0
                : (o.precision == GBR_PREC_FMA)  ? 7600.0
                                                 : 6900.0;
    return c;
}

}  // namespace
}  // namespace gbr

struct gbr_server {
    gbr_server_cfg cfg{};
    int dev = 0, grid = 0, slots = 0;
    bool ozaki = false;
    cudaMemPool_t pool = nullptr;
    cudaStream_t ks = nullptr, cs = nullptr, ps = nullptr;  // kernel, copies, publishing
    // device
    char* dctl = nullptr;                 // head | tail | stop | err | ring | requests | scratch
    long long* d_head = nullptr;
    long long* d_tail = nullptr;
    int* d_stop = nullptr;
    int* d_err = nullptr;
    gbr::RingEntry* d_ring = nullptr;
    gbr::SrvReq* d_reqs = nullptr;
    long long cap = 0;
    // pinned host
    gbr::RingEntry* h_ring = nullptr;     // staging, same positions as the device ring
    gbr::SrvReq* h_reqs = nullptr;        // staging per slot
    gbr::DevCounters* h_ctr = nullptr;    // per slot
    long long* h_ctl = nullptr;           // head read back | tail to publish | stop | err
    int* h_done = nullptr;                // mapped completion words
    int* d_done = nullptr;
    bool kernel_running = false;
    long long tail = 0, head_seen = 0;
    int next_id = 1;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<std::shared_ptr<gbr::Req>> queue;
    std::vector<std::shared_ptr<gbr::Req>> live;   // admitted, not finished
    std::unordered_map<long long, std::shared_ptr<gbr::Req>> reqs;
    size_t rr = 0;                                 // round-robin cursor
    long long next_ticket = 0;
    size_t mem_used = 0;
    bool stop = false;
    int kerr = 0;
    std::thread th;
    // statistics
    long long submitted = 0, completed = 0, failed = 0, passes = 0, appends = 0;
    double peak_mem = 0.0, sum_live = 0.0;
    long long eigs_done = 0, live_samples = 0;
    std::vector<double> lat_ms;
    bool have_first = false;
    gbr::Clock::time_point t_first, t_last;
};

namespace gbr {
namespace {

void finish(gbr_server* s, Req& r, int status) {
    r.status = status;
    r.state = FINISHED;
    r.t_done = Clock::now();
    if (status < 0) s->failed += 1;
    else {
        s->completed += 1;
        s->eigs_done += r.msel;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
        s->t_last = r.t_done;
    }
    s->cv_done.notify_all();
}

void release(gbr_server* s, Req& r) {
    if (r.dmat) cudaFreeAsync(r.dmat, s->cs);
    if (r.dpass) cudaFreeAsync(r.dpass, s->cs);
    r.dmat = r.dpass = nullptr;
    if (r.ev) cudaEventDestroy(r.ev);
    r.ev = nullptr;
    if (r.slot >= 0) s->free_slots.push_back(r.slot);
    r.slot = -1;
    s->mem_used -= r.footprint;
    r.footprint = 0;
}

// Uploads a pass image and the request's table entry; records r.ev.
int upload_pass(gbr_server* s, Req& r) {
    PassImage& p = r.img;
    const size_t bytes = pass_bytes(p, s->ozaki);
    if (r.dpass) GBR_CK(cudaFreeAsync(r.dpass, s->cs), "server free");
    r.dpass = nullptr;
    GBR_CK(cudaMallocFromPoolAsync((void**)&r.dpass, bytes, s->pool, s->cs), "server alloc");
    char* q = r.dpass;
    SchedTask* d_tasks = (SchedTask*)q; q += al256(sizeof(SchedTask) * p.tasks.size());
    Window* d_wins = (Window*)q; q += al256(sizeof(Window) * std::max<size_t>(1, p.wins.size()));
    int* d_deps = (int*)q; q += al256(sizeof(int) * p.tasks.size());
    int* d_soff = (int*)q; q += al256(sizeof(int) * (p.tasks.size() + 1));
    int* d_succ = (int*)q; q += al256(sizeof(int) * std::max<size_t>(1, p.succ.size()));
    double* d_u = (double*)q; q += al256(sizeof(double) * std::max<long long>(1, p.u_doubles));
    unsigned char* d_us = s->ozaki ? (unsigned char*)q : nullptr;
    GBR_CK(cudaMemcpyAsync(d_tasks, p.tasks.data(), sizeof(SchedTask) * p.tasks.size(), cudaMemcpyHostToDevice, s->cs), "H2D tasks");
    if (!p.wins.empty())
        GBR_CK(cudaMemcpyAsync(d_wins, p.wins.data(), sizeof(Window) * p.wins.size(), cudaMemcpyHostToDevice, s->cs), "H2D windows");
    GBR_CK(cudaMemcpyAsync(d_deps, p.deps.data(), sizeof(int) * p.deps.size(), cudaMemcpyHostToDevice, s->cs), "H2D deps");
    GBR_CK(cudaMemcpyAsync(d_soff, p.soff.data(), sizeof(int) * p.soff.size(), cudaMemcpyHostToDevice, s->cs), "H2D succ offsets");
    if (!p.succ.empty())
        GBR_CK(cudaMemcpyAsync(d_succ, p.succ.data(), sizeof(int) * p.succ.size(), cudaMemcpyHostToDevice, s->cs), "H2D succ");
    r.id = s->next_id++;
    SrvReq& R = s->h_reqs[r.slot];
    R.inst = Inst{r.dS, r.dQ, r.d_sel, r.d_ctr, r.n, r.n, r.n, 0};
    R.tasks = d_tasks;
    R.wins = d_wins;
    R.deps = d_deps;
    R.succ_off = d_soff;
    R.succ = d_succ;
    R.upool = d_u;
    R.uslices = d_us;
    R.eig = r.d_eig;
    R.ntasks = (int)p.tasks.size();
    R.id = r.id;
    R.done_slot = r.slot;
    R.pad = 0;
    GBR_CK(cudaMemcpyAsync(s->d_reqs + r.slot, &R, sizeof(SrvReq), cudaMemcpyHostToDevice, s->cs), "H2D request");
    if (!r.ev) GBR_CK(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming), "event");
    GBR_CK(cudaEventRecord(r.ev, s->cs), "event");
    r.fed = 0;
    r.first_pos = -1;
    r.state = UPLOADING;
    s->passes += 1;
    return 0;
}

int admit(gbr_server* s, Req& r) {
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    const size_t mb = mat_bytes(r.n, r.Q != nullptr);
    GBR_CK(cudaMallocFromPoolAsync((void**)&r.dmat, mb, s->pool, s->cs), "server alloc");
    char* q = r.dmat;
    const size_t m = al256((size_t)r.n * r.n * sizeof(double));
    r.dS = (double*)q; q += m;
    if (r.Q) { r.dQ = (double*)q; q += m; }
    r.d_ctr = (DevCounters*)q; q += al256(sizeof(DevCounters));
    r.d_sel = (uint8_t*)q; q += al256((size_t)std::max(1, r.n));
    r.d_eig = (double*)q;
    DevCounters& hc = s->h_ctr[r.slot];
    hc = DevCounters{0, 0, INT_MAX, 0, 0};
    GBR_CK(cudaMemcpyAsync(r.d_ctr, &hc, sizeof hc, cudaMemcpyHostToDevice, s->cs), "H2D counters");
    GBR_CK(cudaMemcpyAsync(r.d_sel, r.sel.data(), r.n, cudaMemcpyHostToDevice, s->cs), "H2D selection");
    GBR_CK(cudaMemcpy2DAsync(r.dS, r.n * sizeof(double), r.S, (size_t)r.ldS * sizeof(double),
                             r.n * sizeof(double), r.n, cudaMemcpyHostToDevice, s->cs), "H2D S");
    if (r.Q)
        GBR_CK(cudaMemcpy2DAsync(r.dQ, r.n * sizeof(double), r.Q, (size_t)r.ldQ * sizeof(double),
                                 r.n * sizeof(double), r.n, cudaMemcpyHostToDevice, s->cs), "H2D Q");
    s->h_done[r.slot] = 0;
    return upload_pass(s, r);
}

// Results to the caller and the counters to the host; records r.ev.
int copy_back(gbr_server* s, Req& r) {
    GBR_CK(cudaMemcpyAsync(&s->h_ctr[r.slot], r.d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s->cs), "D2H counters");
    GBR_CK(cudaMemcpy2DAsync(r.S, (size_t)r.ldS * sizeof(double), r.dS, r.n * sizeof(double),
                             r.n * sizeof(double), r.n, cudaMemcpyDeviceToHost, s->cs), "D2H S");
    if (r.Q)
        GBR_CK(cudaMemcpy2DAsync(r.Q, (size_t)r.ldQ * sizeof(double), r.dQ, r.n * sizeof(double),
                                 r.n * sizeof(double), r.n, cudaMemcpyDeviceToHost, s->cs), "D2H Q");
    if (r.er) GBR_CK(cudaMemcpyAsync(r.er, r.d_eig, sizeof(double) * r.n, cudaMemcpyDeviceToHost, s->cs), "D2H eig");
    if (r.ei) GBR_CK(cudaMemcpyAsync(r.ei, r.d_eig + r.n, sizeof(double) * r.n, cudaMemcpyDeviceToHost, s->cs), "D2H eig");
    GBR_CK(cudaEventRecord(r.ev, s->cs), "event");
    r.state = COPYING;
    return 0;
}

// A further pass after rejected swaps: re-plan from the device state.
// Returns 1 if no block can move any more.
int replan(gbr_server* s, Req& r) {
    std::vector<uint8_t> sub(r.n, 0), sel(r.n);
    std::vector<double> sd(std::max(1, r.n - 1));
    if (r.n > 1)
        GBR_CK(cudaMemcpy2DAsync(sd.data(), sizeof(double), r.dS + 1, (size_t)(r.n + 1) * sizeof(double),
                                 sizeof(double), r.n - 1, cudaMemcpyDeviceToHost, s->cs), "D2H subdiagonal");
    GBR_CK(cudaMemcpyAsync(sel.data(), r.d_sel, r.n, cudaMemcpyDeviceToHost, s->cs), "D2H selection");
    GBR_CK(cudaStreamSynchronize(s->cs), "sync");
    for (int i = 0; i + 1 < r.n; ++i) sub[i] = sd[i] != 0.0;
    PlanState ps;
    init_state(ps, r.n, sub.data(), sel.data());
    std::vector<Window> wins;
    int nch = 0;
    plan_pass(ps, r.w, r.m, wins, nch);
    if (wins.empty()) return 1;
    make_pass(r.n, r.Q != nullptr, std::move(wins), s->grid, server_cost(s->cfg.opts), r.img);
    s->h_done[r.slot] = 0;
    return upload_pass(s, r);
}

// Appends chunks of the feeding requests' tasks to the ring, round-robin,
// publishes the new tail and reads back the kernel's head and error word.
int feed(gbr_server* s) {
    long long low = s->tail;  // lowest ring position still owned by a running pass
    std::vector<Req*> feeders;
    for (auto& rp : s->live) {
        Req& r = *rp;
        if ((r.state == FEEDING || r.state == RUNNING) && r.first_pos >= 0) low = std::min(low, r.first_pos);
        if (r.state == FEEDING) feeders.push_back(&r);
    }
    bool appended = false;
    if (!feeders.empty()) {
        const long long target = 8LL * s->grid;              // published entries not yet taken
        const long long chunk = std::max<long long>(64, 2LL * s->grid);
        for (size_t k = 0; k < feeders.size() * 4 && s->tail - s->head_seen < target; ++k) {
            Req& r = *feeders[(s->rr + k) % feeders.size()];
            const long long left = (long long)r.img.tasks.size() - r.fed;
            if (left <= 0) continue;
            long long cnt = std::min(left, chunk);
            if (r.first_pos < 0) low = std::min(low, s->tail);
            cnt = std::min(cnt, s->cap - (s->tail - low));  // ring space
            if (cnt <= 0) break;
            if (r.first_pos < 0) r.first_pos = s->tail;
            long long pos = s->tail;
            for (long long i = 0; i < cnt; ++i, ++pos)
                s->h_ring[pos % s->cap] = RingEntry{r.slot, (int)(r.fed + i)};
            long long a = s->tail % s->cap, remain = cnt;  // at most two pieces
            while (remain > 0) {
                const long long piece = std::min(remain, s->cap - a);
                GBR_CK(cudaMemcpyAsync(s->d_ring + a, s->h_ring + a, sizeof(RingEntry) * piece,
                                       cudaMemcpyHostToDevice, s->ps), "H2D ring");
                remain -= piece;
                a = (a + piece) % s->cap;
            }
            s->tail += cnt;
            r.fed += cnt;
            if (r.fed == (long long)r.img.tasks.size()) r.state = RUNNING;
            appended = true;
            s->appends += 1;
        }
        s->rr += 1;
    }
    if (appended) {
        s->h_ctl[1] = s->tail;
        GBR_CK(cudaMemcpyAsync(s->d_tail, &s->h_ctl[1], sizeof(long long), cudaMemcpyHostToDevice, s->ps), "H2D tail");
    }
    GBR_CK(cudaMemcpyAsync(&s->h_ctl[0], s->d_head, sizeof(long long), cudaMemcpyDeviceToHost, s->ps), "D2H head");
    GBR_CK(cudaMemcpyAsync(&s->h_ctl[3], s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->ps), "D2H err");
    GBR_CK(cudaStreamSynchronize(s->ps), "sync");
    s->head_seen = std::min(s->h_ctl[0], s->tail);
    s->kerr = (int)(s->h_ctl[3] & 0xffffffff);
    return 0;
}

void fail_all(gbr_server* s, int status) {
    for (auto& rp : s->live) {
        release(s, *rp);
        finish(s, *rp, status);
    }
    s->live.clear();
    while (!s->queue.empty()) {
        finish(s, *s->queue.front(), status);
        s->queue.pop_front();
    }
}

void server_loop(gbr_server* s) {
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progress = false;
        if (s->kerr) fail_all(s, s->kerr == 1 ? GBR_ERR_TIMEOUT : GBR_ERR_CUDA);
        // 1. state changes of the requests in flight
        for (size_t i = 0; i < s->live.size();) {
            Req& r = *s->live[i];
            int rc = 0;
            if (r.state == UPLOADING) {
                if (cudaEventQuery(r.ev) == cudaSuccess) {
                    r.state = FEEDING;
                    progress = true;
                } else {
                    (void)cudaGetLastError();  // not ready
                }
            } else if (r.state == RUNNING) {
                if (*(volatile int*)&s->h_done[r.slot] == r.id) {
                    rc = copy_back(s, r);
                    progress = true;
                }
            } else if (r.state == COPYING) {
                if (cudaEventQuery(r.ev) == cudaSuccess) {
                    progress = true;
                    const DevCounters c = s->h_ctr[r.slot];
                    const int st = (int)std::min<unsigned long long>(c.rejected, INT_MAX);
                    if (c.step_overflow) {
                        release(s, r);
                        finish(s, r, GBR_ERR_CUDA);
                    } else if (c.rejected > r.seen_rej) {
                        r.seen_rej = c.rejected;
                        rc = replan(s, r);
                        if (rc == 1) {  // nothing can move any more
                            rc = 0;
                            release(s, r);
                            finish(s, r, st);
                        }
                    } else {
                        release(s, r);
                        finish(s, r, st);
                    }
                } else {
                    (void)cudaGetLastError();
                }
            }
            if (rc) {
                release(s, r);
                finish(s, r, rc);
            }
            if (r.state == FINISHED) {
                s->live.erase(s->live.begin() + (long)i);
                continue;
            }
            ++i;
        }
        // 2. admission in arrival order, by footprint and slots
        while (!s->queue.empty() && !s->free_slots.empty()) {
            auto rp = s->queue.front();
            if (s->mem_used + rp->footprint > (size_t)s->cfg.mem_cap_bytes) break;
            s->queue.pop_front();
            s->mem_used += rp->footprint;
            s->peak_mem = std::max(s->peak_mem, (double)s->mem_used);
            int rc = admit(s, *rp);
            if (rc) {
                release(s, *rp);
                finish(s, *rp, rc);
                continue;
            }
            s->live.push_back(rp);
            progress = true;
        }
        // 3. the ring
        if (feed(s)) fail_all(s, GBR_ERR_CUDA);
        s->sum_live += (double)s->live.size();
        s->live_samples += 1;
        if (s->stop && s->queue.empty() && s->live.empty()) break;
        if (!progress) {
            bool gpu_busy = false;
            for (auto& rp : s->live) gpu_busy |= rp->state != FEEDING;
            s->cv.wait_for(lk, std::chrono::microseconds(gpu_busy ? 20 : 200));
        }
    }
}

}  // namespace
}  // namespace gbr

using namespace gbr;

extern "C" {

void gbr_server_default_cfg(gbr_server_cfg* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->mem_cap_bytes = 60000000000LL;
    cfg->max_inflight = 512;
    cfg->sms = 0;
    cfg->ring_entries = 1 << 22;
    cfg->idle_limit_ms = 0;
    cfg->device = -1;
    gbr_default_opts(&cfg->opts);
}

static void server_free(gbr_server* s) {
    if (!s) return;
    if (s->ks) cudaStreamDestroy(s->ks);
    if (s->cs) cudaStreamDestroy(s->cs);
    if (s->ps) cudaStreamDestroy(s->ps);
    if (s->dctl) cudaFree(s->dctl);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->h_ring) cudaFreeHost(s->h_ring);
    if (s->h_reqs) cudaFreeHost(s->h_reqs);
    if (s->h_ctr) cudaFreeHost(s->h_ctr);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    if (s->h_done) cudaFreeHost(s->h_done);
    delete s;
}

int gbr_server_create(const gbr_server_cfg* cfg, gbr_server** out) {
    if (!out) return -2;
    *out = nullptr;
    gbr_server_cfg c;
    if (cfg) c = *cfg; else gbr_server_default_cfg(&c);
    if (c.mem_cap_bytes <= 0 || c.max_inflight < 1 || c.sms < 0 || c.ring_entries < 1024 ||
        c.idle_limit_ms < 0)
        return -1;
    if (c.opts.sched != GBR_SCHED_PERSISTENT || c.opts.on_reject != GBR_ON_REJECT_CONTINUE)
        return GBR_ERR_UNSUPPORTED;
    if (c.opts.precision != GBR_PREC_DMMA && c.opts.precision != GBR_PREC_OZAKI &&
        c.opts.precision != GBR_PREC_FMA)
        return GBR_ERR_UNSUPPORTED;
    if (c.opts.precision == GBR_PREC_OZAKI && c.opts.slices != 0 && c.opts.slices != OZ_SLICES)
        return GBR_ERR_UNSUPPORTED;
    if (c.opts.window != GBR_AUTO && (c.opts.window < 4 || c.opts.window > WMAX)) return -1;
    if (c.opts.chain != GBR_AUTO && (c.opts.chain < 1 || (c.opts.window && c.opts.chain > c.opts.window - 2)))
        return -1;
    gbr_server* s = new (std::nothrow) gbr_server;
    if (!s) return GBR_ERR_NOMEM;
    struct Guard {
        gbr_server*& p;
        ~Guard() { server_free(p); }
    } guard{s};
    s->cfg = c;
    s->ozaki = (c.opts.precision == GBR_PREC_OZAKI);
    if (c.device >= 0) GBR_CK(cudaSetDevice(c.device), "cudaSetDevice");
    GBR_CK(cudaGetDevice(&s->dev), "cudaGetDevice");
    s->grid = c.sms > 0 ? std::min(c.sms, num_sms()) : num_sms();
    s->slots = c.max_inflight;
    s->cap = c.ring_entries;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->dev;
    GBR_CK(cudaMemPoolCreate(&s->pool, &props), "cudaMemPoolCreate");
    unsigned long long keep = (unsigned long long)c.mem_cap_bytes;
    GBR_CK(cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep), "pool attribute");
    GBR_CK(cudaStreamCreateWithFlags(&s->ks, cudaStreamNonBlocking), "stream");
    GBR_CK(cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking), "stream");
    GBR_CK(cudaStreamCreateWithFlags(&s->ps, cudaStreamNonBlocking), "stream");
    const size_t b_ctl = 256, b_ring = al256(sizeof(RingEntry) * s->cap);
    const size_t b_reqs = al256(sizeof(SrvReq) * s->slots);
    GBR_CK(cudaMalloc((void**)&s->dctl, b_ctl + b_ring + b_reqs), "cudaMalloc(server)");
    s->d_head = (long long*)s->dctl;
    s->d_tail = (long long*)(s->dctl + 8);
    s->d_stop = (int*)(s->dctl + 16);
    s->d_err = (int*)(s->dctl + 20);
    s->d_ring = (RingEntry*)(s->dctl + b_ctl);
    s->d_reqs = (SrvReq*)(s->dctl + b_ctl + b_ring);
    GBR_CK(cudaMemset(s->dctl, 0, b_ctl), "memset");
    GBR_CK(cudaMemset(s->d_reqs, 0, b_reqs), "memset");
    GBR_CK(cudaMallocHost((void**)&s->h_ring, sizeof(RingEntry) * s->cap), "cudaMallocHost");
    GBR_CK(cudaMallocHost((void**)&s->h_reqs, sizeof(SrvReq) * s->slots), "cudaMallocHost");
    GBR_CK(cudaMallocHost((void**)&s->h_ctr, sizeof(DevCounters) * s->slots), "cudaMallocHost");
    GBR_CK(cudaMallocHost((void**)&s->h_ctl, 64), "cudaMallocHost");
    memset(s->h_ctl, 0, 64);
    GBR_CK(cudaHostAlloc((void**)&s->h_done, sizeof(int) * s->slots, cudaHostAllocMapped), "cudaHostAlloc");
    memset(s->h_done, 0, sizeof(int) * s->slots);
    GBR_CK(cudaHostGetDevicePointer((void**)&s->d_done, s->h_done, 0), "cudaHostGetDevicePointer");
    for (int i = s->slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    GBR_CK(cudaDeviceSynchronize(), "sync");
    SrvParams P{};
    P.ring = s->d_ring;
    P.cap = s->cap;
    P.head = s->d_head;
    P.tail = s->d_tail;
    P.stop = s->d_stop;
    P.err = s->d_err;
    P.reqs = s->d_reqs;
    P.ozaki = s->ozaki ? 1 : 0;
    P.fp64_fma = (c.opts.precision == GBR_PREC_FMA) ? 1 : 0;
    P.done = s->d_done;
    P.strong = c.opts.strong_test;
    const long long lim_ms = c.opts.wait_limit_ms > 0 ? c.opts.wait_limit_ms : 60000;
    P.wait_limit_ns = lim_ms * 1000000;
    P.park_limit_ns = (c.idle_limit_ms > 0 ? c.idle_limit_ms : 3600000LL) * 1000000;
    GBR_CK(launch_server(P, s->grid, s->ks), "server kernel");
    s->kernel_running = true;
    s->th = std::thread(server_loop, s);
    *out = s;
    s = nullptr;
    return 0;
}

long long gbr_server_submit(gbr_server* s, int n, double* S, int ldS, double* Q, int ldQ,
                            const int* select, double* eig_re, double* eig_im) {
    if (!s) return -1;
    if (n < 0) return -2;
    if (n > 0 && !S) return -3;
    if (ldS < std::max(1, n)) return -4;
    if (Q && ldQ < std::max(1, n)) return -6;
    if (n > 0 && !select) return -7;
    auto r = std::make_shared<Req>();
    r->t_submit = Clock::now();
    r->n = n;
    r->S = S;
    r->ldS = ldS;
    r->Q = Q;
    r->ldQ = Q ? ldQ : 1;
    r->er = eig_re;
    r->ei = eig_im;
    bool valid = true;
    if (n > 0) {
        valid = !s->cfg.opts.validate || host_standard(n, S, ldS);
        std::vector<uint8_t> sub(n);
        for (int i = 0; i < n; ++i) sub[i] = (i + 1 < n && S[(size_t)i * ldS + i + 1] != 0.0) ? 1 : 0;
        r->sel.assign(n, 0);
        r->msel = selection_positions(n, sub.data(), select, r->sel.data());
        int w = s->cfg.opts.window, m = s->cfg.opts.chain;
        if (w == GBR_AUTO) {
            int tw = WMAX, tm = WMAX / 2;
            gbr_tune_get(n, &tw, &tm, nullptr);
            w = tw;
            if (m == GBR_AUTO) m = tm;
        }
        if (m == GBR_AUTO) m = std::max(1, w / 2);
        r->w = w;
        r->m = std::min(m, w - 2);
        if (valid) {
            PlanState ps;
            init_state(ps, n, sub.data(), r->sel.data());
            std::vector<Window> wins;
            int nch = 0;
            plan_pass(ps, r->w, r->m, wins, nch);
            make_pass(n, Q != nullptr, std::move(wins), s->grid, server_cost(s->cfg.opts), r->img);
            r->footprint = mat_bytes(n, Q != nullptr) + pass_bytes(r->img, s->ozaki);
            if (r->footprint > (size_t)s->cfg.mem_cap_bytes) return GBR_ERR_NOMEM;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return GBR_ERR_UNSUPPORTED;
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->submitted += 1;
    if (!s->have_first) {
        s->have_first = true;
        s->t_first = r->t_submit;
    }
    if (n == 0 || !valid) {  // nothing to run: complete at once
        finish(s, *r, valid ? 0 : -2);
        return r->ticket;
    }
    s->queue.push_back(r);
    s->cv.notify_all();
    return r->ticket;
}

static int poll_locked(gbr_server* s, long long ticket, int* status, int* m_out) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return -1;
    const Req& r = *it->second;
    if (r.state != FINISHED) return 0;
    if (status) *status = r.status;
    if (m_out) *m_out = r.msel;
    return 1;
}

int gbr_server_poll(gbr_server* s, long long ticket, int* status, int* m_out) {
    if (!s) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    return poll_locked(s, ticket, status, m_out);
}

int gbr_server_wait(gbr_server* s, long long ticket, int* status, int* m_out,
                    long long timeout_ms) {
    if (!s) return -1;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        int r = poll_locked(s, ticket, status, m_out);
        if (r != 0) return r;
        if (timeout_ms >= 0 && Clock::now() >= deadline) return 0;
        s->cv_done.wait_for(lk, std::chrono::milliseconds(5));
    }
}

static double pct(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = (size_t)std::min<double>((double)v.size() - 1,
                                              std::max(0.0, q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)k, v.end());
    return v[k];
}

int gbr_server_get_stats(gbr_server* s, gbr_server_stats* out) {
    if (!s || !out) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->passes = s->passes;
    out->p50_ms = pct(s->lat_ms, 0.50);
    out->p99_ms = pct(s->lat_ms, 0.99);
    double mx = 0.0, sum = 0.0;
    for (double v : s->lat_ms) {
        mx = std::max(mx, v);
        sum += v;
    }
    out->max_ms = mx;
    out->mean_ms = s->lat_ms.empty() ? 0.0 : sum / (double)s->lat_ms.size();
    if (s->completed > 0 && s->have_first) {
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        if (span > 0) {
            out->req_per_s = (double)s->completed / span;
            out->eigs_per_s = (double)s->eigs_done / span;
        }
    }
    out->mean_inflight = s->live_samples ? s->sum_live / (double)s->live_samples : 0.0;
    out->peak_mem_bytes = s->peak_mem;
    return 0;
}

void gbr_server_destroy(gbr_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->dev);
    if (s->kernel_running) {
        // every request has finished: the CTAs leave their waits on the stop word
        s->h_ctl[2] = 1;
        cudaMemcpyAsync(s->d_stop, &s->h_ctl[2], sizeof(int), cudaMemcpyHostToDevice, s->ps);
        cudaStreamSynchronize(s->ps);
        cudaStreamSynchronize(s->ks);
        s->kernel_running = false;
    }
    cudaStreamSynchronize(s->cs);
    server_free(s);
}

}  // extern "C"
