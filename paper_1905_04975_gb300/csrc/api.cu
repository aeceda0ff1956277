// C-ABI entry points, the window planner and the device scratch pool.
//
// Planner (Section 3.2: windows, chains, Fig. 2): selected blocks are
// grouped top to bottom into chains of at most m eigenvalues.  A chain is
// moved up by a sequence of diagonal windows of at most w rows: the first
// window ends at the chain's last block; each window brings the chain's
// blocks to its top; the next window ends where those blocks now end, until
// a window starts at the chain's target position.  Window edges never cut a
// 2x2 block.  The planner simulates every window as the stable partition the
// window kernel produces (selected blocks first, stuck blocks as barriers),
// so the whole window list is known before the first launch.  If the device
// reports rejected swaps, the planner re-runs on the state read back from the
// device (stuck blocks then act as barriers) until nothing can move.
#include "../../include/gbreorder.h"
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <climits>
#include <queue>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace gbr {

static thread_local std::string g_last_error;
static std::vector<long long> g_trace;  // last traced persistent launch, 8 words per task
static double g_last_cp_us = 0.0, g_last_sim_us = 0.0;  // last schedule: critical path, simulated
static double g_last_graph_ms = 0.0, g_last_order_ms = 0.0;  // host time: task graph, queue order

static int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? GBR_ERR_NOMEM : GBR_ERR_CUDA;
}

#define GBR_CK(call, what)                              \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------------------
// Device scratch pool: one grow-only allocation per device and purpose.
// ---------------------------------------------------------------------------
enum PoolSlot { POOL_SCRATCH = 0, POOL_HOST_S = 1, POOL_HOST_Q = 2, POOL_SCHED = 3, POOL_NSLOTS = 4 };
struct DevPool {
    void* ptr[POOL_NSLOTS] = {nullptr, nullptr, nullptr, nullptr};
    size_t bytes[POOL_NSLOTS] = {0, 0, 0, 0};
};
static std::mutex g_mu;  // serializes calls: the pool is shared per device
static DevPool g_pool[64];

static int pool_get(int slot, size_t bytes, void** out) {
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
// Planner
// ---------------------------------------------------------------------------
struct PlanState {
    int n = 0;
    std::vector<uint8_t> bsz;  // size of the block starting at a position, else 0
    std::vector<uint8_t> sel;  // SEL_* per position (uniform inside a block)
};

static void init_state(PlanState& st, int n, const uint8_t* sub, const uint8_t* sel) {
    st.n = n;
    st.bsz.assign(n, 0);
    st.sel.assign(sel, sel + n);
    for (int p = 0; p < n;) {
        int sz = (p + 1 < n && sub[p]) ? 2 : 1;
        st.bsz[p] = (uint8_t)sz;
        p += sz;
    }
}

// The window kernel's effect on the block order of [s, e): every selected
// block moves up past the unselected blocks above it, up to the window top or
// the nearest selected or stuck block; stuck blocks do not move.
static void sim_window(PlanState& st, int s, int e) {
    struct B { uint8_t sz, sel; };
    B out[WMAX], pend[WMAX];
    int no = 0, np = 0;
    for (int p = s; p < e;) {
        B b{st.bsz[p], st.sel[p]};
        if (b.sel == SEL_YES) {
            out[no++] = b;
        } else if (b.sel == SEL_STUCK) {
            for (int i = 0; i < np; ++i) out[no++] = pend[i];
            np = 0;
            out[no++] = b;
        } else {
            pend[np++] = b;
        }
        p += b.sz;
    }
    for (int i = 0; i < np; ++i) out[no++] = pend[i];
    int p = s;
    for (int i = 0; i < no; ++i) {
        for (int t = 0; t < out[i].sz; ++t) {
            st.bsz[p + t] = t == 0 ? out[i].sz : 0;
            st.sel[p + t] = out[i].sel;
        }
        p += out[i].sz;
    }
}

static void plan_pass(PlanState& st, int w, int m, std::vector<Window>& win, int& nchains) {
    const int n = st.n;
    int ks = 0;
    for (;;) {
        int pos = ks, first = -1;
        while (pos < n) {
            int sz = st.bsz[pos];
            if (st.sel[pos] == SEL_STUCK) {
                ks = pos + sz;
            } else if (st.sel[pos] == SEL_YES) {
                if (pos == ks) {
                    ks += sz;
                } else {
                    first = pos;
                    break;
                }
            }
            pos += sz;
        }
        if (first < 0) break;
        int cnt = 0, last_end = first;
        for (int p = first; p < n;) {
            int sz = st.bsz[p];
            if (st.sel[p] == SEL_STUCK) break;
            if (st.sel[p] == SEL_YES) {
                if (cnt > 0 && cnt + sz > m) break;
                cnt += sz;
                last_end = p + sz;
            }
            p += sz;
        }
        const int top = ks;
        int e_cur = last_end;
        for (;;) {
            int s_cur = e_cur - w > top ? e_cur - w : top;
            if (s_cur > top && st.bsz[s_cur] == 0) s_cur += 1;
            int c_in = 0;
            for (int p = s_cur; p < e_cur; p += st.bsz[p])
                if (st.sel[p] == SEL_YES) c_in += st.bsz[p];
            win.push_back(Window{s_cur, e_cur, nchains, 0});
            sim_window(st, s_cur, e_cur);
            if (s_cur == top) break;
            e_cur = s_cur + c_in;
        }
        ks = top + cnt;
        ++nchains;
    }
}

// ---------------------------------------------------------------------------
// Task graph for the persistent scheduler (Section 3.2, Fig. 2).
//
// Program order is the planner's window order; each window i contributes its
// window task W_i and update tiles of UPD_BM panel rows (left panel columns
// and right/Q panel rows on a global UPD_BM grid, so tiles of different
// windows line up).  A task depends on every earlier task whose exact
// rectangle of S (or of Q) overlaps its own -- not on tiles, so two tasks
// that touch different parts of a tile do not wait on each other -- and each
// update tile on its window task (it reads U_i).  Older overlapping tasks are
// skipped once a newer one covers the whole overlap (they are then
// predecessors of that newer task already).
// ---------------------------------------------------------------------------
struct Rect {
    int r0, r1, c0, c1;  // rows [r0, r1) x columns [c0, c1)
};
static inline bool rects_overlap(const Rect& a, const Rect& b) {
    return a.r0 < b.r1 && b.r0 < a.r1 && a.c0 < b.c1 && b.c0 < a.c1;
}
static inline bool rect_covers(const Rect& a, const Rect& b) {
    return a.r0 <= b.r0 && a.r1 >= b.r1 && a.c0 <= b.c0 && a.c1 >= b.c1;
}
static inline Rect rect_isect(const Rect& a, const Rect& b) {
    return Rect{std::max(a.r0, b.r0), std::min(a.r1, b.r1), std::max(a.c0, b.c0),
                std::min(a.c1, b.c1)};
}

struct HostTask {
    int kind, win, y0, rows, mat;  // mat 0 = S, 1 = Q
    Rect rc;
    double dur;                     // estimated duration (microseconds)
};

struct TaskGraph {
    std::vector<HostTask> t;
    std::vector<int> ndeps;
    std::vector<int> soff, succ;    // CSR successors, program order
};

// Duration model for the queue order only (relative values matter): a window
// task takes about 2.6 ms at w = 128 (measured), an update tile is a DMMA
// product of rows x w x w at ~6.9 GFLOP/s per SM.
static double dur_window(int w) { return 2600.0 * (double)w * w / (128.0 * 128.0); }
// flops per microsecond of one SM on an update tile: FP64 DMMA, or the
// split-precision form (28 bf16 slice products, integer combination)
static double g_tile_rate = 6900.0;
static double dur_tile(int rows, int w) { return 2.0 * rows * (double)w * w / g_tile_rate + 2.0; }

// Far-tile height: 256 panel rows up to n = 6000, then growing with n (the
// task count and the host time to order it grow as n^3 / far), at most 1024.
static int far_rows(int n) {
    int f = UPD_FAR;
    while (f < 1024 && f * 24 < n) f *= 2;
    return f;
}

static void build_graph(int n, const std::vector<Window>& wins, bool withQ, TaskGraph& G) {
    const int FAR = far_rows(n);
    std::vector<HostTask>& T = G.t;
    std::vector<std::pair<int, int>> edges;
    T.clear();
    for (int i = 0; i < (int)wins.size(); ++i) {
        const int s = wins[i].s, e = wins[i].e, w = e - s;
        const int iw = (int)T.size();
        T.push_back(HostTask{TASK_W, i, 0, 0, 0, Rect{s, e, s, e}, dur_window(w)});
        // left panel: columns [e, n); 64-column tiles within UPD_NEAR of the
        // window (the next windows of the chain wait on those), far
        // tiles (FAR columns) beyond, each on a global grid so tiles of windows line up
        for (int c = e; c < n;) {
            const int g = (c - e < UPD_NEAR) ? UPD_BM : FAR;
            int ce = std::min(n, (c / g + 1) * g);
            edges.push_back({iw, (int)T.size()});
            T.push_back(HostTask{TASK_L, i, c - e, ce - c, 0, Rect{s, e, c, ce}, dur_tile(ce - c, w)});
            c = ce;
        }
        // right panel: rows [0, s); 64-row tiles within UPD_NEAR above the window
        for (int r = 0; r < s;) {
            const int g = (s - r <= UPD_NEAR) ? UPD_BM : FAR;
            int re = std::min(s, (r / g + 1) * g);
            if (g == FAR && re > s - UPD_NEAR) re = std::max(r + 1, s - UPD_NEAR);
            edges.push_back({iw, (int)T.size()});
            T.push_back(HostTask{TASK_R, i, r, re - r, 0, Rect{r, re, s, e}, dur_tile(re - r, w)});
            r = re;
        }
        // Q panel: no window waits on Q, so far tiles throughout
        if (withQ)
            for (int r = 0; r < n;) {
                int re = std::min(n, (r / FAR + 1) * FAR);
                edges.push_back({iw, (int)T.size()});
                T.push_back(HostTask{TASK_Q, i, r, re - r, 1, Rect{r, re, s, e}, dur_tile(re - r, w)});
                r = re;
            }
    }
    // Dependences in program order on exact rectangles, found through a grid
    // of CB x CB cells: each cell lists the tasks touching it, newest last.
    const int CB = UPD_BM;
    const int nc = (n + CB - 1) / CB;
    std::vector<std::vector<int>> cellv;        // S cells: tasks touching the cell
    cellv.resize((size_t)nc * nc);
    // Q tiles all lie on the FAR row grid, so within a row block two Q
    // tasks conflict exactly when their column ranges overlap: the last Q task
    // per (row block, column) gives the exact, minimal predecessors.
    const int nqb = (n + FAR - 1) / FAR;
    std::vector<int> lastq(withQ ? (size_t)nqb * n : 0, -1);
    std::vector<int> stamp(T.size(), -1);
    // Scanning a cell from the newest task back; an older task is implied once
    // a newer predecessor covers the whole region (it overlaps that one, so it
    // precedes it), and the scan ends there.
    auto scan = [&](std::vector<int>& L, const Rect& X, int t) {
        for (int k = (int)L.size() - 1; k >= 0; --k) {
            const int u = L[k];
            const Rect& U = T[u].rc;
            if (!rects_overlap(U, X)) continue;
            if (stamp[u] != t) {
                stamp[u] = t;
                edges.push_back({u, t});
            }
            if (rect_covers(U, X)) break;
        }
    };
    for (int t = 0; t < (int)T.size(); ++t) {
        const Rect R = T[t].rc;
        const int kind = T[t].kind;
        if (kind == TASK_Q) {
            int* last = &lastq[(size_t)(R.r0 / FAR) * n];
            int prev = -1;
            for (int c = R.c0; c < R.c1; ++c) {
                const int u = last[c];
                if (u >= 0 && u != prev && stamp[u] != t) {
                    stamp[u] = t;
                    edges.push_back({u, t});
                }
                prev = u;
                last[c] = t;
            }
            continue;
        }
        for (int cr = R.r0 / CB; cr * CB < R.r1; ++cr)
            for (int cc = R.c0 / CB; cc * CB < R.c1; ++cc) {
                const Rect cell{cr * CB, std::min(n, (cr + 1) * CB), cc * CB, std::min(n, (cc + 1) * CB)};
                const Rect X = rect_isect(R, cell);
                const size_t ci = (size_t)cr * nc + cc;

                // all S tasks order against every overlapping earlier S task
                scan(cellv[ci], X, t);
                // compaction: an entry whose part of the cell lies inside the new
                // task's part precedes the new task and can never be needed again
                std::vector<int>& L = cellv[ci];
                size_t keep = 0;
                for (size_t k = 0; k < L.size(); ++k) {
                    const Rect I = rect_isect(T[L[k]].rc, cell);
                    if (!rect_covers(X, I)) L[keep++] = L[k];
                }
                L.resize(keep);
                L.push_back(t);
            }
    }
    // No edge is listed twice: the scans stamp each predecessor once per task,
    // and a window task overlaps none of its own tiles.
    const int nt = (int)T.size();
    G.ndeps.assign(nt, 0);
    G.soff.assign(nt + 1, 0);
    G.succ.resize(edges.size());
    for (auto& ed : edges) {
        G.ndeps[ed.second]++;
        G.soff[ed.first + 1]++;
    }
    for (int i = 0; i < nt; ++i) G.soff[i + 1] += G.soff[i];
    std::vector<int> fill(G.soff.begin(), G.soff.end() - 1);
    for (auto& ed : edges) G.succ[fill[ed.first]++] = ed.second;
}

// Program order for the persistent schedule.  Two windows whose row ranges do
// not overlap conflict only through a left update of one and a right update
// of the other, and those commute ((U_a^T X) U_b = U_a^T (X U_b)); so any
// order of whole windows that keeps the planner's order of every pair of
// overlapping windows computes the same result.  Windows are taken by level
// in the overlap graph (1 + the highest level of an earlier overlapping
// window), which interleaves the chains like a pipeline: a chain's early
// windows come before the previous chain's late ones, and the left/right
// updates of different chains are ordered by when their windows run instead
// of by chain.  Without this, each chain's deferred right updates wait for
// the previous chain's left updates and the chains form a convoy.
static void pipeline_order(int n, std::vector<Window>& wins) {
    std::vector<int> cover(n, 0), level(wins.size());
    for (size_t b = 0; b < wins.size(); ++b) {
        int lv = 0;
        for (int p = wins[b].s; p < wins[b].e; ++p) lv = std::max(lv, cover[p]);
        level[b] = lv + 1;
        for (int p = wins[b].s; p < wins[b].e; ++p) cover[p] = std::max(cover[p], lv + 1);
    }
    std::vector<int> idx(wins.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return level[a] < level[b]; });
    std::vector<Window> out(wins.size());
    for (size_t i = 0; i < idx.size(); ++i) out[i] = wins[idx[i]];
    wins.swap(out);
}

// Queue order: a list-scheduling simulation on P processors where the ready
// task with the longest remaining path to the end (bottom level) starts first;
// the queue is the order of simulated start times.  Every predecessor of a
// task starts (and finishes) before it, so it sits earlier in the queue.
static void queue_order(const TaskGraph& G, int P, std::vector<int>& order, double* cp_us = nullptr,
                        double* sim_us = nullptr) {
    const int nt = (int)G.t.size();
    std::vector<double> bl(nt, 0.0);
    for (int t = nt - 1; t >= 0; --t) {
        double m = 0.0;
        for (int i = G.soff[t]; i < G.soff[t + 1]; ++i) m = std::max(m, bl[G.succ[i]]);
        bl[t] = G.t[t].dur + m;
    }
    if (cp_us) {
        double m = 0.0;
        for (int t = 0; t < nt; ++t) m = std::max(m, bl[t]);
        *cp_us = m;
    }
    std::vector<int> indeg(G.ndeps);
    typedef std::pair<double, int> Key;
    std::priority_queue<std::pair<double, int>> ready;  // (bottom level, -index)
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> running;  // (finish, task)
    for (int t = 0; t < nt; ++t)
        if (indeg[t] == 0) ready.push({bl[t], -t});
    order.clear();
    order.reserve(nt);
    int free = P;
    double now = 0.0;
    while ((int)order.size() < nt) {
        while (free > 0 && !ready.empty()) {
            int t = -ready.top().second;
            ready.pop();
            order.push_back(t);
            running.push({now + G.t[t].dur, t});
            --free;
        }
        if (running.empty()) break;  // cannot happen for an acyclic graph
        now = running.top().first;
        if (sim_us) *sim_us = now;
        while (!running.empty() && running.top().first <= now) {
            int t = running.top().second;
            running.pop();
            ++free;
            for (int i = G.soff[t]; i < G.soff[t + 1]; ++i)
                if (--indeg[G.succ[i]] == 0) ready.push({bl[G.succ[i]], -G.succ[i]});
        }
    }
}

static int num_sms() {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        sms[dev] = v;
    }
    return sms[dev];
}

// Runs one planned pass with the persistent scheduler.  Returns 0 or an error.
static int run_persistent(int n, std::vector<Window> wins, double* S, int ldS, double* Q,
                          int ldQ, uint8_t* d_sel, DevCounters* d_ctr, const gbr_opts& o,
                          long long* ntasks_out, double* ms_out, cudaStream_t st) {
    const bool ozaki = (o.precision == GBR_PREC_OZAKI);
    g_tile_rate = ozaki ? 60000.0 : 6900.0;
    auto th0 = std::chrono::steady_clock::now();
    pipeline_order(n, wins);
    TaskGraph G;
    build_graph(n, wins, Q != nullptr, G);
    auto th1 = std::chrono::steady_clock::now();
    const int P = num_sms();
    std::vector<int> order;
    queue_order(G, P, order, &g_last_cp_us, &g_last_sim_us);
    auto th2 = std::chrono::steady_clock::now();
    g_last_graph_ms = std::chrono::duration<double, std::milli>(th1 - th0).count();
    g_last_order_ms = std::chrono::duration<double, std::milli>(th2 - th1).count();
    const int nt = (int)G.t.size();
    if ((int)order.size() != nt) {
        g_last_error = "scheduler: task graph is not acyclic";
        return GBR_ERR_CUDA;
    }
    std::vector<int> pos(nt);
    for (int q = 0; q < nt; ++q) pos[order[q]] = q;
    std::vector<SchedTask> tq(nt);
    std::vector<int> deps(nt), soff(nt + 1, 0), succ(G.succ.size());
    for (int q = 0; q < nt; ++q) {
        const HostTask& h = G.t[order[q]];
        tq[q] = SchedTask{h.kind, h.win, h.y0, h.rows};
        deps[q] = G.ndeps[order[q]];
        soff[q + 1] = soff[q] + (G.soff[order[q] + 1] - G.soff[order[q]]);
    }
    for (int q = 0; q < nt; ++q) {
        int t = order[q], o2 = soff[q];
        for (int i = G.soff[t]; i < G.soff[t + 1]; ++i) succ[o2++] = pos[G.succ[i]];
    }
    if ((o.inject & GBR_INJECT_STALL) && nt > 1) deps[nt - 1] += 1;  // a predecessor that never ends
    // device buffers (pool): tasks | wins | deps | soff | succ | head,err | U pool
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_tasks = al(sizeof(SchedTask) * nt), b_wins = al(sizeof(Window) * wins.size());
    const size_t b_deps = al(sizeof(int) * nt), b_soff = al(sizeof(int) * (nt + 1));
    const size_t b_succ = al(sizeof(int) * std::max<size_t>(1, succ.size())), b_ctl = 256;
    const size_t b_u = (size_t)wins.size() * WMAX * WMAX * sizeof(double);
    const size_t b_tr = (o.timing >= 2) ? al(sizeof(unsigned long long) * 4 * nt) : 0;
    const size_t b_us = ozaki ? al(OZ_USLICE_BYTES * wins.size()) : 0;
    const size_t b_oz = ozaki ? al(sizeof(double) * UPD_FAR * WMAX * (size_t)P) : 0;
    void* base = nullptr;
    int rc = pool_get(POOL_SCHED,
                      b_tasks + b_wins + b_deps + b_soff + b_succ + b_ctl + b_tr + b_us + b_oz + b_u,
                      &base);
    if (rc) return rc;
    char* p = (char*)base;
    SchedTask* d_tasks = (SchedTask*)p; p += b_tasks;
    Window* d_wins = (Window*)p; p += b_wins;
    int* d_deps = (int*)p; p += b_deps;
    int* d_soff = (int*)p; p += b_soff;
    int* d_succ = (int*)p; p += b_succ;
    int* d_ctl = (int*)p; p += b_ctl;
    unsigned long long* d_tr = b_tr ? (unsigned long long*)p : nullptr; p += b_tr;
    unsigned char* d_us = b_us ? (unsigned char*)p : nullptr; p += b_us;
    double* d_oz = b_oz ? (double*)p : nullptr; p += b_oz;
    double* d_u = (double*)p;
    GBR_CK(cudaMemcpyAsync(d_tasks, tq.data(), sizeof(SchedTask) * nt, cudaMemcpyHostToDevice, st), "H2D tasks");
    GBR_CK(cudaMemcpyAsync(d_wins, wins.data(), sizeof(Window) * wins.size(), cudaMemcpyHostToDevice, st), "H2D windows");
    GBR_CK(cudaMemcpyAsync(d_deps, deps.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st), "H2D deps");
    GBR_CK(cudaMemcpyAsync(d_soff, soff.data(), sizeof(int) * (nt + 1), cudaMemcpyHostToDevice, st), "H2D succ offsets");
    if (!succ.empty())
        GBR_CK(cudaMemcpyAsync(d_succ, succ.data(), sizeof(int) * succ.size(), cudaMemcpyHostToDevice, st), "H2D succ");
    GBR_CK(cudaMemsetAsync(d_ctl, 0, 256, st), "memset control");
    SchedParams P2;
    P2.n = n; P2.ldS = ldS; P2.ldQ = ldQ; P2.strong = o.strong_test; P2.ntasks = nt;
    P2.S = S; P2.Q = Q; P2.sel = d_sel; P2.ctr = d_ctr;
    P2.tasks = d_tasks; P2.wins = d_wins; P2.deps_left = d_deps; P2.succ_off = d_soff; P2.succ = d_succ;
    P2.upool = d_u; P2.head = d_ctl; P2.err = d_ctl + 1;
    const long long lim_ms = o.wait_limit_ms > 0 ? o.wait_limit_ms : 60000;
    P2.wait_limit = lim_ms * 1000000 / 128;
    P2.trace = d_tr;
    P2.uslices = d_us;
    P2.ozscratch = d_oz;
    if (d_tr) GBR_CK(cudaMemsetAsync(d_tr, 0, b_tr, st), "memset trace");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (o.timing) {
        GBR_CK(cudaEventCreate(&e0), "event");
        GBR_CK(cudaEventCreate(&e1), "event");
        GBR_CK(cudaEventRecord(e0, st), "event");
    }
    GBR_CK(launch_sched(P2, P, st), "scheduler kernel");
    if (o.timing) GBR_CK(cudaEventRecord(e1, st), "event");
    int h_err = 0;
    GBR_CK(cudaMemcpyAsync(&h_err, d_ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H err");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (o.timing) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *ms_out += ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    *ntasks_out += nt;
    if (d_tr) {
        std::vector<unsigned long long> raw((size_t)4 * nt);
        GBR_CK(cudaMemcpy(raw.data(), d_tr, sizeof(unsigned long long) * 4 * nt,
                          cudaMemcpyDeviceToHost), "D2H trace");
        g_trace.assign((size_t)8 * nt, 0);
        for (int q = 0; q < nt; ++q) {
            const SchedTask& k = tq[q];
            long long* r = &g_trace[(size_t)8 * q];
            r[0] = k.kind; r[1] = k.win; r[2] = k.y0; r[3] = k.rows;
            r[4] = (long long)raw[4 * q + 0];
            r[5] = (long long)raw[4 * q + 1];
            r[6] = (long long)raw[4 * q + 2];
            r[7] = (long long)raw[4 * q + 3];
        }
    }
    if (h_err) {
        g_last_error = "persistent scheduler: a task waited longer than wait_limit_ms";
        return GBR_ERR_TIMEOUT;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Reorder on device-resident S, Q.
// ---------------------------------------------------------------------------
static int check_opts(const gbr_opts* o) {
    if (o->window < 4 || o->window > WMAX) return -10;
    if (o->chain < 1 || o->chain > o->window - 2) return -10;
    if (o->precision != GBR_PREC_DMMA && o->precision != GBR_PREC_OZAKI) return GBR_ERR_UNSUPPORTED;
    if (o->precision == GBR_PREC_OZAKI &&
        (o->sched != GBR_SCHED_PERSISTENT || (o->slices != 0 && o->slices != OZ_SLICES)))
        return GBR_ERR_UNSUPPORTED;
    if (o->on_reject != GBR_ON_REJECT_CONTINUE) return GBR_ERR_UNSUPPORTED;
    if (o->sched != GBR_SCHED_PERSISTENT && o->sched != GBR_SCHED_SEQUENTIAL) return -10;
    if (o->wait_limit_ms < 0) return -10;
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
    if (o.validate) GBR_CK(launch_validate(n, S, ldS, d_ctr, st), "validate kernel");
    GBR_CK(launch_subdiag(n, S, ldS, d_sub, st), "subdiag kernel");
    std::vector<uint8_t> sub(n), sel(n);
    GBR_CK(cudaMemcpyAsync(sub.data(), d_sub, n, cudaMemcpyDeviceToHost, st), "D2H subdiag");
    GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (h_ctr.bad_column != INT_MAX) return -2;

    // selection per position; a 2x2 block is selected if either row is
    int msel = 0;
    for (int p = 0; p < n;) {
        int sz = (p + 1 < n && sub[p]) ? 2 : 1;
        uint8_t v = select[p] != 0;
        if (sz == 2) v |= select[p + 1] != 0;
        for (int t = 0; t < sz; ++t) sel[p + t] = v;
        msel += v * sz;
        p += sz;
    }
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
        plan_pass(ps, o.window, o.chain, win, nchains);
        if (win.empty()) break;
        if (o.sched == GBR_SCHED_PERSISTENT) {
            int rcs = run_persistent(n, win, S, ldS, Q, ldQ, d_sel, d_ctr, o, &ntasks, &ms_sched, st);
            if (rcs) return rcs;
            launches += 1;
            for (const Window& wdw : win) {
                double ww = (double)(wdw.e - wdw.s);
                flops += 2.0 * ww * ww * ((double)(n - wdw.e) + wdw.s + (Q ? n : 0));
            }
        } else
        for (const Window& wdw : win) {
            if (o.timing) GBR_CK(mark(evw), "event");
            GBR_CK(launch_window(n, wdw, S, ldS, d_sel, d_u, o.strong_test, d_ctr, st), "window kernel");
            if (o.timing) { GBR_CK(mark(evw), "event"); GBR_CK(mark(evu), "event"); }
            GBR_CK(launch_update(n, wdw, S, ldS, Q, ldQ, d_u, st), "update kernel");
            if (o.timing) GBR_CK(mark(evu), "event");
            double ww = (double)(wdw.e - wdw.s);
            flops += 2.0 * ww * ww * ((double)(n - wdw.e) + wdw.s + (Q ? n : 0));
            launches += 2;
        }
        nwin += (long long)win.size();
        GBR_CK(cudaMemcpyAsync(&h_ctr, d_ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st), "D2H counters");
        GBR_CK(cudaStreamSynchronize(st), "sync");
        if (h_ctr.rejected == seen_rej) break;  // the simulated plan was exact
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
        g_last_error = "window kernel exceeded its step bound";
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
        stats->tasks = ntasks;
        stats->sched_cp_ms = ntasks ? g_last_cp_us / 1e3 : 0.0;
        stats->sched_sim_ms = ntasks ? g_last_sim_us / 1e3 : 0.0;
        stats->ms_graph = ntasks ? g_last_graph_ms : 0.0;
        stats->ms_order = ntasks ? g_last_order_ms : 0.0;
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
    o->precision = GBR_PREC_DMMA;
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
    std::lock_guard<std::mutex> lock(g_mu);
    size_t mat = (size_t)n * n * sizeof(double);
    void *dS = nullptr, *dQ = nullptr;
    rc = pool_get(POOL_HOST_S, mat, &dS);
    if (rc) return rc;
    if (Q) {
        rc = pool_get(POOL_HOST_Q, mat, &dQ);
        if (rc) return rc;
    }
    GBR_CK(cudaMemcpy2DAsync(dS, n * sizeof(double), S, (size_t)ldS * sizeof(double),
                             n * sizeof(double), n, cudaMemcpyHostToDevice, st), "H2D S");
    if (Q)
        GBR_CK(cudaMemcpy2DAsync(dQ, n * sizeof(double), Q, (size_t)ldQ * sizeof(double),
                                 n * sizeof(double), n, cudaMemcpyHostToDevice, st), "H2D Q");
    rc = reorder_device(n, (double*)dS, n, (double*)dQ, n, select, eig_re, eig_im, m_out, o, stats, st);
    if (rc < 0) return rc;
    GBR_CK(cudaMemcpy2DAsync(S, (size_t)ldS * sizeof(double), dS, n * sizeof(double),
                             n * sizeof(double), n, cudaMemcpyDeviceToHost, st), "D2H S");
    if (Q)
        GBR_CK(cudaMemcpy2DAsync(Q, (size_t)ldQ * sizeof(double), dQ, n * sizeof(double),
                                 n * sizeof(double), n, cudaMemcpyDeviceToHost, st), "D2H Q");
    GBR_CK(cudaStreamSynchronize(st), "sync");
    if (stats)
        stats->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int gbr_plan(int n, const unsigned char* sub, const int* select, int window, int chain,
             int with_q, int* windows, int max_windows, int* chains, double* upd_flops) {
    if (n < 0) return -1;
    if (n > 0 && (!sub || !select)) return -2;
    if (window < 4 || window > WMAX) return -4;
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
// reorder: code running while a stream is being captured into a CUDA graph,
// programs whose memory is all handed out by their own arena, or processes
// where a cudaMalloc would synchronize the device at a bad moment.  For them
// this entry point takes its scratch (counters, block flags, selection
// flags, eigenvalue staging and one window accumulator) from a fixed array
// in device global memory that is part of the library image instead of the
// library's pool.  Every GPU that loads the library holds this array
// (GBR_NOALLOC_SCRATCH_BYTES) until the process exits.
// ---------------------------------------------------------------------------
static constexpr size_t kNoallocBytes = scratch_layout(GBR_NOALLOC_MAX_N).total;
static_assert(kNoallocBytes == GBR_NOALLOC_SCRATCH_BYTES, "header and layout disagree");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of g_noalloc_scratch for each device, looked up once with
// that device current (in host code the symbol is only a host-side stand-in).
static void* g_noalloc_ptr[64];

static int noalloc_scratch(char** out) {
    int dev = 0;
    GBR_CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) return GBR_ERR_CUDA;
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        GBR_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = (char*)g_noalloc_ptr[dev];
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
    if (o.precision != GBR_PREC_DMMA) return GBR_ERR_UNSUPPORTED;
    if (stats) memset(stats, 0, sizeof *stats);
    if (n == 0) {
        if (m_out) *m_out = 0;
        return 0;
    }
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
        case -10: return "invalid argument 10: window must be 4..128 and chain 1..window-2";
        case GBR_ERR_CUDA: return "CUDA error (see gbr_last_error)";
        case GBR_ERR_NOMEM: return "out of device memory";
        case GBR_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case GBR_ERR_UNSUPPORTED: return "unsupported option value";
        case GBR_ERR_NOALLOC_LIMIT:
            return "n exceeds GBR_NOALLOC_MAX_N, the size the no-allocation entry point supports";
        default: return "invalid argument";
    }
}

const char* gbr_last_error(void) { return g_last_error.c_str(); }

void gbr_release(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    for (int s = 0; s < POOL_NSLOTS; ++s) {
        if (g_pool[dev].ptr[s]) cudaFree(g_pool[dev].ptr[s]);
        g_pool[dev].ptr[s] = nullptr;
        g_pool[dev].bytes[s] = 0;
    }
}

int gbr_version(void) { return 100; }

}  // extern "C"
