// Host side of the library: errors, the window planner, the task graph of
// the persistent scheduler and its launch image.
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
// reports rejected swaps, the caller re-plans from the state read back from
// the device (stuck blocks then act as barriers) until nothing can move.
#include "host.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <queue>
#include <thread>

namespace gbr {

static thread_local std::string g_last_error;

void set_last_error(const std::string& s) { g_last_error = s; }
const char* last_error_cstr() { return g_last_error.c_str(); }

int cuda_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? GBR_ERR_NOMEM : GBR_ERR_CUDA;
}

int refuse_capture(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e == cudaErrorStreamCaptureImplicit || (e == cudaSuccess && cs != cudaStreamCaptureStatusNone)) {
        if (e != cudaSuccess) (void)cudaGetLastError();
        set_last_error("the stream is being captured into a CUDA graph; this call synchronizes it");
        return GBR_ERR_CAPTURING;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    return 0;
}

int num_sms() {
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

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------

void init_state(PlanState& st, int n, const uint8_t* sub, const uint8_t* sel) {
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
void sim_window(PlanState& st, int s, int e) {
    struct B { uint8_t sz, sel; };
    B out[WMAX_WIDE], pend[WMAX_WIDE];
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

void plan_pass(PlanState& st, int w, int m, std::vector<Window>& win, int& nchains) {
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

//

int selection_positions(int n, const uint8_t* sub, const int* select, uint8_t* sel) {
    int msel = 0;
    for (int p = 0; p < n;) {
        const int sz = (p + 1 < n && sub[p]) ? 2 : 1;
        uint8_t v = select[p] != 0;
        if (sz == 2) v |= select[p + 1] != 0;
        for (int t = 0; t < sz; ++t) sel[p + t] = v;
        msel += v * sz;
        p += sz;
    }
    return msel;
}

double update_flops(int n, const std::vector<Window>& win, bool withQ) {
    double fl = 0.0;
    for (const Window& w : win) {
        const double ww = (double)(w.e - w.s);
        fl += 2.0 * ww * ww * ((double)(n - w.e) + w.s + (withQ ? n : 0));
    }
    return fl;
}

// Windows of one sweep, in program order: chain by chain (chain c holds
// bulges [c nbc, c nbc + nb_c)), each chain's windows top to bottom.  A
// window [s, e) runs the chain steps [t0, t1) during which every active
// bulge j (k_j = tau - 3 j - 1) has its input column at or below s and its
// rows k_j + 1 .. k_j + 4 above e (or e = n): t1 = e - 3 unless e = n; the
// next window starts at the top bulge's position.  The first window of a
// chain starts at row 0 and holds all of the chain's introductions
// (3 (nb_c - 1) < w - 3).  Returns -1 (and no windows) if a window is too
// short to move its chain (w <= 3 nb_c + 1).
int plan_sweep(int n, int nbulges, int w, int nbc, std::vector<SweepWin>& out) {
    out.clear();
    if (n < 3 || nbulges <= 0) return 0;
    for (int c = 0, b0 = 0; b0 < nbulges; ++c, b0 += nbc) {
        const int nbk = std::min(nbc, nbulges - b0);
        const int t_end = (n - 3) + 3 * (nbk - 1) + 2;  // exclusive
        int t0 = 0, s = 0;
        for (;;) {
            const int e = std::min(n, s + w);
            const int t1 = (e == n) ? t_end : std::min(t_end, e - 3);
            // a window too short for the chain makes no progress
            if (t1 <= t0) {
                out.clear();
                return -1;
            }
            out.push_back(SweepWin{s, e, t0, t1, b0, nbk});
            if (t1 >= t_end) break;
            const int ktop = t1 - 3 * (nbk - 1) - 1;
            s = std::max(0, ktop);
            t0 = t1;
        }
    }
    return 0;
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
// Duration model for the queue order only (relative values matter): a window
// task takes about cm.win_us_128 at w = 128, an update tile is a product of
// rows x w x w at cm.tile_rate flops per microsecond of one SM.
static double dur_window(const CostModel& cm, int w) { return cm.win_us_128 * (double)w * w / (128.0 * 128.0); }
static double dur_tile(const CostModel& cm, int rows, int w) {
    return 2.0 * rows * (double)w * w / cm.tile_rate + cm.task_us;
}

// Far-tile height: 256 panel rows up to n = 6000, then growing with n (the
// task count and the host time to order it grow as n^3 / far), at most 1024.
int far_rows(int n) {
    int f = UPD_FAR;
    while (f < 1024 && f * 24 < n) f *= 2;
    return f;
}

void build_graph(int n, const std::vector<Window>& wins, bool withQ, const CostModel& cm,
                 TaskGraph& G, int far, int threads, bool withZ) {
    const int FAR = far > 0 ? far : far_rows(n);
    std::vector<HostTask>& T = G.t;
    std::vector<std::pair<int, int>> edges;
    T.clear();
    {
        // capacity: per window its task and at most the near tiles, the far
        // tiles of the left / right panels and the Q and Z tiles
        const size_t per = 2 + 4 * (size_t)UPD_NEAR / UPD_BM + 4 * ((size_t)n / FAR + 1);
        T.reserve(wins.size() * per);
        edges.reserve(wins.size() * per);
    }
    for (int i = 0; i < (int)wins.size(); ++i) {
        const int s = wins[i].s, e = wins[i].e, w = e - s;
        const int iw = (int)T.size();
        T.push_back(HostTask{TASK_W, i, 0, 0, 0, Rect{s, e, s, e}, dur_window(cm, w)});
        // left panel: columns [e, n); 64-column tiles within UPD_NEAR of the
        // window (the next windows of the chain wait on those), far
        // tiles (FAR columns) beyond, each on a global grid so tiles of windows line up
        for (int c = e; c < n;) {
            const int g = (c - e < UPD_NEAR) ? UPD_BM : FAR;
            int ce = std::min(n, (c / g + 1) * g);
            edges.push_back({iw, (int)T.size()});
            T.push_back(HostTask{TASK_L, i, c - e, ce - c, 0, Rect{s, e, c, ce},
                                 cm.lr_mats * dur_tile(cm, ce - c, w)});
            c = ce;
        }
        // right panel: rows [0, s); 64-row tiles within UPD_NEAR above the window
        for (int r = 0; r < s;) {
            const bool near = (s - r <= UPD_NEAR);
            const int g = near ? UPD_BM : FAR;
            int re = std::min(s, (r / g + 1) * g);
            if (!near && re > s - UPD_NEAR) re = std::max(r + 1, s - UPD_NEAR);
            edges.push_back({iw, (int)T.size()});
            T.push_back(HostTask{TASK_R, i, r, re - r, 0, Rect{r, re, s, e},
                                 cm.lr_mats * dur_tile(cm, re - r, w)});
            r = re;
        }
        // Q panel: no window waits on Q, so far tiles throughout
        if (withQ)
            for (int r = 0; r < n;) {
                int re = std::min(n, (r / FAR + 1) * FAR);
                edges.push_back({iw, (int)T.size()});
                T.push_back(HostTask{TASK_Q, i, r, re - r, 1, Rect{r, re, s, e}, dur_tile(cm, re - r, w)});
                r = re;
            }
        // Z panel of a generalized form: like Q, on its own matrix
        if (withZ)
            for (int r = 0; r < n;) {
                int re = std::min(n, (r / FAR + 1) * FAR);
                edges.push_back({iw, (int)T.size()});
                T.push_back(HostTask{TASK_Z, i, r, re - r, 2, Rect{r, re, s, e}, dur_tile(cm, re - r, w)});
                r = re;
            }
    }
    // Dependences in program order on exact rectangles, found through a grid
    // of CB x CB cells: each cell lists the tasks touching it, newest last,
    // with each task's rectangle clipped to the cell (cell-relative bytes).
    // Within one cell, every task ends up ordered (directly or through newer
    // tasks) after every earlier task that overlaps it there.  A pair of
    // overlapping tasks is therefore looked at only in the first cell row
    // where their rectangles overlap: the cell rows are split among threads
    // (row cr to thread cr mod NT), each thread runs the whole task list over
    // its own rows, and no pair is emitted by two threads.
    const int CB = UPD_BM;
    static_assert(UPD_BM <= 255, "cell-relative coordinates are bytes");
    const int nc = (n + CB - 1) / CB;
    struct Entry {
        int task;
        uint8_t r0, r1, c0, c1;  // clipped rectangle, relative to the cell
        uint8_t starts;          // the task's rectangle starts in this cell row
    };
    constexpr int INLINE = 14;   // entries kept in the cell itself (lists are short)
    struct Cell {
        int cnt = 0;
        Entry e[INLINE];
        std::vector<Entry> more;  // entries beyond INLINE (rare)
        Entry& at(int k) { return k < INLINE ? e[k] : more[k - INLINE]; }
        void push(const Entry& x) {
            if (cnt < INLINE) e[cnt] = x;
            else if ((int)more.size() > cnt - INLINE) more[cnt - INLINE] = x;
            else more.push_back(x);
            ++cnt;
        }
    };
    const int nqb = (n + FAR - 1) / FAR;
    const int NT = std::max(1, std::min(threads, nc));
    std::vector<std::vector<std::pair<int, int>>> tedges(NT);
    auto worker = [&](int k) {
        std::vector<std::pair<int, int>>& out = tedges[k];
        const int myrows = (nc - k + NT - 1) / NT;
        std::vector<Cell> cells((size_t)std::max(0, myrows) * nc);
        // Q tiles all lie on the FAR row grid, so within a row block two Q
        // tasks conflict exactly when their column ranges overlap: the last Q
        // task per (row block, column) gives the exact, minimal predecessors.
        // (the same for the Z tiles of a generalized form, in lastz)
        const int myq = (nqb - k + NT - 1) / NT;
        std::vector<int> lastq(withQ ? (size_t)std::max(0, myq) * n : 0, -1);
        std::vector<int> lastz(withZ ? (size_t)std::max(0, myq) * n : 0, -1);
        std::vector<int> stamp(T.size(), -1);
        for (int t = 0; t < (int)T.size(); ++t) {
            const Rect R = T[t].rc;
            if (T[t].kind == TASK_Q || T[t].kind == TASK_Z) {
                const int qb = R.r0 / FAR;
                if (qb % NT != k) continue;
                int* last = &(T[t].kind == TASK_Q ? lastq : lastz)[(size_t)(qb / NT) * n];
                int prev = -1;
                for (int c = R.c0; c < R.c1; ++c) {
                    const int u = last[c];
                    if (u >= 0 && u != prev && stamp[u] != t) {
                        stamp[u] = t;
                        out.push_back({u, t});
                    }
                    prev = u;
                    last[c] = t;
                }
                continue;
            }
            int cr = R.r0 / CB;
            cr += (k - cr % NT + NT) % NT;  // first of this thread's rows
            for (; cr * CB < R.r1; cr += NT) {
                const int br = cr * CB;
                const uint8_t tstarts = R.r0 >= br ? 1 : 0;
                for (int cc = R.c0 / CB; cc * CB < R.c1; ++cc) {
                    const int bc = cc * CB;
                    const Entry X{t, (uint8_t)(std::max(R.r0, br) - br), (uint8_t)(std::min(R.r1, br + CB) - br),
                                  (uint8_t)(std::max(R.c0, bc) - bc), (uint8_t)(std::min(R.c1, bc + CB) - bc),
                                  tstarts};
                    Cell& C = cells[(size_t)(cr / NT) * nc + cc];
                    // scanning from the newest, an older task is implied once a
                    // newer predecessor covers the whole region, and the scan ends
                    for (int j = C.cnt - 1; j >= 0; --j) {
                        const Entry& U = C.at(j);
                        if (U.r0 >= X.r1 || X.r0 >= U.r1 || U.c0 >= X.c1 || X.c0 >= U.c1) continue;
                        if ((tstarts | U.starts) && stamp[U.task] != t) {
                            stamp[U.task] = t;
                            out.push_back({U.task, t});
                        }
                        if (U.r0 <= X.r0 && U.r1 >= X.r1 && U.c0 <= X.c0 && U.c1 >= X.c1) break;
                    }
                    // compaction: an entry whose part of the cell lies inside the
                    // new task's part precedes it and can never be needed again
                    int keep = 0;
                    for (int j = 0; j < C.cnt; ++j) {
                        const Entry U = C.at(j);
                        if (!(X.r0 <= U.r0 && X.r1 >= U.r1 && X.c0 <= U.c0 && X.c1 >= U.c1)) C.at(keep++) = U;
                    }
                    C.cnt = keep;
                    C.push(X);
                }
            }
        }
    };
    if (NT == 1) {
        worker(0);
    } else {
        std::vector<std::thread> th;
        for (int k = 0; k < NT; ++k) th.emplace_back(worker, k);
        for (auto& x : th) x.join();
    }
    // No edge is listed twice: a pair is emitted only in its first common cell
    // row, where the thread stamps each predecessor once per task, and a
    // window task overlaps none of its own tiles.  CSR straight from the
    // window-to-tile edges and the threads' lists, in that order.
    const int nt = (int)T.size();
    G.ndeps.assign(nt, 0);
    G.soff.assign(nt + 1, 0);
    size_t ne = edges.size();
    for (const auto& v : tedges) ne += v.size();
    G.succ.resize(ne);
    auto count = [&](const std::vector<std::pair<int, int>>& v) {
        for (const auto& ed : v) {
            G.ndeps[ed.second]++;
            G.soff[ed.first + 1]++;
        }
    };
    count(edges);
    for (const auto& v : tedges) count(v);
    for (int i = 0; i < nt; ++i) G.soff[i + 1] += G.soff[i];
    std::vector<int> fill(G.soff.begin(), G.soff.end() - 1);
    for (const auto& ed : edges) G.succ[fill[ed.first]++] = ed.second;
    for (const auto& v : tedges)
        for (const auto& ed : v) G.succ[fill[ed.first]++] = ed.second;
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
void pipeline_order(int n, std::vector<Window>& wins) {
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
void queue_order(const TaskGraph& G, int P, std::vector<int>& order, double* cp_us,
                 double* sim_us) {
    const int nt = (int)G.t.size();
    std::vector<double> dur(nt), bl(nt, 0.0);
    for (int t = 0; t < nt; ++t) dur[t] = G.t[t].dur;
    for (int t = nt - 1; t >= 0; --t) {
        double m = 0.0;
        for (int i = G.soff[t]; i < G.soff[t + 1]; ++i) m = std::max(m, bl[G.succ[i]]);
        bl[t] = dur[t] + m;
    }
    if (cp_us) {
        double m = 0.0;
        for (int t = 0; t < nt; ++t) m = std::max(m, bl[t]);
        *cp_us = m;
    }
    std::vector<int> indeg(G.ndeps);
    // ready: max-heap on (bottom level, lower index first); running: min-heap
    // on finish time.  Both are plain binary heaps over small structs.
    struct RK {
        double key;
        int t;
    };
    auto ready_less = [](const RK& a, const RK& b) {  // a below b in the max-heap
        return a.key < b.key || (a.key == b.key && a.t > b.t);
    };
    auto run_less = [](const RK& a, const RK& b) {  // a below b in the min-heap
        return a.key > b.key || (a.key == b.key && a.t > b.t);
    };
    std::vector<RK> ready, running;
    ready.reserve(1024);
    running.reserve((size_t)P + 1);
    for (int t = 0; t < nt; ++t)
        if (indeg[t] == 0) ready.push_back({bl[t], t});
    std::make_heap(ready.begin(), ready.end(), ready_less);
    order.clear();
    order.reserve(nt);
    int free = P;
    double now = 0.0;
    while ((int)order.size() < nt) {
        while (free > 0 && !ready.empty()) {
            std::pop_heap(ready.begin(), ready.end(), ready_less);
            const int t = ready.back().t;
            ready.pop_back();
            order.push_back(t);
            running.push_back({now + dur[t], t});
            std::push_heap(running.begin(), running.end(), run_less);
            --free;
        }
        if (running.empty()) break;  // cannot happen for an acyclic graph
        now = running.front().key;
        if (sim_us) *sim_us = now;
        while (!running.empty() && running.front().key <= now) {
            std::pop_heap(running.begin(), running.end(), run_less);
            const int t = running.back().t;
            running.pop_back();
            ++free;
            for (int i = G.soff[t]; i < G.soff[t + 1]; ++i) {
                const int s = G.succ[i];
                if (--indeg[s] == 0) {
                    ready.push_back({bl[s], s});
                    std::push_heap(ready.begin(), ready.end(), ready_less);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launch image of the persistent scheduler over one or more instances.
// ---------------------------------------------------------------------------
int sched_prepare(std::vector<InstPlan>& plans, const gbr_opts& o, const CostModel& cm, int grid,
                  const std::function<void*(size_t)>& alloc, SchedLaunch* L, SchedInfo* info,
                  cudaStream_t st) {
    const bool ozaki = (o.precision == GBR_PREC_OZAKI);
    const size_t ni = plans.size();
    auto th0 = std::chrono::steady_clock::now();
    // per-instance program order and task graph; instances are independent
    std::vector<TaskGraph> Gs(ni);
    const unsigned nth = std::min<unsigned>(16, std::max(1u, std::thread::hardware_concurrency()));
    auto work = [&](size_t i) {
        if (!plans[i].in_pipeline_order) pipeline_order(plans[i].d.n, plans[i].wins);
        build_graph(plans[i].d.n, plans[i].wins, plans[i].d.Q != nullptr, cm, Gs[i], plans[i].far,
                    ni >= 64 ? 1 : (int)nth, plans[i].d.T != nullptr && plans[i].d.Z != nullptr);
    };
    if (ni >= 64 && nth > 1) {
        std::vector<std::thread> th;
        for (unsigned k = 0; k < nth; ++k)
            th.emplace_back([&, k] {
                for (size_t i = k; i < ni; i += nth) work(i);
            });
        for (auto& t : th) t.join();
    } else {
        for (size_t i = 0; i < ni; ++i) work(i);
    }
    // merge: windows and tasks of instance i follow those of instance i - 1
    TaskGraph M;
    std::vector<Window> wins;
    long long u_total = 0;
    size_t nt_total = 0, ne_total = 0;
    for (size_t i = 0; i < ni; ++i) {
        nt_total += Gs[i].t.size();
        ne_total += Gs[i].succ.size();
    }
    M.t.reserve(nt_total);
    M.ndeps.reserve(nt_total);
    M.soff.reserve(nt_total + 1);
    M.succ.reserve(ne_total);
    M.soff.push_back(0);
    for (size_t i = 0; i < ni; ++i) {
        const int wbase = (int)wins.size(), tbase = (int)M.t.size();
        for (Window w : plans[i].wins) {
            w.inst = (int)i;
            w.u_off = u_total;
            // a generalized instance keeps UQ and UZ per window
            u_total += (long long)(w.e - w.s) * (w.e - w.s) * (plans[i].d.T ? 2 : 1);
            wins.push_back(w);
        }
        const TaskGraph& G = Gs[i];
        for (size_t t = 0; t < G.t.size(); ++t) {
            HostTask h = G.t[t];
            h.win += wbase;
            M.t.push_back(h);
            M.ndeps.push_back(G.ndeps[t]);
            for (int k = G.soff[t]; k < G.soff[t + 1]; ++k) M.succ.push_back(G.succ[k] + tbase);
            M.soff.push_back((int)M.succ.size());
        }
    }
    auto th1 = std::chrono::steady_clock::now();
    std::vector<int> order;
    double cp = 0.0, sim = 0.0;
    queue_order(M, grid, order, &cp, &sim);
    auto th2 = std::chrono::steady_clock::now();
    const int nt = (int)M.t.size();
    if ((int)order.size() != nt) {
        set_last_error("scheduler: task graph is not acyclic");
        return GBR_ERR_CUDA;
    }
    if (info) {
        info->tasks += nt;
        info->cp_us = cp;
        info->sim_us = sim;
        info->graph_ms = std::chrono::duration<double, std::milli>(th1 - th0).count();
        info->order_ms = std::chrono::duration<double, std::milli>(th2 - th1).count();
    }
    std::vector<int> pos(nt);
    for (int q = 0; q < nt; ++q) pos[order[q]] = q;
    std::vector<SchedTask> tq(nt);
    std::vector<int> deps(nt), soff(nt + 1, 0), succ(M.succ.size());
    for (int q = 0; q < nt; ++q) {
        const HostTask& h = M.t[order[q]];
        tq[q] = SchedTask{h.kind, h.win, h.y0, h.rows};
        deps[q] = M.ndeps[order[q]];
        soff[q + 1] = soff[q] + (M.soff[order[q] + 1] - M.soff[order[q]]);
    }
    for (int q = 0; q < nt; ++q) {
        int t = order[q], o2 = soff[q];
        for (int i = M.soff[t]; i < M.soff[t + 1]; ++i) succ[o2++] = pos[M.succ[i]];
    }
    if ((o.inject & GBR_INJECT_STALL) && nt > 1) deps[nt - 1] += 1;  // a predecessor that never ends
    std::vector<Inst> itab(ni);
    for (size_t i = 0; i < ni; ++i) itab[i] = plans[i].d;

    // device image: inst | tasks | wins | deps | deps_init | soff | succ | ctl | trace | U slices
    // | split-precision scratch | U pool
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_inst = al(sizeof(Inst) * std::max<size_t>(1, ni));
    const size_t b_tasks = al(sizeof(SchedTask) * std::max(1, nt));
    const size_t b_wins = al(sizeof(Window) * std::max<size_t>(1, wins.size()));
    const size_t b_deps = al(sizeof(int) * std::max(1, nt));
    const size_t b_soff = al(sizeof(int) * (nt + 1));
    const size_t b_succ = al(sizeof(int) * std::max<size_t>(1, succ.size()));
    const size_t b_ctl = 256;
    const size_t b_tr = (o.timing >= 2) ? al(sizeof(unsigned long long) * 4 * std::max(1, nt)) : 0;
    // digit slices per window: one U, or UQ and UZ for a generalized instance
    bool pair = false;
    for (size_t i = 0; i < ni; ++i) pair |= (plans[i].d.T != nullptr);
    const size_t b_us = ozaki ? al(OZ_USLICE_BYTES * wins.size() * (pair ? 2 : 1)) : 0;
    // windows wider than WMAX: the wide kernel instance, with a packed-window
    // scratch area per CTA (reordering of standard forms, FP64 tiles only)
    int wmax_win = 0;
    for (const Window& w : wins) wmax_win = std::max(wmax_win, w.e - w.s);
    const bool wide = wmax_win > WMAX;
    if (wide && (ozaki || pair || wmax_win > WMAX_WIDE)) {
        set_last_error("scheduler: windows wider than 128 need FP64 updates of a standard form");
        return GBR_ERR_UNSUPPORTED;
    }
    const size_t b_wscr = wide ? al(sizeof(double) * WIDE_SP_STRIDE * (size_t)grid) : 0;
    const size_t b_u = al(sizeof(double) * std::max<long long>(1, u_total));
    // ABORT on rejection: one word per window (its task did nothing); every
    // window task writes its own before its tiles read it
    const bool abort = (o.on_reject == GBR_ON_REJECT_ABORT);
    const size_t b_ws = abort ? al(sizeof(int) * std::max<size_t>(1, wins.size())) : 0;
    const size_t total = b_inst + b_tasks + b_wins + 2 * b_deps + b_soff + b_succ + b_ctl + b_tr +
                         b_us + b_ws + b_wscr + b_u;
    char* p = (char*)alloc(total);
    if (!p) return GBR_ERR_NOMEM;
    Inst* d_inst = (Inst*)p; p += b_inst;
    SchedTask* d_tasks = (SchedTask*)p; p += b_tasks;
    Window* d_wins = (Window*)p; p += b_wins;
    int* d_deps = (int*)p; p += b_deps;
    int* d_deps0 = (int*)p; p += b_deps;
    int* d_soff = (int*)p; p += b_soff;
    int* d_succ = (int*)p; p += b_succ;
    int* d_ctl = (int*)p; p += b_ctl;
    unsigned long long* d_tr = b_tr ? (unsigned long long*)p : nullptr; p += b_tr;
    unsigned char* d_us = b_us ? (unsigned char*)p : nullptr; p += b_us;
    int* d_ws = b_ws ? (int*)p : nullptr; p += b_ws;
    double* d_wscr = b_wscr ? (double*)p : nullptr; p += b_wscr;
    double* d_u = (double*)p;
    GBR_CK(cudaMemcpyAsync(d_inst, itab.data(), sizeof(Inst) * ni, cudaMemcpyHostToDevice, st), "H2D instances");
    if (nt) {
        GBR_CK(cudaMemcpyAsync(d_tasks, tq.data(), sizeof(SchedTask) * nt, cudaMemcpyHostToDevice, st), "H2D tasks");
        GBR_CK(cudaMemcpyAsync(d_deps0, deps.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st), "H2D deps");
    }
    if (!wins.empty())
        GBR_CK(cudaMemcpyAsync(d_wins, wins.data(), sizeof(Window) * wins.size(), cudaMemcpyHostToDevice, st), "H2D windows");
    GBR_CK(cudaMemcpyAsync(d_soff, soff.data(), sizeof(int) * (nt + 1), cudaMemcpyHostToDevice, st), "H2D succ offsets");
    if (!succ.empty())
        GBR_CK(cudaMemcpyAsync(d_succ, succ.data(), sizeof(int) * succ.size(), cudaMemcpyHostToDevice, st), "H2D succ");
    GBR_CK(cudaStreamSynchronize(st), "sync");  // the host vectors go out of scope

    SchedParams& P = L->P;
    P = SchedParams{};
    P.strong = o.strong_test;
    P.ntasks = nt;
    P.inst = d_inst;
    P.tasks = d_tasks;
    P.wins = d_wins;
    P.deps_left = d_deps;
    P.succ_off = d_soff;
    P.succ = d_succ;
    P.upool = d_u;
    P.uslices = d_us;
    P.fp64_fma = (o.precision == GBR_PREC_FMA) ? 1 : 0;
    P.head = d_ctl;
    P.err = d_ctl + 1;
    P.abort_word = abort ? d_ctl + 2 : nullptr;   // reset with the control words per launch
    P.wskip = d_ws;
    const long long lim_ms = o.wait_limit_ms > 0 ? o.wait_limit_ms : 60000;
    P.wait_limit_ns = lim_ms * 1000000;
    P.trace = d_tr;
    P.mode = wide ? 3 : 0;
    P.wscr = d_wscr;
    L->grid = grid;
    L->deps_init = d_deps0;
    L->ctl = d_ctl;
    L->trace_bytes = b_tr;
    if (b_tr) L->tq.swap(tq);
    else L->tq.clear();
    return 0;
}

int sched_enqueue(const SchedLaunch& L, cudaStream_t st, const std::function<int(cudaStream_t)>& pre) {
    if (L.P.ntasks > 0)
        GBR_CK(cudaMemcpyAsync(L.P.deps_left, L.deps_init, sizeof(int) * L.P.ntasks,
                               cudaMemcpyDeviceToDevice, st), "restore dependency counters");
    GBR_CK(cudaMemsetAsync(L.ctl, 0, 256, st), "memset control");
    if (L.trace_bytes) GBR_CK(cudaMemsetAsync(L.P.trace, 0, L.trace_bytes, st), "memset trace");
    if (pre) {
        int rc = pre(st);
        if (rc) return rc;
    }
    if (L.P.ntasks > 0) GBR_CK(launch_sched(L.P, L.grid, st), "scheduler kernel");
    return 0;
}

}  // namespace gbr
