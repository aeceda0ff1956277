// Host-only check of the persistent scheduler's task graph (compiled with the
// library's planner source by tests/test_task_graph.py; no GPU).  For a
// seeded block structure and selection (or a sweep plan) it builds the
// windows, the program order, the task graph and the queue order, and checks
// the sequential consistency the scheduler relies on:
//   * every dependence goes forward in program order;
//   * every pair of tasks whose rectangles overlap on the same matrix is
//     ordered: the later one is reachable from the earlier one;
//   * every tile depends on its window task;
//   * the queue order is a topological order of the graph.
// For a reordering it also checks the cuts of the chunked launches: every
// pair of overlapping windows keeps its planner order in the pipeline order
// (so every prefix of the pipeline order holds all earlier windows that
// overlap its windows), and the graph of each chunk (first 1/16, next 3/16,
// last 3/4) passes the same checks on its own.
// Prints "OK <edges>" or "FAIL <reason>" and exits 0 / 1.
#include "../paper_1905_04975_gb300/csrc/host.h"

#include <cstdio>
#include <cstdlib>
#include <vector>

using namespace gbr;
namespace gbr {
cudaError_t launch_sched(const SchedParams&, int, cudaStream_t) { return cudaSuccess; }
}  // namespace gbr

static unsigned long long rng_state = 88172645463325252ull;
static unsigned rnd() {
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return (unsigned)(rng_state >> 11);
}

static int mat_of(const HostTask& t) { return t.kind == TASK_Q ? 1 : (t.kind == TASK_Z ? 2 : 0); }

static bool overlap(const Rect& a, const Rect& b) {
    return a.r0 < b.r1 && b.r0 < a.r1 && a.c0 < b.c1 && b.c0 < a.c1;
}

// The checks of one task graph over windows in program order; *edges gets
// the edge count.  Prints the first failure.
static bool check_graph(int n, const std::vector<Window>& wins, bool withQ, bool withZ,
                        const CostModel& cm, long long* edges) {
    TaskGraph G;
    build_graph(n, wins, withQ, cm, G, 0, 3, withZ);
    const int nt = (int)G.t.size();
    // forward edges; reachability by bitsets in reverse program order
    const int W64 = (nt + 63) / 64;
    std::vector<unsigned long long> R((size_t)nt * W64, 0ull);
    for (int u = nt - 1; u >= 0; --u)
        for (int i = G.soff[u]; i < G.soff[u + 1]; ++i) {
            const int v = G.succ[i];
            if (v <= u) { printf("FAIL backward edge %d -> %d\n", u, v); return false; }
            R[(size_t)u * W64 + v / 64] |= 1ull << (v % 64);
            for (int k = 0; k < W64; ++k) R[(size_t)u * W64 + k] |= R[(size_t)v * W64 + k];
        }
    auto reach = [&](int a, int b) { return (R[(size_t)a * W64 + b / 64] >> (b % 64)) & 1ull; };
    std::vector<int> wtask(wins.size(), -1);
    for (int t = 0; t < nt; ++t)
        if (G.t[t].kind == TASK_W) wtask[G.t[t].win] = t;
    for (int t = 0; t < nt; ++t) {
        const HostTask& b = G.t[t];
        if (b.kind != TASK_W && !reach(wtask[b.win], t)) {
            printf("FAIL tile %d not after its window task\n", t);
            return false;
        }
        for (int a = 0; a < t; ++a) {
            const HostTask& x = G.t[a];
            if (mat_of(x) == mat_of(b) && overlap(x.rc, b.rc) && !reach(a, t)) {
                printf("FAIL overlapping tasks %d, %d unordered\n", a, t);
                return false;
            }
        }
    }
    std::vector<int> order;
    queue_order(G, 152, order);
    if ((int)order.size() != nt) { printf("FAIL order size\n"); return false; }
    std::vector<int> pos(nt, -1);
    for (int q = 0; q < nt; ++q) pos[order[q]] = q;
    for (int u = 0; u < nt; ++u)
        for (int i = G.soff[u]; i < G.soff[u + 1]; ++i)
            if (pos[G.succ[i]] <= pos[u]) { printf("FAIL queue order\n"); return false; }
    *edges = (long long)G.succ.size();
    return true;
}

int main(int argc, char** argv) {
    if (argc < 8) return 2;
    const int n = atoi(argv[1]), w = atoi(argv[2]), m = atoi(argv[3]);
    const bool withQ = atoi(argv[4]) != 0, withZ = atoi(argv[5]) != 0;
    rng_state += (unsigned long long)atoll(argv[6]) * 0x9E3779B97F4A7C15ull;
    const bool sweep = atoi(argv[7]) != 0;
    std::vector<Window> wins;
    if (sweep) {
        std::vector<SweepWin> sw;
        plan_sweep(n, m, w, std::max(1, w / 6), sw);  // m = bulges
        for (const SweepWin& x : sw) wins.push_back(Window{x.s, x.e, x.b0, 0, 0, x.t0, x.t1, x.b0, x.nb});
    } else {
        std::vector<uint8_t> sub(n, 0), sel(n, 0);
        for (int i = 0; i + 1 < n; ++i)
            if (rnd() % 10 < 4 && (i == 0 || !sub[i - 1])) sub[i] = 1;  // 2x2 blocks
        for (int i = 0; i < n;) {
            const int sz = sub[i] ? 2 : 1;
            const uint8_t s = (rnd() % 100) < 40 ? 1 : 0;
            for (int k = 0; k < sz; ++k) sel[i + k] = s;
            i += sz;
        }
        PlanState ps;
        init_state(ps, n, sub.data(), sel.data());
        int nch = 0;
        plan_pass(ps, w, m, wins, nch);
    }
    std::vector<Window> planner = wins;
    pipeline_order(n, wins);
    CostModel cm;
    if (withZ) cm.lr_mats = 2.0;
    if (!sweep) {
        // overlapping windows keep their planner order in the pipeline order
        auto key = [](const Window& x) { return ((long long)x.chain << 40) | ((long long)x.s << 20) | x.e; };
        std::vector<long long> kp(wins.size());
        for (size_t i = 0; i < wins.size(); ++i) kp[i] = key(wins[i]);
        std::vector<int> ppos(planner.size(), -1);
        for (size_t i = 0; i < planner.size(); ++i)
            for (size_t k = 0; k < wins.size(); ++k)
                if (kp[k] == key(planner[i])) { ppos[i] = (int)k; break; }
        for (size_t i = 0; i < planner.size(); ++i) {
            if (ppos[i] < 0) { printf("FAIL window lost by the pipeline order\n"); return 1; }
            for (size_t k = i + 1; k < planner.size(); ++k)
                if (planner[i].s < planner[k].e && planner[k].s < planner[i].e && ppos[i] > ppos[k]) {
                    printf("FAIL overlapping windows %zu, %zu reordered\n", i, k);
                    return 1;
                }
        }
        // each chunk of the pipeline order on its own
        const size_t nw = wins.size();
        const size_t cuts[4] = {0, nw / 16, nw / 4, nw};
        for (int c = 0; c < 3; ++c) {
            std::vector<Window> part(wins.begin() + (long)cuts[c], wins.begin() + (long)cuts[c + 1]);
            long long te = 0;
            if (!check_graph(n, part, withQ, withZ, cm, &te)) return 1;
        }
    }
    long long edges = 0;
    if (!check_graph(n, wins, withQ, withZ, cm, &edges)) return 1;
    printf("OK %lld\n", edges);
    return 0;
}

