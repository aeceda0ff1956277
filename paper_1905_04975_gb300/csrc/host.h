// Host-side internals shared by the entry points (api.cu, batch.cu,
// server.cu): error reporting, the window planner, the task graph and the
// persistent-scheduler launch image.
#pragma once

#include "../../include/gbreorder.h"
#include "common.cuh"

#include <nvtx3/nvToolsExt.h>

#include <functional>
#include <mutex>
#include <string>
#include <vector>

namespace gbr {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_last_error(const std::string& s);
const char* last_error_cstr();
int cuda_fail(cudaError_t e, const char* what);
// GBR_ERR_CAPTURING if st is being captured into a CUDA graph (or is the
// legacy stream while another stream captures), else 0.  Touches nothing on
// st; the error a refused query leaves behind is cleared.
int refuse_capture(cudaStream_t st);

#define GBR_CK(call, what)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::gbr::cuda_fail(e_, what); \
    } while (0)

int num_sms();

// Device scratch pool (api.cu): one grow-only allocation per device and slot;
// callers hold api_mutex() while they use it.
constexpr int POOL_GEN_SCRATCH = 6, POOL_GEN_HOST = 7, POOL_GEN_SCHED = 8, POOL_SWEEP = 9,
              POOL_SWEEP_SCHED = 10, POOL_SCHED_ALT = 11, POOL_GEN_SCHED_ALT = 12,
              POOL_NSLOTS = 13;
int pool_get(int slot, size_t bytes, void** out);
std::mutex& api_mutex();

// A named range of the call's host timeline for profilers (NVTX; costs
// nothing when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// CUDA events around the copies of the host-buffer entry points when
// opts.timing is set: [0, 1] bracket the host-to-device copies, [2, 3] the
// device-to-host copies.  report() runs after the stream has synchronized.
struct CopyTimer {
    cudaEvent_t ev[4] = {};
    bool on = false;
    explicit CopyTimer(bool timing) : on(timing) {
        for (int i = 0; on && i < 4; ++i)
            if (cudaEventCreate(&ev[i]) != cudaSuccess) on = false;
    }
    ~CopyTimer() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
    CopyTimer(const CopyTimer&) = delete;
    CopyTimer& operator=(const CopyTimer&) = delete;
    void mark(int i, cudaStream_t st) {
        if (on && cudaEventRecord(ev[i], st) != cudaSuccess) on = false;
    }
    void report(gbr_stats* s) const {
        if (!on || !s) return;
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, ev[0], ev[1]) == cudaSuccess) s->ms_h2d = a;
        if (cudaEventElapsedTime(&b, ev[2], ev[3]) == cudaSuccess) s->ms_d2h = b;
    }
};

// ---------------------------------------------------------------------------
// Planner (Section 3.2: windows and chains)
// ---------------------------------------------------------------------------
struct PlanState {
    int n = 0;
    std::vector<uint8_t> bsz;  // size of the block starting at a position, else 0
    std::vector<uint8_t> sel;  // SEL_* per position (uniform inside a block)
};

void init_state(PlanState& st, int n, const uint8_t* sub, const uint8_t* sel);
void sim_window(PlanState& st, int s, int e);
void plan_pass(PlanState& st, int w, int m, std::vector<Window>& win, int& nchains);
// Per-position selection from the caller's per-eigenvalue flags (a 2x2 block
// is selected if either row is); returns the number of selected positions.
int selection_positions(int n, const uint8_t* sub, const int* select, uint8_t* sel);
// Update flops of a window list: 2 w^2 (panel rows of L, R and Q).
double update_flops(int n, const std::vector<Window>& win, bool withQ);

// Bulge-chasing sweep (sweep.cu): one window of a chain of bulges [b0, b0 + nb)
// over rows / columns [s, e), running chain steps [t0, t1).
struct SweepWin {
    int s, e, t0, t1, b0, nb;
};
int plan_sweep(int n, int nbulges, int w, int nbc, std::vector<SweepWin>& out);

// ---------------------------------------------------------------------------
// Task graph and queue order (Section 3.2, Fig. 2)
// ---------------------------------------------------------------------------
struct Rect {
    int r0, r1, c0, c1;  // rows [r0, r1) x columns [c0, c1)
};

struct HostTask {
    int kind, win, y0, rows, mat;  // mat 0 = S (and T), 1 = Q, 2 = Z
    Rect rc;
    double dur;                     // estimated duration (microseconds)
};

struct TaskGraph {
    std::vector<HostTask> t;
    std::vector<int> ndeps;
    std::vector<int> soff, succ;    // CSR successors, program order
};

// Duration model of the queue order (microseconds).
struct CostModel {
    double win_us_128 = 2600.0;  // window task at w = 128 (scales as w^2)
    double tile_rate = 6900.0;   // update flops per microsecond of one SM
    double task_us = 2.0;        // fixed cost per update task
    double lr_mats = 1.0;        // matrices a left/right tile updates (2 for (S, T))
};

int far_rows(int n);
void pipeline_order(int n, std::vector<Window>& wins);
// far: panel rows of the update tiles away from the window (0: far_rows(n));
// threads: host threads for the dependence search.
void build_graph(int n, const std::vector<Window>& wins, bool withQ, const CostModel& cm,
                 TaskGraph& G, int far = 0, int threads = 1, bool withZ = false);
void queue_order(const TaskGraph& G, int P, std::vector<int>& order, double* cp_us = nullptr,
                 double* sim_us = nullptr);

// ---------------------------------------------------------------------------
// Persistent-scheduler launch over one or more instances
// ---------------------------------------------------------------------------
struct InstPlan {
    Inst d;                    // device pointers and sizes
    std::vector<Window> wins;  // planner order (pipeline order is applied here)
    int far = 0;               // far update-tile rows (0: far_rows(n))
    bool in_pipeline_order = false;  // wins is already a part of a pipeline order
};

struct SchedInfo {
    long long tasks = 0;
    double cp_us = 0.0, sim_us = 0.0, graph_ms = 0.0, order_ms = 0.0;
};

// Device image of a scheduler launch: prepared once, launched one or more
// times (each launch restores the dependency counters from deps_init).
struct SchedLaunch {
    SchedParams P{};
    int grid = 0;
    int* deps_init = nullptr;
    int* ctl = nullptr;               // head, err (and spare words), 256 bytes
    size_t trace_bytes = 0;
    std::vector<SchedTask> tq;        // host copy of the queue (trace decoding)
};

// Plans the task graph of all instances, orders it for `grid` CTAs, and
// uploads it into device memory obtained from alloc(bytes) (which must
// return 256-byte aligned memory that outlives the launches, or null).
int sched_prepare(std::vector<InstPlan>& plans, const gbr_opts& o, const CostModel& cm, int grid,
                  const std::function<void*(size_t)>& alloc, SchedLaunch* L, SchedInfo* info,
                  cudaStream_t st);
// Enqueues one launch: dependency counters restored, control words reset,
// then pre(st) if given (it may set *P.err to stop the launch early), then
// the kernel.  Only stream operations: capturable into a CUDA graph.
int sched_enqueue(const SchedLaunch& L, cudaStream_t st,
                  const std::function<int(cudaStream_t)>& pre = nullptr);
// Keeps the per-task timeline of a finished traced launch (opts.timing = 2)
// for gbr_last_trace.
int store_trace(const SchedLaunch& L);

// One planned pass of one instance through the persistent scheduler (api.cu).
// The windows are put in pipeline order; a large pass is cut into chunks
// that run as consecutive launches, each planned and uploaded while the
// previous one runs, from two launch images that alternate between the pool
// slots slot[0] and slot[1].
struct PassLaunch {
    Inst inst;                 // the instance (T and Z set for a pair)
    CostModel cm;              // duration model of the queue order
    int slot[2];               // pool slots of the two launch images
    int mode = -1;             // scheduler instance forced after planning (-1: as planned)
    const char* timeout_msg;   // message of GBR_ERR_TIMEOUT
};
// Adds the tasks, the launches and (with opts.timing) the launches' device
// time to the outputs; *info receives the chunks' planning figures summed.
int run_pass_persistent(const std::vector<Window>& wins, const PassLaunch& pl, const gbr_opts& o,
                        long long* ntasks_out, double* ms_out, long long* launches_out,
                        SchedInfo* info, cudaStream_t st);

}  // namespace gbr
