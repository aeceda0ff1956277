// Persistent device scheduler for the window and update tasks (Section 3.2,
// Fig. 2: window tasks W and right/left update tasks, executed in a
// sequentially consistent order without global synchronization, with several
// windows in flight).  One launch may carry the tasks of many independent
// reordering problems (an instance table; each window names its instance).
//
// One CTA per SM loops over a task queue that the host has put in a
// critical-path-first order.  Each task is either a window task (one diagonal
// window, window_body) or an update tile (BM rows of one window's left, right
// or Q panel, update_tile).  A task waits until its predecessors -- the
// earlier tasks whose exact row/column rectangles overlap its own -- have
// finished: a per-task counter of unfinished predecessors, decremented by
// each predecessor on completion.  Tasks are taken strictly in queue order
// and every predecessor sits earlier in the queue, so a waiting CTA only ever
// waits on tasks already taken by running CTAs: no deadlock, no co-residency
// requirement.  Every wait is bounded; a wait that runs out sets an error
// flag, and all CTAs leave the loop at their next check.
#include "update_body.cuh"
#include "window_body.cuh"

namespace gbr {

namespace {

constexpr int SCHED_THREADS = win::WIN_THREADS;
constexpr size_t kMax2(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSchedSmem = kMax2(kMax2(win::kWindowSmem, upd::kUpdateSmem), oz::kSmem);

__device__ __forceinline__ int ld_volatile(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__global__ void __launch_bounds__(SCHED_THREADS, 1)
sched_kernel(SchedParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int task_id, u_win;
    const int tid = threadIdx.x;
    if (tid == 0) u_win = -1;
    for (;;) {
        if (tid == 0) {
            int t = atomicAdd(P.head, 1);
            if (P.trace && t < P.ntasks) {
                P.trace[4 * t + 0] = smid();
                P.trace[4 * t + 1] = global_ns();
            }
            if (t < P.ntasks) {
                long long spins = 0;
                while (ld_volatile(&P.deps_left[t]) > 0) {
                    if (ld_volatile(P.err) != 0) { t = -1; break; }
                    if (++spins > P.wait_limit) {
                        atomicExch(P.err, 1);
                        t = -1;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            if (t >= 0 && ld_volatile(P.err) != 0) t = -1;
            task_id = t;
        }
        __syncthreads();
        const int t = task_id;
        if (t < 0 || t >= P.ntasks) break;
        __threadfence();
        if (P.trace && tid == 0) P.trace[4 * t + 2] = global_ns();
        const SchedTask tk = P.tasks[t];
        const Window wd = P.wins[tk.win];
        const Inst I = P.inst[wd.inst];
        double* Ug = P.upool + wd.u_off;
        if (tk.kind == TASK_W) {
            win::window_body(I.n, I.S, I.ldS, wd.s, wd.e - wd.s, I.sel, Ug, P.strong, I.ctr,
                             smem_raw,
                             P.uslices ? P.uslices + (size_t)tk.win * OZ_USLICE_BYTES : nullptr);
            if (tid == 0) u_win = -1;  // shared memory no longer holds a U
        } else {
            double* base;
            long long rs, ks;
            int R;
            upd::panel_geom(tk.kind - TASK_L, I.n, wd.s, wd.e, I.S, I.ldS, I.Q, I.ldQ, &base, &rs,
                            &ks, &R);
            bool load_u = (u_win != tk.win);
            __syncthreads();
            if (P.uslices) {
                for (int r = 0; r < tk.rows; r += UPD_FAR)
                    upd::update_tile_ozaki(base, rs, ks, tk.y0 + r, min(UPD_FAR, tk.rows - r),
                                           wd.e - wd.s, P.uslices + (size_t)tk.win * OZ_USLICE_BYTES,
                                           P.ozscratch + (size_t)blockIdx.x * UPD_FAR * WMAX,
                                           smem_raw);
                load_u = true;  // shared memory no longer holds U
            } else
            for (int r = 0; r < tk.rows; r += upd::BM) {
                upd::update_tile(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r), wd.e - wd.s, Ug,
                                 load_u, smem_raw);
                load_u = false;
            }
            if (tid == 0) u_win = P.uslices ? -1 : tk.win;
        }
        // release: every thread's writes are ordered before the counters drop
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (P.trace) P.trace[4 * t + 3] = global_ns();
            for (int i = P.succ_off[t]; i < P.succ_off[t + 1]; ++i)
                atomicSub(&P.deps_left[P.succ[i]], 1);
        }
    }
}

}  // namespace

size_t sched_smem_bytes() { return kSchedSmem; }
int sched_threads() { return SCHED_THREADS; }

cudaError_t sched_configure() {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && configured[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(sched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSchedSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) configured[dev] = true;
    return e;
}

cudaError_t launch_sched(const SchedParams& P, int grid, cudaStream_t st) {
    cudaError_t e = sched_configure();
    if (e != cudaSuccess) return e;
    sched_kernel<<<grid, SCHED_THREADS, kSchedSmem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace gbr
