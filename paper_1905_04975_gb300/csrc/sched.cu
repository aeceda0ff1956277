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
#include "scan_body.cuh"
#include "gen_body.cuh"
#include "ozaki.cuh"
#include "sweep_body.cuh"
#include "update_body.cuh"
#include "window_body.cuh"

namespace gbr {

namespace {

constexpr int SCHED_THREADS = win::WIN_THREADS;
constexpr size_t kMax2(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSchedSmem = kMax2(kMax2(win::kWindowSmem, upd::kUpdateSmem), oz::kSmem);
// the generalized (pair) and the sweep instances of the kernel
constexpr size_t kSchedSmemPair = kMax2(kMax2(gen::kGenWindowSmem, upd::kUpdateSmem), oz::kSmem);
constexpr size_t kSchedSmemSweep = kMax2(swp::kSweepSmem, upd::kUpdateSmem);
constexpr size_t kSchedSmemWide = kMax2(win::kWindowSmemWide, upd::kUpdateSmemWide);

__device__ __forceinline__ int ld_volatile(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Deadline of a bounded wait that starts now: limit_ns of %globaltimer time.
// The spin cap is a backstop only (every poll is an L2 round trip of well
// over 16 ns), so that a stopped timer could not make a wait endless.
struct WaitBound {
    unsigned long long deadline;
    long long spins, max_spins;
    __device__ __forceinline__ explicit WaitBound(long long limit_ns);
    // true once the wait has run out
    __device__ __forceinline__ bool expired();
};

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ WaitBound::WaitBound(long long limit_ns)
    : deadline(global_ns() + (unsigned long long)limit_ns), spins(0),
      max_spins(limit_ns / 16 + 1) {}

__device__ __forceinline__ bool WaitBound::expired() {
    return ++spins > max_spins || global_ns() > deadline;
}

// Runs one window task or update task of window wd of instance I.  u_key
// names the U held in shared memory by the previous task of this CTA (an
// update tile of the same window reuses it); key names this task's window.
// Split-precision tiles run on the tensor cores with the CTA's tensor memory
// (tmem); if one of their bounded waits runs out, *err is set.  MODE 1: the
// instance is a generalized form (S, T); MODE 2: a bulge-chasing sweep on
// the Hessenberg matrix in I.S (each its own kernel instance, so that the
// reordering's code and register allocation are untouched); MODE 3: a
// reordering with windows wider than WMAX (window tasks keep the packed S
// window in gsp, this CTA's global scratch; tiles read U from global memory).
template <int MODE>
__device__ __forceinline__ void run_task(const SchedTask& tk, const Window& wd, const Inst& I,
                                         double* Ug, unsigned char* uslices,
                                         int strong, unsigned long long key,
                                         unsigned long long* u_key, unsigned char* smem_raw,
                                         uint32_t tmem, int* err, bool fma,
                                         int* abort_word = nullptr, int* wskip = nullptr,
                                         double* gsp = nullptr) {
    const int tid = threadIdx.x;
    const int w = wd.e - wd.s;
    // ABORT: the update tasks of a window whose task did nothing do nothing
    // (its U was never formed); the window task ran before them (a predecessor)
    if (wskip && tk.kind != TASK_W && __ldcg(wskip) != 0) return;
    if (tk.kind == TASK_W) {
        if constexpr (MODE == 1) {
            gen::window_gen_body(I.n, I.S, I.ldS, I.T, I.ldT, wd.s, w, I.sel, Ug, Ug + w * w, strong,
                                 I.ctr, smem_raw);
            if (uslices) {
                // split precision: digit slices of UQ, then of UZ (from the
                // factors the task just wrote; the barrier orders the reads)
                __syncthreads();
                win::write_u_slices(Ug, w, uslices);
                __syncthreads();
                win::write_u_slices(Ug + w * w, w, uslices + OZ_USLICE_BYTES);
            }
        } else if constexpr (MODE == 2)
            swp::sweep_body(I.n, I.S, I.ldS, wd.s, w, wd.t0, wd.t1, wd.nb, I.sp + 2 * wd.b0, Ug,
                            I.ctr, smem_raw);
        else if constexpr (MODE == 3)
            win::window_body_t<WMAX_WIDE>(I.n, I.S, I.ldS, wd.s, w, I.sel, Ug, strong, I.ctr,
                                          smem_raw, nullptr, abort_word, wskip, gsp);
        else
            win::window_body(I.n, I.S, I.ldS, wd.s, w, I.sel, Ug, strong, I.ctr, smem_raw, uslices,
                             abort_word, wskip);
        if (tid == 0) *u_key = ~0ull;  // shared memory no longer holds a U
        return;
    }
    if constexpr (MODE == 1) {
        // generalized form: left tiles of S and T by UQ, right tiles of S and
        // T by UZ, Q by UQ, Z by UZ (UQ then UZ at the window's U offset)
        const bool byZ = (tk.kind == TASK_R || tk.kind == TASK_Z);
        const double* U = byZ ? Ug + w * w : Ug;
        const unsigned long long k2 = (key << 1) | (byZ ? 1ull : 0ull);
        bool load_u = (*u_key != k2);
        __syncthreads();
        const int nm = (tk.kind == TASK_L || tk.kind == TASK_R) ? 2 : 1;
        for (int mi = 0; mi < nm; ++mi) {
            double* base;
            long long rs, ks;
            int R;
            const int panel = tk.kind == TASK_Z ? upd::PANEL_Q : tk.kind - TASK_L;
            double* X = mi ? I.T : I.S;
            const int ldX = mi ? I.ldT : I.ldS;
            upd::panel_geom(panel, I.n, wd.s, wd.e, X, ldX, tk.kind == TASK_Z ? I.Z : I.Q,
                            tk.kind == TASK_Z ? I.ldZ : I.ldQ, &base, &rs, &ks, &R);
            if (uslices) {
                // split precision on the tensor cores (the slices of UQ or UZ)
                if (!oz::update_tile_tc(base, rs, ks, tk.y0, tk.rows, w,
                                        uslices + (byZ ? OZ_USLICE_BYTES : 0), smem_raw, tmem) &&
                    tid == 0)
                    atomicExch(err, 1);
                __syncthreads();
                continue;
            }
            for (int r = 0; r < tk.rows; r += upd::BM) {
                if (fma)
                    upd::update_tile_fma(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r), w, U,
                                         load_u, smem_raw, &I.ctr->upd_issued);
                else
                    upd::update_tile(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r), w, U,
                                     load_u, smem_raw, &I.ctr->upd_issued);
                load_u = false;
            }
        }
        if (tid == 0) *u_key = uslices ? ~0ull : k2;
        return;
    }
    double* base;
    long long rs, ks;
    int R;
    upd::panel_geom(tk.kind - TASK_L, I.n, wd.s, wd.e, I.S, I.ldS, I.Q, I.ldQ, &base, &rs, &ks, &R);
    bool load_u = (*u_key != key);
    __syncthreads();
    if constexpr (MODE == 3) {
        // wide window: FP64 tiles only, U read from global memory
        for (int r = 0; r < tk.rows; r += upd::BM) {
            if (fma)
                upd::update_tile_fma<true>(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r), w,
                                           Ug, load_u, smem_raw, &I.ctr->upd_issued);
            else
                upd::update_tile<true>(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r), w, Ug,
                                       load_u, smem_raw, &I.ctr->upd_issued);
            load_u = false;
        }
        if (tid == 0) *u_key = key;
        return;
    }
    if (uslices) {
        if (!oz::update_tile_tc(base, rs, ks, tk.y0, tk.rows, wd.e - wd.s, uslices, smem_raw, tmem) &&
            tid == 0)
            atomicExch(err, 1);
        if (tid == 0) *u_key = ~0ull;  // shared memory no longer holds U
    } else {
        for (int r = 0; r < tk.rows; r += upd::BM) {
            if (fma)
                upd::update_tile_fma(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r),
                                     wd.e - wd.s, Ug, load_u, smem_raw, &I.ctr->upd_issued);
            else
                upd::update_tile(base, rs, ks, tk.y0 + r, min(upd::BM, tk.rows - r), wd.e - wd.s,
                                 Ug, load_u, smem_raw, &I.ctr->upd_issued);
            load_u = false;
        }
        if (tid == 0) *u_key = key;
    }
}

// Tensor memory for the split-precision tiles: one warp allocates all
// oz::TMEM_COLS columns at the start of a persistent launch (one CTA per SM,
// so the allocation never waits) and frees them when the CTA leaves.
__device__ __forceinline__ uint32_t tmem_acquire(bool need, uint32_t* slot) {
    if (!need) return 0u;
    if ((threadIdx.x >> 5) == 0) oz::tmem_alloc(slot, oz::TMEM_COLS);
    oz::tc_fence_before();
    __syncthreads();
    oz::tc_fence_after();
    return *slot;
}
__device__ __forceinline__ void tmem_release(bool need, uint32_t tmem) {
    if (!need) return;
    oz::tc_fence_before();
    __syncthreads();
    oz::tc_fence_after();
    if ((threadIdx.x >> 5) == 0) oz::tmem_dealloc(tmem, oz::TMEM_COLS);
}

template <int MODE>
__global__ void __launch_bounds__(SCHED_THREADS, 1)
sched_kernel(SchedParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int task_id;
    __shared__ unsigned long long u_key;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x;
    if (tid == 0) u_key = ~0ull;
    const bool oz = P.uslices != nullptr;
    const uint32_t tmem = tmem_acquire(oz, &tmem_slot);
    for (;;) {
        if (tid == 0) {
            int t = atomicAdd(P.head, 1);
            if (P.trace && t < P.ntasks) {
                P.trace[4 * t + 0] = smid();
                P.trace[4 * t + 1] = global_ns();
            }
            if (t < P.ntasks && ld_volatile(&P.deps_left[t]) > 0) {
                WaitBound wb(P.wait_limit_ns);
                while (ld_volatile(&P.deps_left[t]) > 0) {
                    if (ld_volatile(P.err) != 0) { t = -1; break; }
                    if (wb.expired()) {
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
        run_task<MODE>(tk, wd, I, P.upool + wd.u_off,
                 P.uslices ? P.uslices + (size_t)tk.win * OZ_USLICE_BYTES * (MODE == 1 ? 2 : 1)
                           : nullptr,
                 P.strong, (unsigned long long)tk.win, &u_key, smem_raw, tmem, P.err,
                 P.fp64_fma != 0, P.abort_word, P.wskip ? P.wskip + tk.win : nullptr,
                 P.wscr ? P.wscr + (size_t)blockIdx.x * WIDE_SP_STRIDE : nullptr);
        // release: every thread's writes are ordered before the counters drop
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (P.trace) P.trace[4 * t + 3] = global_ns();
            for (int i = P.succ_off[t]; i < P.succ_off[t + 1]; ++i)
                atomicSub(&P.deps_left[P.succ[i]], 1);
        }
    }
    tmem_release(oz, tmem);
}

// ---------------------------------------------------------------------------
// Server kernel: one long-lived launch fed through a ring of (request, task)
// entries that the host appends while it runs.  Positions are taken in ring
// order; a position beyond the published tail is held until the host
// publishes it or sets the stop word.  A request's tasks appear in the ring
// in its own queue order, so every predecessor of a task sits at an earlier
// position and has been taken by a running CTA: waits end.  The last task of
// a request (TASK_E) depends on all others: it reads the eigenvalues off the
// final blocks and writes the request's completion word to host memory.
// Loads of host-written tables bypass L1 (their memory is reused).
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long ld_volatile64(const long long* p) {
    return *reinterpret_cast<const volatile long long*>(p);
}

__global__ void __launch_bounds__(SCHED_THREADS, 1)
server_kernel(SrvParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long pos_s;
    __shared__ RingEntry ent_s;
    __shared__ unsigned long long u_key;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x;
    if (tid == 0) u_key = ~0ull;
    const bool oz = P.ozaki != 0;
    const uint32_t tmem = tmem_acquire(oz, &tmem_slot);
    for (;;) {
        if (tid == 0) {
            long long t = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(P.head), 1ull);
            // hold the position until it is published
            if (t >= ld_volatile64(P.tail)) {
              WaitBound park(P.park_limit_ns);
              while (t >= ld_volatile64(P.tail)) {
                if (ld_volatile(P.stop) != 0 || ld_volatile(P.err) != 0) { t = -1; break; }
                if (park.expired()) {
                    atomicExch(P.err, 3);
                    t = -1;
                    break;
                }
                __nanosleep(1024);
              }
            }
            RingEntry e{-1, -1};
            if (t >= 0) {
                const RingEntry* rp = P.ring + (t % P.cap);
                e.req = __ldcg(&rp->req);
                e.local = __ldcg(&rp->local);
                const int* deps = reinterpret_cast<const int*>(__ldcg(
                    reinterpret_cast<const unsigned long long*>(&P.reqs[e.req].deps)));
                WaitBound wb(P.wait_limit_ns);
                while (ld_volatile(&deps[e.local]) > 0) {
                    if (ld_volatile(P.err) != 0) { t = -1; break; }
                    if (wb.expired()) {
                        atomicExch(P.err, 1);
                        t = -1;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            pos_s = t;
            ent_s = e;
        }
        __syncthreads();
        if (pos_s < 0) break;
        __threadfence();
        const RingEntry e = ent_s;
        const SrvReq* Rg = P.reqs + e.req;
        SrvReq R;
        {
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(Rg);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(&R);
            for (int k = 0; k < (int)(sizeof(SrvReq) / 8); ++k) dst[k] = __ldcg(src + k);
        }
        SchedTask tk;
        {
            const int4 v = __ldcg(reinterpret_cast<const int4*>(R.tasks + e.local));
            tk = SchedTask{v.x, v.y, v.z, v.w};
        }
        if (tk.kind == TASK_E) {
            const Inst& I = R.inst;
            for (int i = tid; i < I.n; i += blockDim.x) {
                double re, im;
                eig_at(I.n, I.S, I.ldS, i, &re, &im);
                R.eig[i] = re;
                R.eig[I.n + i] = im;
            }
        } else {
            Window wd;
            {
                const Window* wp = R.wins + tk.win;
                wd.s = __ldcg(&wp->s);
                wd.e = __ldcg(&wp->e);
                wd.chain = 0;
                wd.inst = 0;
                wd.u_off = __ldcg(&wp->u_off);
            }
            run_task<0>(tk, wd, R.inst, R.upool + wd.u_off,
                     R.uslices ? R.uslices + (size_t)tk.win * OZ_USLICE_BYTES : nullptr,
                     P.strong, ((unsigned long long)(unsigned)R.id << 32) | (unsigned)tk.win, &u_key,
                     smem_raw, tmem, P.err, P.fp64_fma != 0);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (tk.kind == TASK_E) {
                __threadfence_system();
                *reinterpret_cast<volatile int*>(P.done + R.done_slot) = R.id;
                __threadfence_system();
            } else {
                const int* so = R.succ_off;
                const int a = __ldcg(&so[e.local]), b = __ldcg(&so[e.local + 1]);
                for (int i = a; i < b; ++i) atomicSub(&R.deps[__ldcg(&R.succ[i])], 1);
                atomicSub(&R.deps[R.ntasks - 1], 1);  // the request's final task
            }
        }
    }
    tmem_release(oz, tmem);
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
    e = cudaFuncSetAttribute(sched_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSchedSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sched_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSchedSmemPair);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sched_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSchedSmemSweep);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sched_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSchedSmemWide);
    if (e == cudaSuccess && dev >= 0 && dev < 64) configured[dev] = true;
    return e;
}

cudaError_t launch_server(const SrvParams& P, int grid, cudaStream_t st) {
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(server_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSchedSmem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    server_kernel<<<grid, SCHED_THREADS, kSchedSmem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_sched(const SchedParams& P, int grid, cudaStream_t st) {
    cudaError_t e = sched_configure();
    if (e != cudaSuccess) return e;
    if (P.mode == 1)
        sched_kernel<1><<<grid, SCHED_THREADS, kSchedSmemPair, st>>>(P);
    else if (P.mode == 2)
        sched_kernel<2><<<grid, SCHED_THREADS, kSchedSmemSweep, st>>>(P);
    else if (P.mode == 3)
        sched_kernel<3><<<grid, SCHED_THREADS, kSchedSmemWide, st>>>(P);
    else
        sched_kernel<0><<<grid, SCHED_THREADS, kSchedSmem, st>>>(P);
    return cudaGetLastError();
}

}  // namespace gbr
