// Internal definitions shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace gbr {

// Largest diagonal window whose packed upper-Hessenberg S window and dense
// accumulator U both fit in one CTA's shared memory.
constexpr int WMAX = 128;

// Wide windows, WMAX < w <= WMAX_WIDE: the window task keeps its packed S
// window in a per-CTA global scratch area (WIDE_SP_STRIDE doubles per CTA)
// and forms U in place in the U pool; both stay in the SM's L1 and in L2.
constexpr int WMAX_WIDE = 256;
constexpr size_t WIDE_SP_STRIDE = ((size_t)(WMAX_WIDE * (WMAX_WIDE + 3)) / 2 + 31) & ~(size_t)31;

// Split-precision (Ozaki) updates: OZ_SLICES signed 8-bit digit slices per
// FP64 operand; one window's U slices take OZ_USLICE_BYTES (bf16 digits
// [slice][column n][row k], then one int exponent per column).
constexpr int OZ_SLICES = 7;
constexpr size_t OZ_UDIG_ELEMS = (size_t)OZ_SLICES * WMAX * WMAX;
constexpr size_t OZ_USLICE_BYTES = OZ_UDIG_ELEMS * 2 + (size_t)WMAX * 4;

// Panel rows per update tile (update_body.cuh, scheduler tasks): tiles near
// a window (within UPD_NEAR rows or columns) are UPD_BM rows, the others
// UPD_FAR rows, processed by one task as UPD_FAR / UPD_BM tiles of UPD_BM.
constexpr int UPD_BM = 64;
constexpr int UPD_FAR = 256;
constexpr int UPD_NEAR = 256;

// Column-major element access.
__host__ __device__ inline size_t cm(int i, int j, int ld) {
    return (size_t)j * (size_t)ld + (size_t)i;
}

// Per-position selection state kept on the device during a reorder.
enum : uint8_t { SEL_NO = 0, SEL_YES = 1, SEL_STUCK = 2 };

// Device-side counters, one set per call.
struct DevCounters {
    unsigned long long swaps;
    unsigned long long rejected;
    int bad_column;      // validation: first column violating the standard form, or INT_MAX
    int step_overflow;   // windows that hit the step cap (a logic error if nonzero)
    unsigned long long win_flops;  // FP64 flops of in-window updates of accepted swaps
    unsigned long long upd_issued; // flops issued by the DMMA update tiles (zero rows of U skipped)
    int aborted;         // on_reject = ABORT: set by the window task that rejected a swap
    int pad;
};

// One reordering problem on the device: a scheduler launch may carry many.
struct Inst {
    double* S;
    double* Q;           // null: no Schur vectors
    uint8_t* sel;        // SEL_* per position
    DevCounters* ctr;
    int n, ldS, ldQ, pad;
    double* T;           // generalized form (S, T): T, else null
    double* Z;           // generalized form: right factor Z, or null
    int ldT, ldZ;
    const double* sp;    // bulge-chasing sweep (S holds H): (s, p) per bulge, else null
};

// One diagonal window in program order.
struct Window {
    int s, e;            // rows/cols [s, e) of S
    int chain;           // chain index (within its instance)
    int inst;            // instance index (scheduler launches)
    long long u_off;     // offset (in doubles) of this window's U in the U pool
    int t0, t1, b0, nb;  // bulge-chasing sweep: chain steps [t0, t1) of bulges [b0, b0 + nb)
};

// Persistent scheduler (sched.cu): task kinds and launch parameters.
enum : int { TASK_W = 0, TASK_L = 1, TASK_R = 2, TASK_Q = 3,  // L/R/Q = TASK_L + panel
             TASK_E = 4,    // server: eigenvalues + completion of a request (its last task)
             TASK_Z = 5 };  // generalized form: a tile of Z's panel (Z <- Z UZ)

struct SchedTask {
    int kind;   // TASK_*
    int win;    // window index
    int y0;     // first panel row of an update tile
    int rows;   // panel rows of an update tile
};

struct SchedParams {
    int strong, ntasks;
    int mode;                 // 0: reordering, 1: generalized (S, T) with Q and Z,
                              // 2: bulge-chasing sweep (window tasks chase bulges),
                              // 3: reordering with windows wider than WMAX
    const Inst* inst;         // instance table
    const SchedTask* tasks;   // queue order
    const Window* wins;
    int* deps_left;           // unfinished predecessors per task
    const int* succ_off;      // CSR successors
    const int* succ;
    double* upool;            // U of every window, at Window::u_off (w x w, column-major;
                              // a generalized instance's window has UQ then UZ there)
    unsigned char* uslices;   // null (FP64 updates) or OZ_USLICE_BYTES per window
    int fp64_fma;             // FP64 updates: 1 = DFMA register tiles, 0 = DMMA tiles
    int* abort_word;          // on_reject = ABORT: set at the first rejected swap, else null
    int* wskip;               // ABORT: per window, 1 if its task did nothing (tiles skip)
    int* head;                // next queue position
    int* err;                 // nonzero: a wait ran out (1) or the plan does not fit S (2)
    long long wait_limit_ns;  // a dependency wait gives up after this long (%globaltimer)
    unsigned long long* trace;  // null, or 4 words per queue position:
                                // smid | wait start | exec start | end (ns)
    double* wscr;             // mode 3: WIDE_SP_STRIDE doubles per CTA (packed S window)
};

// Server kernel (sched.cu): a ring of (request slot, local task) entries and
// a table of requests, all in device memory written by the host.
struct RingEntry {
    int req;     // request slot
    int local;   // task index in the request's queue order
};

struct SrvReq {
    Inst inst;                  // S, Q, selection, counters, sizes
    const SchedTask* tasks;     // queue order; the last one is TASK_E
    const Window* wins;         // u_off: offset of the window's U in upool
    int* deps;                  // unfinished predecessors per task
    const int* succ_off;        // CSR successors (local indices)
    const int* succ;
    double* upool;
    unsigned char* uslices;     // null, or OZ_USLICE_BYTES per window
    double* eig;                // 2n: real parts, imaginary parts
    int ntasks;
    int id;                     // unique per admitted pass (written to the completion word)
    int done_slot;              // completion word index
    int pad;
};

struct SrvParams {
    const RingEntry* ring;
    long long cap;              // ring entries
    long long* head;            // next position to take
    const long long* tail;      // positions below are published
    const int* stop;            // nonzero: leave when idle
    int* err;                   // 1: a dependency wait ran out; 3: the ring stayed empty too long
    const SrvReq* reqs;
    int* done;                  // completion words (host memory, mapped)
    int strong;
    int ozaki;                  // nonzero: split-precision updates (tensor memory held)
    int fp64_fma;               // FP64 updates: 1 = DFMA register tiles, 0 = DMMA tiles
    long long wait_limit_ns;    // a dependency wait gives up after this long (%globaltimer)
    long long park_limit_ns;    // a wait for the ring to fill gives up after this long
};

// Launchers (each .cu file owns its kernels).
cudaError_t launch_validate(int n, const double* S, int ldS, DevCounters* ctr, cudaStream_t st);
cudaError_t launch_subdiag(int n, const double* S, int ldS, uint8_t* sub, cudaStream_t st);
cudaError_t launch_eigs(int n, const double* S, int ldS, double* wr, double* wi, cudaStream_t st);
cudaError_t launch_window(int n, const Window& w, double* S, int ldS, uint8_t* sel, double* U,
                          int strong, DevCounters* ctr, cudaStream_t st, bool abort = false);
cudaError_t launch_update(int n, const Window& w, double* S, int ldS, double* Q, int ldQ,
                          const double* U, DevCounters* ctr, cudaStream_t st, bool fma = false);
size_t window_smem_bytes(int w);
size_t update_smem_bytes(int w);
cudaError_t launch_sched(const SchedParams& P, int grid, cudaStream_t st);
cudaError_t sched_configure();  // kernel attributes for the current device (once)
cudaError_t launch_server(const SrvParams& P, int grid, cudaStream_t st);
// Batched scans over an instance table: validation (bad_column per instance),
// the subdiagonal pattern (sub + off[i], or a comparison with it that sets
// *mismatch), and eigenvalues (wr/wi + off[i]).
cudaError_t launch_validate_batched(int count, const Inst* inst, cudaStream_t st);
cudaError_t launch_subdiag_batched(int count, const Inst* inst, const long long* off,
                                   uint8_t* sub, int* mismatch, cudaStream_t st);
cudaError_t launch_eigs_batched(int count, const Inst* inst, const long long* off, double* wr,
                                double* wi, cudaStream_t st);
size_t sched_smem_bytes();
int sched_threads();
// One panel update Y <- Y U (panel.cu): element (r, k) of Y at Y[r rs + k ks]
// with rs == 1 or ks == 1; Ug is w x w column-major (ld w).  The split-
// precision launch writes U's digit slices to us (OZ_USLICE_BYTES) first and
// sets *err if a tile's bounded wait runs out.
cudaError_t launch_panel_dmma(int rows, int w, double* Y, long long rs, long long ks,
                              const double* Ug, cudaStream_t st, bool fma = false);
cudaError_t launch_panel_ozaki(int rows, int w, double* Y, long long rs, long long ks,
                               const double* Ug, unsigned char* us, int* err, int grid,
                               cudaStream_t st);
// Eigenvectors (eigvec.cu).  blocks: (j, nb, output column, -) per selected
// diagonal block, the nreal 1x1 blocks first; rscratch: 3 n doubles per CTA
// of the launch when eigvec_rhs_smem(n) == 0, else unused.
size_t eigvec_rhs_smem(int n);
cudaError_t launch_colmax(int n, const double* S, int ldS, double* cmA, double* cmB,
                          cudaStream_t st);
cudaError_t launch_eigvec(int n, const double* S, int ldS, const int4* d_blocks, int nblk,
                          int nreal, double* Y, int ldY, double* cmA, double* cmB,
                          double* rscratch, int* nscale, cudaStream_t st);
cudaError_t launch_evgemm(int rows, int cols, const double* A, int ldA, const double* B, int ldB,
                          double* C, int ldC, const int* d_kmax, cudaStream_t st);
int evgemm_col_block();
cudaError_t launch_evnorm(int n, const int4* d_blocks, int nblk, double* X, int ldX, cudaStream_t st);

}  // namespace gbr
