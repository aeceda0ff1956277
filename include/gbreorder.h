/*
 * gbreorder -- eigenvalue reordering of a real Schur form on one GPU (sm_103a).
 *
 * The operation (Section 2, Eq. 7 of Myllykoski & Kjelgaard Mikkelsen,
 * "Introduction to StarNEig"): given S in standard real Schur form
 * (Eq. 4: upper quasi-triangular with 1x1 and 2x2 diagonal blocks, each
 * 2x2 block standardized as [[a, b], [c, a]] with bc < 0), an orthogonal Q
 * and a selection of eigenvalues, compute an orthogonal Q3 such that
 *
 *     S_hat = Q3^T S Q3
 *
 * is again in standard real Schur form with the selected eigenvalues in
 * its leading diagonal blocks; S is overwritten by S_hat and Q by Q Q3.
 * Selected blocks keep their relative order, and so do unselected ones.
 *
 * Method (Section 3.2): chains of adjacent block swaps are applied inside
 * small diagonal windows and accumulated into an orthogonal matrix U per
 * window (Fig. 1b); U is then applied to the rest of S and to Q as dense
 * matrix products (the left/right update tasks of Section 3.2), and the
 * windows of successive chains are pipelined.
 *
 * Conventions for every entry point:
 *   - matrices are column-major FP64 with a leading dimension (ld >= n),
 *     as in LAPACK/ScaLAPACK (Section 4.2);
 *   - `select` has one int per diagonal position; a 2x2 block is selected
 *     if either of its two positions is;
 *   - a non-NULL `cuda_stream` is a cudaStream_t; NULL means the legacy
 *     default stream;
 *   - calls are synchronous: they return after all GPU work has finished;
 *     so a call on a stream that is being captured into a CUDA graph is
 *     refused with GBR_ERR_CAPTURING before anything is enqueued (the
 *     capture stays valid);
 *   - the library never frees caller memory.  Its own scratch (window
 *     accumulators, block plan, counters) comes from a per-device pool the
 *     library owns, grown on demand and kept until gbr_release().
 *
 * Return value (int):
 *     0            success;
 *     k > 0        k block swaps were rejected by the stability test: the
 *                  reordering is partial, but S and Q are still an exact
 *                  orthogonal similarity in standard form (a rejected
 *                  block stays in place and later selected blocks stop
 *                  below it);
 *     -i (1..12)   argument i is invalid (e.g. -1: n < 0, -3: ldS < n,
 *                  -2: S is not in standard real Schur form);
 *     GBR_ERR_*    the negative codes below.
 */
#ifndef GBREORDER_H
#define GBREORDER_H

#ifdef __cplusplus
extern "C" {
#endif

#define GBR_ERR_CUDA    (-1001) /* a CUDA call failed (message: gbr_last_error) */
#define GBR_ERR_NOMEM   (-1002) /* device or host allocation failed */
#define GBR_ERR_TIMEOUT (-1003) /* a bounded device-side wait gave up; S and Q are
                                   then partially updated and must be discarded */
#define GBR_ERR_UNSUPPORTED (-1004) /* option value not supported */
#define GBR_ERR_NOALLOC_LIMIT (-1005) /* n > GBR_NOALLOC_MAX_N in gbr_reorder_noalloc */
#define GBR_ERR_PLAN_MISMATCH (-1006) /* gbr_batch_run: an S no longer has the block
                                         structure it was planned for; nothing was
                                         modified */
#define GBR_ERR_CAPTURING (-1007) /* cuda_stream is being captured into a CUDA graph
                                     (or is the legacy stream while another stream
                                     captures): the call synchronizes its stream and
                                     reads results back, which a capture refuses.
                                     Checked with cudaStreamIsCapturing before
                                     anything is enqueued: nothing was modified and
                                     the capture stays valid */

#define GBR_PREC_DMMA   0  /* off-diagonal updates on FP64 tensor cores (DMMA) */
#define GBR_PREC_OZAKI  1  /* off-diagonal updates as split-precision emulated FP64:
                              7 signed 8-bit digit slices per operand, 28 exact
                              bf16 tensor-core slice products, integer combination,
                              one rounding to double; the windows stay in FP64 */
#define GBR_PREC_FMA    2  /* off-diagonal updates in FP64 on the FP64 FMA pipe (DFMA
                              register tiles, no tensor cores); same arithmetic
                              type as GBR_PREC_DMMA, another instruction mix */

#define GBR_ON_REJECT_CONTINUE 0 /* a rejected block stays; later blocks stop below it */
#define GBR_ON_REJECT_ABORT    1 /* the first rejected swap stops the reordering: the
                                    window task that rejected it finishes its current
                                    step and restores the standard form of its 2x2
                                    blocks; window tasks that start later do nothing;
                                    tasks already running complete.  S and Q remain an
                                    exact orthogonal similarity, partially reordered
                                    (as LAPACK's dtrsen with info = 1); which blocks
                                    moved before the stop depends on the schedule.
                                    gbr_reorder, gbr_reorder_host and
                                    gbr_reorder_noalloc only */

/* Options; gbr_default_opts() fills the defaults shown. */
typedef struct gbr_opts {
    int window;        /* diagonal window size w, 4..256        (default 128);
                          above 128 (the window of S and its U no longer fit
                          in one SM's shared memory: the window task keeps
                          them in L1/L2-resident global memory) only with the
                          persistent schedule and FP64 updates (FMA or DMMA),
                          else GBR_ERR_UNSUPPORTED; gbr_reorder,
                          gbr_reorder_host and gbr_plan only (the other
                          entry points take 4..128).
                          GBR_AUTO in batched calls: chosen per instance by
                          the autotuner (gbr_autotune)                        */
    int chain;         /* selected eigenvalues per chain m, 1..w-2 (default 64);
                          GBR_AUTO with window = GBR_AUTO                     */
    int precision;     /* GBR_PREC_FMA (default: the faster FP64 path on this
                          GPU), GBR_PREC_DMMA or GBR_PREC_OZAKI (persistent
                          schedule only)                                      */
    int slices;        /* split-precision digit slices per operand: 0 (default)
                          or 7, the only count built: 7 balanced 8-bit digits
                          hold the 55-bit fixed-point form of every entry, so
                          the slices lose nothing of a binary64 significand
                          (fewer would drop its low bits, more add nothing);
                          any other value: GBR_ERR_UNSUPPORTED             */
    int strong_test;   /* 1: weak + strong stability test       (default 1)   */
    int on_reject;     /* GBR_ON_REJECT_CONTINUE (default) or GBR_ON_REJECT_ABORT */
    int validate;      /* 1: check the standard-form input      (default 1)   */
    int timing;        /* 1: time the kernels with CUDA events into gbr_stats;
                          2: also record a per-task timeline of the persistent
                          scheduler (gbr_last_trace)              (default 0)  */
    int sched;         /* GBR_SCHED_PERSISTENT (default) or GBR_SCHED_SEQUENTIAL */
    int inject;        /* fault injection for tests: GBR_INJECT_STALL makes one
                          scheduler task wait for a predecessor that never
                          finishes, so the bounded wait runs out (default 0) */
    long long wait_limit_ms; /* bound on any device-side wait of the persistent
                          scheduler, milliseconds; 0 = default (60000)   */
} gbr_opts;

#define GBR_AUTO 0 /* opts.window / opts.chain of batched calls: autotuned */

#define GBR_SCHED_PERSISTENT 0 /* one persistent launch runs all window and update
                                  tasks, several windows in flight (Section 3.2) */
#define GBR_SCHED_SEQUENTIAL 1 /* one window, then its update, at a time */
#define GBR_INJECT_STALL 1

/* Per-call statistics (all optional). */
typedef struct gbr_stats {
    long long swaps;      /* accepted block swaps                      */
    long long rejected;   /* rejected block swaps                      */
    long long windows;    /* diagonal windows processed                */
    long long chains;     /* window chains                             */
    long long launches;   /* kernels launched by the call              */
    double upd_flops;     /* flops of the off-diagonal updates         */
    double ms_total;      /* wall time of the call                     */
    double ms_window;     /* summed window-kernel time (opts.timing, sequential) */
    double ms_update;     /* summed update-kernel time (opts.timing, sequential) */
    double ms_sched;      /* persistent-scheduler kernel time (opts.timing)      */
    double win_flops;     /* FP64 flops of the in-window updates of accepted swaps */
    long long tasks;      /* scheduler tasks (window tasks + update tiles)       */
    double sched_cp_ms;   /* longest dependence path of the task graph under the
                             scheduler's duration model                          */
    double sched_sim_ms;  /* makespan of the scheduler's list-scheduling model   */
    double ms_graph;      /* host time building the task graph                   */
    double ms_order;      /* host time computing the queue order                 */
    double upd_flops_issued; /* flops the FP64 update tiles (FMA or DMMA) issued:
                             upd_flops less the products with the all-zero rows
                             of U each warp skips (0 for split precision)         */
    double ms_h2d;        /* host-buffer entry points with opts.timing: time of the
                             host-to-device copies of the call (CUDA events)     */
    double ms_d2h;        /* the same for the device-to-host copies              */
} gbr_stats;

/* Fill *opts with the defaults. */
void gbr_default_opts(gbr_opts *opts);

/*
 * Reorder a Schur form resident in device memory (Eq. 7).
 *
 *  1 n        order of S (n >= 0)
 *  2 S        device pointer, n x n column-major, overwritten by S_hat
 *  3 ldS      leading dimension of S, >= max(1, n)
 *  4 Q        device pointer or NULL; n x n column-major, overwritten by Q Q3
 *  5 ldQ      leading dimension of Q, >= max(1, n) when Q != NULL
 *  6 select   host pointer, n ints; nonzero selects the eigenvalue at that
 *             diagonal position
 *  7 eig_re   host pointer or NULL; n doubles: real parts of the
 *             eigenvalues of S_hat in diagonal order
 *  8 eig_im   host pointer or NULL; n doubles: imaginary parts (a
 *             conjugate pair gives +im first, then -im)
 *  9 m_out    host pointer or NULL; number of selected eigenvalues (the
 *             dimension of the leading invariant subspace when status 0)
 * 10 opts     options or NULL for the defaults
 * 11 stats    host pointer or NULL; filled with per-call statistics
 * 12 cuda_stream  cudaStream_t or NULL
 */
int gbr_reorder(int n, double *S, int ldS, double *Q, int ldQ, const int *select,
                double *eig_re, double *eig_im, int *m_out, const gbr_opts *opts,
                gbr_stats *stats, void *cuda_stream);

/*
 * Same operation with S and Q in HOST memory (pageable or pinned): the
 * call copies them to the device, reorders, and copies them back.  The
 * arguments mean what they mean for gbr_reorder, except that S and Q are
 * host pointers.  Device buffers come from the library's pool.
 */
int gbr_reorder_host(int n, double *S, int ldS, double *Q, int ldQ, const int *select,
                     double *eig_re, double *eig_im, int *m_out, const gbr_opts *opts,
                     gbr_stats *stats, void *cuda_stream);

/*
 * Reorder a generalized real Schur form (S, T) resident in device memory
 * (Section 2, Eq. 7, second form): orthogonal Q3, Z3 with
 * (S_hat, T_hat) = Q3^T (S, T) Z3 again in generalized real Schur form and
 * the selected generalized eigenvalues in its leading diagonal blocks.
 *
 * Input form: S upper quasi-triangular (1x1 and 2x2 diagonal blocks, a 2x2
 * block marked by S[j+1][j] != 0 and carrying a complex-conjugate pair of
 * the 2x2 pencil), T upper triangular (also inside the 2x2 blocks).  The
 * output keeps that form; the 2x2 blocks of S are not standardized further.
 *
 *  1 n          order (n >= 0)
 *  2 S, 3 ldS   device, n x n column-major, overwritten by S_hat
 *  4 T, 5 ldT   device, n x n column-major, overwritten by T_hat
 *  6 Q, 7 ldQ   device or NULL; overwritten by Q Q3
 *  8 Z, 9 ldZ   device or NULL; overwritten by Z Z3
 * 10 select     host, n ints, as for gbr_reorder
 * 11 eig_re, 12 eig_im  host or NULL: generalized eigenvalues lambda =
 *               alpha / beta of (S_hat, T_hat) in diagonal order (a 1x1
 *               block gives s/t, +-inf if t = 0; a 2x2 block its conjugate
 *               pair, +im first)
 * 13 m_out      host or NULL: number of selected eigenvalues
 * 14 opts       options or NULL for the defaults.  window > 64 is reduced
 *               to 64 and chain then to at most 32 (both factors of a window
 *               live in shared memory); both schedules; precision
 *               GBR_PREC_FMA or GBR_PREC_DMMA, or GBR_PREC_OZAKI on the
 *               persistent schedule (split-precision updates from the digit
 *               slices of UQ and UZ)
 * 15 stats      host or NULL (upd_flops counts S, T, Q and Z panels)
 * 16 cuda_stream  cudaStream_t or NULL
 *
 * Returns the number of rejected swaps (>= 0) or a negative error: -1 bad
 * n, -2 (S, T) not in generalized real Schur form (also a NULL S or T),
 * -3 bad ldS/ldT, -5 bad ldQ/ldZ, -6 NULL select, -10 bad window/chain.
 */
int gbr_reorder_gen(int n, double *S, int ldS, double *T, int ldT, double *Q, int ldQ,
                    double *Z, int ldZ, const int *select, double *eig_re, double *eig_im,
                    int *m_out, const gbr_opts *opts, gbr_stats *stats, void *cuda_stream);

/*
 * One bulge-chasing sweep of the Schur reduction on an upper Hessenberg H
 * resident in device memory (Section 3.2): one pipelined QR iteration, a
 * bulge per pair of shifts introduced at the top and chased to the bottom by
 * overlapping 3x3 Householder reflectors, H <- Q3^T H Q3, Q <- Q Q3.  At chain
 * step tau bulge j of a chain sits at k_j = tau - 3 j - 1; the introduction
 * uses the first column of (H - sigma1 I)(H - sigma2 I); a chase step maps
 * H[k+1..k+3, k] onto beta e_0 and leaves exact zeros below beta.
 *
 *  1 n            order (n >= 0; n < 3 or no shifts: nothing to do)
 *  2 H, 3 ldH     device, n x n column-major, upper Hessenberg (entries two
 *                 or more below the diagonal must be zero), overwritten
 *  4 Q, 5 ldQ     device or NULL; overwritten by Q Q3
 *  6 nshifts      even; 7 shift_re, 8 shift_im: host, the shifts; each pair
 *                 (2i, 2i+1) is two real shifts or a complex-conjugate pair
 *  9 opts         NULL for window 64 and 16 shifts per chain (otherwise the
 *                 gbr_default_opts values); window = window size (8 .. 128,
 *                 capped at 96), chain = shifts per chain of bulges (capped
 *                 at w / 3);
 *                 precision GBR_PREC_FMA or GBR_PREC_DMMA (FP64 updates);
 *                 validate checks the form
 * 10 stats        host or NULL (windows, chains, update and window flops,
 *                 kernel times with opts.timing)
 * 11 cuda_stream  cudaStream_t or NULL
 *
 * Returns 0, or -1 bad n, -2 NULL H or H not upper Hessenberg, -3 bad ldH,
 * -5 bad ldQ, -6 bad shifts (odd count, NULL, a pair neither real nor
 * conjugate), -10 bad options, GBR_ERR_UNSUPPORTED (split precision).
 */
int gbr_qr_sweep(int n, double *H, int ldH, double *Q, int ldQ, int nshifts,
                 const double *shift_re, const double *shift_im, const gbr_opts *opts,
                 gbr_stats *stats, void *cuda_stream);

/* gbr_reorder_gen with S, T, Q, Z in HOST memory (copied to the device and
 * back inside the call; device buffers from the library's pool). */
int gbr_reorder_gen_host(int n, double *S, int ldS, double *T, int ldT, double *Q, int ldQ,
                         double *Z, int ldZ, const int *select, double *eig_re,
                         double *eig_im, int *m_out, const gbr_opts *opts,
                         gbr_stats *stats, void *cuda_stream);

/*
 * Same operation as gbr_reorder, for callers that must not allocate device
 * memory: programs whose device memory is all handed out by their own arena
 * or allocator, and processes where a cudaMalloc (which may synchronize the
 * device) must not happen in the middle of their work.  The paper has no
 * counterpart: this is an interface convenience.
 *
 * Arguments and return values are those of gbr_reorder, plus
 * GBR_ERR_NOALLOC_LIMIT when n > GBR_NOALLOC_MAX_N (checked before anything
 * else is touched).  The call never calls cudaMalloc, cudaFree or any other
 * allocating routine, and creates no CUDA events (opts->timing is ignored).
 * It runs the window/update launch pairs (opts->sched is not used) with
 * FP64 updates, FMA or DMMA tiles as opts->precision says
 * (GBR_ERR_UNSUPPORTED for split precision and for windows above 128).  Like gbr_reorder it
 * synchronizes cuda_stream during the call (the planner reads the block
 * structure and the rejection counters back to the host between passes) and
 * returns after the stream work has completed.
 *
 * Its scratch is a fixed array of GBR_NOALLOC_SCRATCH_BYTES in device global
 * memory, part of the library image: every GPU that loads the library holds
 * it until the process exits, and each process (each CUDA context) has its
 * own copy.  Every call looks up the array's device address in the current
 * context (cudaGetSymbolAddress, with the device current).  All calls of one
 * process share the array, which keeps the previous call's contents (each
 * call re-initialises what must start at zero); the library serializes the
 * calls of one process (a lock held until the call's stream work has
 * completed), so they never overlap on the GPU.
 */
#define GBR_NOALLOC_MAX_N 16384
#define GBR_NOALLOC_SCRATCH_BYTES (256 + 2 * 16384 + 2 * 16384 * 8 + 128 * 128 * 8)
int gbr_reorder_noalloc(int n, double *S, int ldS, double *Q, int ldQ, const int *select,
                        double *eig_re, double *eig_im, int *m_out, const gbr_opts *opts,
                        gbr_stats *stats, void *cuda_stream);

/*
 * One off-diagonal update on one panel, in place:
 *
 *     Y <- Y U
 *
 * This is the level-3 step of Section 3.2 (Fig. 1b): the accumulated
 * orthogonal transformation U of a diagonal window applied to a section of
 * the matrix.  gbr_reorder runs it on three panels per window: the left
 * update S[win, right] <- U^T S[win, right] (Y = that block read
 * transposed, row-major: rs = ldS, ks = 1), the right update
 * S[above, win] <- S[above, win] U and the Q update Q[:, win] <- Q[:, win] U
 * (Y = the column-major block: rs = 1, ks = ld).  Exposed on its own so that
 * the update arithmetic can be used and checked separately.
 *
 *  1 rows       panel rows (>= 0; 0 is a no-op)
 *  2 w          window size = columns of Y = order of U, 1..128
 *  3 Y          device: element (r, k) at Y[r * rs + k * ks], updated in place
 *  4 rs, 5 ks   strides in elements, >= 1, with rs == 1 or ks == 1
 *                 (-4 if not)
 *  6 U          device: w x w, column-major, leading dimension ldU; read only
 *  7 ldU        >= w
 *  8 precision  GBR_PREC_DMMA: FP64 tensor-core products (DMMA);
 *               GBR_PREC_FMA: FP64 fused multiply-adds, one chain per output
 *               over k in increasing order from +0 (register tiles);
 *               GBR_PREC_OZAKI: emulated FP64 on the bf16 tensor cores (7
 *               balanced 8-bit digit slices of every entry, relative to
 *               the largest exponent of its row of Y or column of U; the 28
 *               slice products with p + q <= 8 summed exactly; one rounding
 *               to double).  Per product term, the truncation of both
 *               operands and the dropped digit products are below
 *               2^-50 |y|max |u|max; results below the normal range are
 *               flushed to zero.
 *  9 cuda_stream  as for gbr_reorder
 * Returns 0, -i for an invalid argument i, GBR_ERR_TIMEOUT if a bounded
 * tensor-core wait gave up (Y is then partially updated), or GBR_ERR_*.
 * Scratch (a contiguous copy of U and its digit slices) comes from the
 * library's pool.
 */
int gbr_update_panel(int rows, int w, double *Y, long long rs, long long ks, const double *U,
                     int ldU, int precision, void *cuda_stream);

/*
 * Eigenvectors of a real Schur form (Section 2, Eq. 5) and their back-
 * transformation (Eq. 6):
 *
 *     (S - lambda I) y = 0,   x = Q y,
 *
 * for the selected eigenvalues, protected against floating-point overflow.
 * Each y comes from back substitution over the diagonal blocks above its
 * eigenvalue.  Pivots below max(eps |lambda|, DBL_MIN / eps) are raised to
 * that value.  The vector is scaled by exact powers of two (2^-512) before
 * any solve or update that could exceed 2^900.  The result is normalized:
 * max |x_i| = 1 for a real vector, max (|re x_i| + |im x_i|) = 1 for a
 * complex one.  The back-transformation runs on the FP64 tensor cores (DMMA).
 *
 *  1 n        order of S (>= 0)
 *  2 S        device, standard real Schur form (-2 if not), column-major; read only
 *  3 ldS      >= max(1, n)
 *  4 Q        device, n x n orthogonal factor (column-major), or NULL for x = y
 *  5 ldQ      >= max(1, n) if Q is given
 *  6 select   host, n ints (a 2x2 block is selected if either row is), or NULL
 *             for every eigenvalue
 *  7 X        device, n x m output (m = number of selected positions), or NULL
 *             to query m only.  Columns in diagonal order: one per real
 *             eigenvalue; a conjugate pair gives two, the real and the
 *             imaginary part of the vector of the eigenvalue with positive
 *             imaginary part
 *  8 ldX      >= max(1, n)
 *  9 m_out    host or NULL: m
 * 10 nscale   host, m ints or NULL: per column, the number of 2^-512 scalings
 *             the overflow protection applied
 * 11 stats    host or NULL: kernel times (CUDA events on the stream) and the
 *             algorithmic flops of the back substitution (the right-hand-side
 *             updates, 2 per real multiply-add, doubled for complex vectors)
 *             and of the back-transformation
 * 12 cuda_stream
 * Returns 0, -i for an invalid argument i, or GBR_ERR_*.  Scratch (the
 * vectors before back-transformation, bounds, right-hand sides) comes from
 * the library's pool.
 */
typedef struct gbr_ev_stats {
    double ms_solve;            /* column bounds + back substitution */
    double ms_backtransform;    /* X = Q Y (0 without Q) */
    double ms_normalize;
    double solve_flops;
    double backtransform_flops;
} gbr_ev_stats;
int gbr_eigenvectors(int n, const double *S, int ldS, const double *Q, int ldQ,
                     const int *select, double *X, int ldX, int *m_out, int *nscale,
                     gbr_ev_stats *stats, void *cuda_stream);

/*
 * Batched reordering: many independent problems (Eq. 7 for each), planned
 * together into one task graph and run by one persistent-scheduler launch
 * captured in a CUDA graph.  No counterpart in the paper, which reorders one
 * (distributed) matrix; the window, chain and update tasks of each instance
 * are those of Section 3.2.
 *
 * gbr_batch_create plans a batch and captures its CUDA graph:
 *  1 count    number of instances (>= 0)
 *  2 n        host, count ints: order of each instance (>= 0)
 *  3 S        host array of count device pointers (column-major, ldS[i]);
 *             the caller keeps them allocated until gbr_batch_destroy
 *  4 ldS      host, count ints, ldS[i] >= max(1, n[i])
 *  5 Q        host array of count device pointers (entries may be NULL), or
 *             NULL for no Schur vectors at all
 *  6 ldQ      host, count ints (ignored where Q[i] is NULL); may be NULL if Q is
 *  7 select   host, sum(n) ints: the selections, concatenated in instance order
 *  8 opts     options or NULL; window/chain = GBR_AUTO picks them per
 *             instance from the autotuner's table for the current device
 *             (built-in defaults for sizes it has not tuned); precision,
 *             strong_test, validate, wait_limit_ms as for gbr_reorder;
 *             opts.sched must be GBR_SCHED_PERSISTENT
 *  9 status   host, count ints or NULL: 0, or -2 for an instance not in
 *             standard form (it is left out of the plan and never touched)
 * 10 out      receives the batch handle
 * 11 cuda_stream  stream for the planning work; the handle runs on the
 *             stream given to gbr_batch_run
 * Returns 0, -i for an invalid argument i, or GBR_ERR_*.  The handle owns
 * its device memory (plan, accumulators, staging) until gbr_batch_destroy.
 *
 * gbr_batch_run reorders the current contents of the batch's S and Q in
 * place.  They must have the block structure (positions of the 2x2 blocks)
 * they had when the batch was planned: the graph checks this first on the
 * device and, if any instance differs, modifies nothing and the call
 * returns GBR_ERR_PLAN_MISMATCH.
 *  eig_re, eig_im  host, sum(n) doubles each, or NULL: eigenvalues of each
 *             S_hat in diagonal order, concatenated
 *  m_out      host, count ints or NULL: selected eigenvalues per instance
 *  status     host, count ints or NULL: 0, +k (k swaps rejected; the
 *             instance then got further passes outside the graph, as in
 *             gbr_reorder), or -2 (invalid, untouched)
 *  stats      host or NULL: totals over the batch (ms_sched = the scheduler
 *             kernel's time when opts.timing)
 * Returns 0 if every valid instance returned 0, else the number of
 * instances with rejected swaps, or GBR_ERR_*.
 *
 * gbr_reorder_batched = create + run + destroy.
 */
typedef struct gbr_batch gbr_batch;

int gbr_batch_create(int count, const int *n, double *const *S, const int *ldS,
                     double *const *Q, const int *ldQ, const int *select,
                     const gbr_opts *opts, int *status, gbr_batch **out, void *cuda_stream);
int gbr_batch_run(gbr_batch *batch, double *eig_re, double *eig_im, int *m_out, int *status,
                  gbr_stats *stats, void *cuda_stream);
void gbr_batch_destroy(gbr_batch *batch);
int gbr_reorder_batched(int count, const int *n, double *const *S, const int *ldS,
                        double *const *Q, const int *ldQ, const int *select,
                        double *eig_re, double *eig_im, int *m_out, int *status,
                        const gbr_opts *opts, gbr_stats *stats, void *cuda_stream);

/*
 * Autotuner of the batched path.  For each size class n in (16, 32],
 * (32, 64], ... up to n_max, it builds a seeded synthetic batch of
 * `per_class` instances of that class (standard Schur forms with 60% of
 * positions in 1x1 blocks, 20-60% of the eigenvalues selected, Q present),
 * runs it under every candidate (window w in {32, 64, 96, 128} not above
 * the class, chain m in {w/4, w/2, 3w/4}, far update-tile height in
 * {64, 256}), times the scheduler kernel with CUDA events, and keeps the
 * fastest candidate per class in a table for the current device.
 * Returns the number of classes tuned, or GBR_ERR_*.
 */
int gbr_autotune(int n_max, int per_class, void *cuda_stream);

/*
 * The autotuner's choice for an instance of order n on the current device:
 * window, chain and far update-tile height (NULL outputs are skipped).
 * Returns 1 if the class was tuned, 0 if these are the built-in defaults.
 */
int gbr_tune_get(int n, int *window, int *chain, int *tile);

/*
 * Saves the current device's autotuner table to a JSON file, one object per
 * tuned size class:
 *   {"tune": [{"n_max": 32, "window": 32, "chain": 24, "tile": 64}, ...]}
 * (n_max: the largest n of the class, a power of two >= 32; tile 0 means the
 * built-in far tile height).  Returns the number of classes written, -1 (NULL
 * path) or -2 (the file cannot be written).
 */
int gbr_tune_save(const char *path);

/*
 * Loads a table written by gbr_tune_save into the current device's table
 * (the classes it lists replace the tuned or default ones), so that a tuning
 * can be reused across processes.  Every class is checked first (n_max a
 * power of two >= 32, window 4..128, chain 1..window-2, tile 0, 64 or 256);
 * on any error nothing is changed.  Returns the number of classes loaded, -1
 * (NULL path), -2 (the file cannot be read) or -3 (malformed or invalid
 * content).  Host only: no GPU work.
 */
int gbr_tune_load(const char *path);

/*
 * Reordering server: continuous batching of requests on one GPU.  No
 * counterpart in the paper; each request is the reordering of Eq. 7 with
 * the tasks of Section 3.2.
 *
 * One long-lived kernel (one CTA per SM, or cfg.sms of them) runs the tasks
 * of every request; a server thread feeds it through a ring of (request,
 * task) entries in device memory, appending a chunk of each request's tasks
 * in turn, so a request that arrives while others are on the GPU starts
 * within one chunk of their tasks.  Requests are validated and planned on
 * the submitting thread, admitted in arrival order while their device
 * footprint (S, Q, window accumulators, task graph) fits under
 * mem_cap_bytes and a request slot is free, copied to device memory owned
 * by the server where they stay until they complete, and copied back to
 * the caller's buffers at the end.  A request's result does not depend on
 * the other requests in flight.  While a server exists, its kernel occupies
 * its SMs: other kernels of the process wait for them.
 */
typedef struct gbr_server gbr_server;

typedef struct gbr_server_cfg {
    long long mem_cap_bytes; /* device memory for admitted requests (default 60e9) */
    int max_inflight;        /* request slots on the device (default 512)          */
    int sms;                 /* CTAs of the server kernel, 0 = one per SM (default) */
    long long ring_entries;  /* task ring capacity (default 4M entries, 32 MB)      */
    long long idle_limit_ms; /* the kernel gives up after this long with nothing to
                                do (0: one hour); requests in flight then fail   */
    int device;              /* CUDA device (default -1: current at create)       */
    gbr_opts opts;           /* per-request options (gbr_default_opts); window
                                and chain GBR_AUTO use the autotuner table       */
} gbr_server_cfg;

typedef struct gbr_server_stats {
    long long submitted, completed, failed;
    long long passes;       /* planned passes uploaded (> completed after rejections) */
    double p50_ms, p99_ms, max_ms;  /* latency: submit to results in the caller's buffers */
    double mean_ms;
    double req_per_s;       /* completed / (last completion - first submit) */
    double eigs_per_s;      /* selected eigenvalues of completed requests, same span */
    double mean_inflight;   /* requests on the device, averaged over server iterations */
    double peak_mem_bytes;  /* largest admitted footprint */
} gbr_server_stats;

void gbr_server_default_cfg(gbr_server_cfg *cfg);

/* Starts a server.  Returns 0, -1 (cfg invalid), or GBR_ERR_*. */
int gbr_server_create(const gbr_server_cfg *cfg, gbr_server **out);

/*
 * Submits one request: n, host S (ldS), host Q or NULL (ldQ), host select
 * (n ints), and optional host eig_re/eig_im (n doubles each).  Every buffer
 * must stay valid and untouched until the request completes; S and Q are
 * overwritten with the result then.  Pinned (page-locked) buffers copy
 * fastest.  Returns a ticket >= 0, or -i / GBR_ERR_* (a request larger than
 * the memory cap gives GBR_ERR_NOMEM).
 */
long long gbr_server_submit(gbr_server *srv, int n, double *S, int ldS, double *Q, int ldQ,
                            const int *select, double *eig_re, double *eig_im);

/* 1 if the request completed (status and m written, when non-NULL), 0 if
   not yet, -1 for an unknown ticket.  status as for gbr_reorder. */
int gbr_server_poll(gbr_server *srv, long long ticket, int *status, int *m_out);

/* Waits up to timeout_ms (< 0: no limit) for a request; returns as poll. */
int gbr_server_wait(gbr_server *srv, long long ticket, int *status, int *m_out,
                    long long timeout_ms);

/* Latency and throughput of the requests completed so far. */
int gbr_server_get_stats(gbr_server *srv, gbr_server_stats *out);

/* Waits for all submitted requests, stops the server and frees it. */
void gbr_server_destroy(gbr_server *srv);

/*
 * Window plan of a bulge-chasing sweep (gbr_qr_sweep), on the host only (no
 * GPU work): chains of bulges, each chain's windows top to bottom, in
 * program order.  A window (s, e, t0, t1, b0, nb) runs chain steps
 * [t0, t1) of the bulges [b0, b0 + nb) over rows / columns [s, e): at step
 * tau bulge j of the chain sits at k_j = tau - 3 j - 1, and every active
 * bulge (-1 <= k_j <= n - 3) has its input column at or below s (or is
 * introduced, s = 0) and its rows k_j + 1 .. k_j + 4 above e (or e = n).
 *
 *  n, nshifts     order and (even) shift count
 *  window, chain  as for gbr_qr_sweep (window 8 .. 128, capped at 96,
 *                 chain = shifts per chain, at most window / 3)
 *  out            host, 6 * max_windows ints or NULL
 *  max_windows    capacity of out
 * Returns the number of windows (only the first max_windows are written),
 * or -1 (n < 0 or odd / negative nshifts), -10 (bad window or chain).
 */
int gbr_plan_sweep(int n, int nshifts, int window, int chain, int *out, int max_windows);

/*
 * Window plan of a reordering, on the host only (no GPU work): the diagonal
 * windows that gbr_reorder launches, in program order, assuming no swap is
 * rejected (Section 3.2, Fig. 2: one chain of windows per group of at most
 * `chain` selected eigenvalues, each window at most `window` rows, never
 * cutting a 2x2 block).
 *
 *  n          order of S
 *  sub        host, n bytes: sub[i] != 0 iff S[i+1, i] != 0 (2x2 block at i)
 *  select     host, n ints, as for gbr_reorder
 *  window, chain   as in gbr_opts
 *  with_q     nonzero to count the flops of the Q update
 *  windows    host, 2 * max_windows ints or NULL: (s, e) of each window
 *  max_windows  capacity of `windows`
 *  chains     host or NULL: number of chains
 *  upd_flops  host or NULL: flops of all off-diagonal updates,
 *             sum over windows of 2 w^2 ((n - e) + s + (with_q ? n : 0))
 * Returns the number of windows (only the first max_windows are written),
 * or -1 (n < 0), -2 (sub or select NULL), -4/-5 (bad window/chain).
 */
int gbr_plan(int n, const unsigned char *sub, const int *select, int window, int chain,
             int with_q, int *windows, int max_windows, int *chains, double *upd_flops);

/*
 * Timeline of the last persistent-scheduler launch made with opts.timing = 2
 * by gbr_reorder, gbr_reorder_host (a pass of a single launch: traced calls
 * are not cut into chunks) or gbr_batch_run (the batch's scheduler launch;
 * window indices run over all instances in their order) (tracing; no
 * counterpart in the paper).  Writes up to max_tasks records of
 * 8 long longs each, in queue order: task kind (0 window, 1 left tile,
 * 2 right tile, 3 Q tile), window index, first panel row, panel rows, SM id,
 * time the CTA took the task, time it started executing (its predecessors
 * had finished), time it ended (nanoseconds of the GPU global timer).
 * Returns the number of records available.  `out` may be NULL.
 */
int gbr_last_trace(long long *out, int max_tasks);

/* Human-readable text for a status code (static storage). */
const char *gbr_status_string(int status);

/* Text of the last CUDA error seen by the calling thread ("" if none). */
const char *gbr_last_error(void);

/* Bytes of device memory the library's scratch pool holds on the current
 * device (all slots; 0 before the first allocating call and after
 * gbr_release), or -1 if no device is current.  Diagnostic only. */
long long gbr_pool_bytes(void);

/* Release the library's device scratch pool on the current device. */
void gbr_release(void);

/* Library version, e.g. 100 for 0.1.0. */
int gbr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBREORDER_H */
