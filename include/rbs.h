/*
 * rbs.h - C ABI of the GB300 (sm_103a) reproducible PBiCGStab library.
 *
 * Method: Iakymchuk & Aliaga, "General framework for re-assuring numerical
 * reliability in parallel Krylov solvers: A case of BiCGStab methods"
 * (arXiv 2302.04180). The library computes the data-parallel hot path of the
 * paper's reproducible and accurate preconditioned BiCGStab (Fig. 2) and
 * pipelined preconditioned BiCGStab (Fig. 4): the exact, correctly rounded dot
 * product (Sec. 2, Sec. 3.2), the fma-ordered CSR SpMV and the Jacobi and
 * axpy-like updates (Sec. 3.3, Sec. 4.1), and the scalar recurrences of both
 * loops. All arithmetic is IEEE-754 binary64, round to nearest even, plus exact
 * integer accumulation; every result is bitwise independent of the launch
 * configuration and of scheduling.
 *
 * Conventions for every entry point:
 *  - Pointers are plain C pointers. Unless an argument says otherwise it must
 *    point to device memory of the current CUDA device; arguments marked
 *    "host or device" may point to either (the library asks the CUDA runtime
 *    which one it is and stages host data through its own device buffers).
 *  - Vectors are contiguous binary64 arrays, 8-byte aligned; 16-byte alignment
 *    enables the vectorised load path (results are identical either way).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *    enqueued on it in order. Calls that return results in host memory
 *    synchronise the stream before returning.
 *  - The caller owns every buffer it passes and keeps it alive until the
 *    stream has finished the call. The library owns a per-(device, stream)
 *    workspace that it creates on first use and frees in rbs_release().
 *  - Errors are returned as an int status (RBS_OK = 0); no C++ exception
 *    crosses the ABI. rbs_last_error() gives a one-line message for the
 *    calling thread's last failure.
 *  - Kernels never read out of bounds. The standalone SpMV checks every CSR
 *    index on the device before use; a bad index is kept in range and
 *    recorded in the workspace's error word, and rbs_stream_status() (or a
 *    synchronising call) then returns RBS_EINVAL. The solvers validate the
 *    whole structure once at set-up (rowptr rising from 0 to nnz, columns in
 *    [0, n)), return RBS_EINVAL if it fails, and then iterate with kernels
 *    that do not re-check it: the matrix must not change during a solve.
 *  - Device-side waits are bounded; one that expires (a staging copy that
 *    never lands) returns RBS_ETIMEOUT instead of hanging.
 */
#ifndef RBS_H
#define RBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define RBS_OK 0
#define RBS_EINVAL 1      /* bad argument: null pointer, n < 0, invalid CSR, zero or missing diagonal */
#define RBS_ENOMEM 2      /* device or pinned host allocation failed */
#define RBS_ECUDA 3       /* a CUDA runtime call failed (message in rbs_last_error) */
#define RBS_EBREAKDOWN 4  /* a zero denominator stopped the solver (history so far is kept) */
#define RBS_ENAN 5        /* a non-finite scalar stopped the solver */
#define RBS_ETIMEOUT 6    /* a bounded device-side wait expired */

/* ---- sparse matrix ----------------------------------------------------------
 * CSR, n x n: rowptr[n+1] (int64, rowptr[0] = 0, non-decreasing,
 * rowptr[n] = nnz), col[nnz] (int32, 0 <= col < n), val[nnz] (binary64). The
 * stored order of each row is the order of its fma chain and is never changed;
 * duplicate column entries are allowed and kept. Device pointers (rbs_solve
 * also accepts host pointers). */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
} rbs_csr;

/* ---- exact dot product (Sec. 2 "ExBLAS ... exdot"; Sec. 3.2) ------------------
 * out = RN(sum_{i<n} x[i]*y[i]): every product is formed exactly (53x53-bit
 * integer significands), accumulated exactly in a Kulisch-style fixed-point
 * accumulator covering 2^-2148 .. 2^2200, and rounded once to nearest even.
 * An exact zero gives +0.0; n == 0 gives +0.0. A NaN operand, an inf*0 product
 * or infinite products of both signs give NaN; otherwise an infinite product
 * gives that infinity; finite products are always summed exactly, and an exact
 * sum beyond the binary64 range rounds to +-inf.
 * x, y: n binary64 (host or device). out: 1 binary64 (host or device; host
 * output synchronises the stream). Asynchronous with device output. */
int rbs_exdot(const double *x, const double *y, int64_t n, double *out, void *stream);

/* k exact dots over the same length in one pass (Sec. 4.1: S10 and S11 merged
 * in one reduction; Sec. 4.2: the two- and four-dot reductions of Fig. 4).
 * xs[j], ys[j] (j < k, 1 <= k <= 6): host arrays of device pointers; operands may
 * repeat (e.g. <r0,r> and <r,r>). out: k binary64 (host or device). */
int rbs_exdot_multi(int k, const double *const *xs, const double *const *ys, int64_t n,
                    double *out, void *stream);

/* Long-accumulator export for row-block ranks (Sec. 3.2): a rank's exact
 * partial sum of x[i]*y[i] as RBS_LIMBS int64 limbs, limb j weighing
 * 2^(32j - 2148), plus a flags word (bit 0: NaN, bit 1: +inf product,
 * bit 2: -inf product). Limb values are signed and partially normalised
 * (|limb| < 2^34), so ranks may add limb arrays as plain integers, in any
 * order, up to 2^28 of them, OR the flags, and round once with
 * rbs_round_limbs: the result is bitwise the single-rank rbs_exdot.
 * limbs: RBS_LIMBS int64 (device); flags: 1 int32 (device). */
#define RBS_LIMBS 136
int rbs_exdot_partial(const double *x, const double *y, int64_t n, int64_t *limbs,
                      int32_t *flags, void *stream);
/* out = RN(value of the limb array) (host or device out; device limbs). */
int rbs_round_limbs(const int64_t *limbs, const int32_t *flags, double *out, void *stream);

/* Lightweight FPE-8 dot (Sec. 3.2: floating-point expansions of size eight
 * with early exit, and a check that warns when the condition number or the
 * dynamic range is too large to keep every bit). Each thread accumulates
 * TwoProd results (Alg. 2) in an expansion of at most eight binary64 terms with
 * TwoSum cascades (Alg. 1); the expansions are merged exactly and rounded once
 * (correct rounding, the role of NearSum in the paper). If a thread needs a
 * ninth term, a TwoProd may be inexact (|x*y| < 2^-969) or a value is not
 * finite, the call falls back to rbs_exdot and sets *fell_back = 1 (nullable).
 * Either way out = rbs_exdot's value, bit for bit. x, y: host or device;
 * out: host or device. Synchronises the stream. */
int rbs_fpe_dot(const double *x, const double *y, int64_t n, double *out, int32_t *fell_back,
                void *stream);

/* Allocation-free variant of rbs_exdot_multi (the paper has no counterpart; it
 * is a deployment aid). For callers that cannot allocate when they call: code
 * running while a CUDA graph is captured, latency-critical loops that cannot
 * take an allocation's implicit synchronisation, applications whose own pool
 * owns the device memory. Same results, bit for bit, as rbs_exdot_multi.
 * Its scratch is one 8 KiB file-scope device array inside the library, held
 * by every GPU that loads the library until the process exits; it holds at most
 * RBS_NOALLOC_MAX_DOTS accumulators, and larger k returns RBS_EINVAL. xs, ys
 * (host arrays of device pointers), out (k binary64): device memory only.
 * The first call on a device sets up that device (finds the array's device
 * address and clears it, synchronously): make it before any stream capture.
 * Every call clears the array on `stream` before use. All calls on a device
 * share the array, so calls that overlap on the GPU race; order them. */
#define RBS_NOALLOC_MAX_DOTS 6
int rbs_exdot_noalloc(int k, const double *const *xs, const double *const *ys, int64_t n,
                      double *out, void *stream);

/* ---- fma-ordered SpMV (Sec. 4.1 "Sparse matrix-vector product"; Sec. 3.3) ----
 * y[i] = fma(val[last], x[col[last]], ... fma(val[first], x[col[first]], +0.0))
 * over row i in stored order, every step rounded to nearest even; an empty row
 * gives +0.0. x: A->n binary64, y: A->n binary64 (device; y must not alias x).
 * Asynchronous. */
int rbs_spmv_csr(const rbs_csr *A, const double *x, double *y, void *stream);

/* ---- Jacobi preconditioner (Sec. 4: M = diag(A), applied element-wise) ------
 * invd[i] = RN(1 / d[i]) with d = diag (if non-null) else the first stored
 * entry (i, i) of row i. Synchronises; RBS_EINVAL on a zero, NaN or missing
 * diagonal. invd: n binary64 (device). */
int rbs_jacobi_invd(const rbs_csr *A, const double *diag, double *invd, void *stream);
/* phat[i] = RN(p[i] * invd[i]). Asynchronous. */
int rbs_jacobi_apply(int64_t n, const double *invd, const double *p, double *phat,
                     void *stream);

/* ---- solver ------------------------------------------------------------------ */
#define RBS_CLASSIC 0   /* PBiCGStab, Fig. 2 */
#define RBS_PIPELINED 1 /* p-PBiCGStab, Fig. 4 */

#define RBS_DOT_EXACT 0 /* reproducible: exact dots rounded once (the method) */
#define RBS_DOT_PLAIN 1 /* comparator: binary64 dots with atomic accumulation,
                           run-to-run non-reproducible (the paper's "original") */

#define RBS_LOOP_GRAPH 0 /* the loop runs on the device: one iteration is the body of a
                            CUDA-graph conditional WHILE node (no host round trips) */
#define RBS_LOOP_HOST 1  /* the host enqueues iterations in chunks and reads the stop flag */

typedef struct {
    int32_t dot_mode;    /* RBS_DOT_EXACT (default) or RBS_DOT_PLAIN */
    int32_t check_every; /* RBS_LOOP_HOST: iterations enqueued between host reads of the
                            stop flag; 0 = library default */
    int32_t profile;     /* 1: time every kernel launch with CUDA events, see rbs_prof
                            (uses RBS_LOOP_HOST) */
    int32_t loop_mode;   /* RBS_LOOP_GRAPH (default) or RBS_LOOP_HOST. Results do not
                            depend on loop_mode or check_every. */
} rbs_opts;

typedef struct {
    int32_t iters;     /* loop bodies executed */
    int32_t converged; /* 1 iff tau <= tau_max at exit and status == RBS_OK */
    int32_t status;    /* RBS_OK, RBS_EBREAKDOWN or RBS_ENAN (also the return value) */
    int32_t reserved;
    double tau0;       /* RN(sqrt(<r0, r0>)) */
    double tau_final;  /* tau of the last iteration (tau0 if none) */
    double rho0;       /* <r0, r0> */
    double tau_max;    /* RN(tol * tau0) */
    double alpha0;     /* pipelined: RN(<r0,r0> / <r0,w0>) (NaN if not computed) */
    double mu0;        /* pipelined: <r0, w0> */
} rbs_info;

/* Per-iteration record of every scalar, RBS_HIST_W binary64 each; fields not
 * computed in an iteration hold the quiet NaN 0x7ff8000000000000.
 *  classic:   0 sigma=<r0,s> 1 alpha 2 gamma=<q,y> 3 delta=<y,y> 4 omega
 *             5 rho'=<r0,r> 6 theta=<r,r> 7 tau 8 beta
 *  pipelined: 0 gamma=<q,y> 1 delta=<y,y> 2 omega 3 rho'=<r0,r> 4 <r0,w>
 *             5 <r0,s> 6 <r0,z> 7 theta=<r,r> 8 tau 9 beta 10 alpha denominator
 *             11 next alpha
 * rec: host array of cap * RBS_HIST_W binary64; len receives the number of
 * records written (= iters, at most cap). */
#define RBS_HIST_W 12
typedef struct {
    int32_t cap;
    int32_t len;
    double *rec;
} rbs_history;

/* Kernel timing from rbs_opts.profile: per kernel kind, launches and summed
 * CUDA-event milliseconds over the whole solve. The host enqueues iterations
 * ahead of reading the stop flag, so a few launches return at once because the
 * loop has already stopped: those (every launch of an iteration index >= iters,
 * and the launches after the stopping kernel in the last iteration: classic K5,
 * pipelined S18) are left out of launches/ms. The optional per-launch trace
 * lists every launch in enqueue order, left-out ones included. */
#define RBS_PROF_KINDS 8
typedef struct {
    int64_t launches[RBS_PROF_KINDS];
    double ms[RBS_PROF_KINDS];
    /* kinds: 0 classic K1 (SpMV + <r0,s>), 1 vector update without dots
       (classic K2, K5), 2 set-up, 3 standalone SpMV (pipelined S10/S18),
       4 pipelined vector update with dots (P1, P3), 5 classic K3 (SpMV +
       <q,y>, <y,y>), 6 classic K4 (x, r update + <r0,r>, <r,r>), 7 unused */
    int32_t trace_cap;   /* entries of the three trace arrays (0 or null arrays: no trace) */
    int32_t trace_len;   /* entries written (at most trace_cap) */
    int32_t *trace_kind; /* host: kernel kind of each launch */
    int32_t *trace_iter; /* host: iteration index of the launch, -1 for set-up */
    float *trace_ms;     /* host: the launch's CUDA-event duration in milliseconds */
} rbs_prof;

/* Solve A x = b with Jacobi-preconditioned BiCGStab (Fig. 2) or pipelined
 * BiCGStab (Fig. 4), with reproducible exact dots, stopping when
 * tau = RN(sqrt(<r,r>)) <= RN(tol * tau0) or after maxit iterations.
 * Readings of the figures (all bitwise-pinned against the CPU oracle):
 *  r0 = RN(b - A x0) element-wise (x0 NULL: zero and r0 = b); invd = RN(1/d);
 *  x-update fma(omega, qhat, fma(alpha, phat, x)); classic p-update
 *  fma(beta, fma(-omega, s, p), r); beta = RN(RN(rho'/rho) * RN(alpha/omega));
 *  pipelined alpha denominator fma(-RN(beta*omega), <r0,z>, fma(beta, <r0,s>, <r0,w>));
 *  pipelined tau from a fifth dot <r,r> in the S16 reduction; pipelined
 *  iteration 0 starts from copies (beta = 0); <y,y> == 0 gives omega = 0; the
 *  stop test runs as soon as tau is known; zero denominators stop with
 *  RBS_EBREAKDOWN; non-finite scalars stop with RBS_ENAN.
 * A, b, x0, jacobi_diag: host or device. x_out: n binary64, host or device.
 * info (host, required), hist (host, nullable), prof (host, nullable),
 * opts (host, nullable = defaults). Synchronises the stream. */
int rbs_solve(const rbs_csr *A, const double *b, const double *x0, const double *jacobi_diag,
              double tol, int32_t maxit, int32_t variant, double *x_out, rbs_info *info,
              rbs_history *hist, void *stream);
int rbs_solve_ex(const rbs_csr *A, const double *b, const double *x0,
                 const double *jacobi_diag, double tol, int32_t maxit, int32_t variant,
                 const rbs_opts *opts, double *x_out, rbs_info *info, rbs_history *hist,
                 rbs_prof *prof, void *stream);

/* ---- batched solves ----------------------------------------------------------------
 * Many independent systems (each as in rbs_solve, Fig. 2 or Fig. 4 per system)
 * in one persistent launch: thread-block clusters of 8 CTAs take systems from a
 * queue, largest first, and run each solve to completion. Every system's
 * iterates, history and x are bitwise those rbs_solve gives for it alone, in any
 * batch. All pointers of an rbs_system are device memory; x0 and jacobi_diag
 * may be NULL. systems, infos (nsys each) and hists (nsys, nullable; a record
 * with cap == 0 keeps no history) are host arrays. Synchronises the stream.
 * Returns RBS_EINVAL if any system fails the argument or structure checks
 * (those systems report status RBS_EINVAL and are not solved; the others are),
 * else RBS_OK; per-system breakdowns are in infos[i].status. */
typedef struct {
    rbs_csr A;
    const double *b;
    const double *x0;
    const double *jacobi_diag;
    double *x;
    double tol;
    int32_t maxit;
    int32_t variant;
} rbs_system;
int rbs_solve_batched(int32_t nsys, const rbs_system *systems, rbs_info *infos, rbs_history *hists,
                      void *stream);

/* Schedule of a batched solve (the library's own tuning; the paper has
 * none). cluster 1, 2, 4, 8 or 16: one persistent launch of thread-block
 * clusters of `cluster` CTAs (16 needs the device's non-portable cluster
 * size); systems are queued largest first, one with at least `split` unknowns
 * is solved by a whole cluster (rows split across its CTAs, dots reduced
 * through distributed shared memory), and from the first smaller one on every
 * CTA takes systems alone. cluster 0, the stepped schedule: every system
 * advances one iteration per step, one launch per phase of Fig. 2 / Fig. 4 for
 * all of them, each system on blocks of `split` rows (0: sized per chunk of
 * steps from the rows still iterating, about four waves of blocks), so a large
 * system spreads over as many SMs as its rows fill (x must be 16-byte
 * aligned). `ms` is the tuner's measured time of its proxy run (0 otherwise).
 * Results never depend on the schedule: every system's iterates are bitwise
 * those of rbs_solve. */
typedef struct {
    int32_t cluster;
    int32_t pad;
    int64_t split;
    double ms;
} rbs_batch_schedule;

/* rbs_solve_batched with an explicit schedule (NULL: the schedule the last
 * rbs_batch_tune on this device chose, else cluster 8 and split 0). Returns
 * RBS_EINVAL for a malformed schedule or one whose clusters do not fit. */
int rbs_solve_batched_ex(int32_t nsys, const rbs_system *systems, rbs_info *infos, rbs_history *hists,
                         const rbs_batch_schedule *sched, void *stream);

/* Autotune the batched schedule for this batch: times proxy solves of the
 * systems (each stopped after a number of iterations) under candidate
 * schedules -- every cluster size at the median split, then every split
 * candidate (system-size quantiles, 0 and "no cluster") at the best size, then
 * the stepped schedule with adaptive, 2048 and 8192 rows per block -- and returns
 * the fastest in *best, which later rbs_solve_batched calls on this
 * device use. The proxy iteration cap of system i is proxy_iters, or, given a
 * previous solve's infos (`prev`, nsys entries, nullable), proxy_iters scaled
 * by prev[i].iters / max_j prev[j].iters so that systems keep their relative
 * costs. Proxy solves write x into library scratch, not the callers' buffers,
 * and keep no history. Synchronises the stream. */
int rbs_batch_tune(int32_t nsys, const rbs_system *systems, const rbs_info *prev, int32_t proxy_iters,
                   rbs_batch_schedule *best, void *stream);

/* ---- serving ---------------------------------------------------------------------
 * A request loop with per-iteration continuous batching (the library's own
 * runtime; the paper has no counterpart). Clients submit solves (rbs_system,
 * device pointers; x 16-byte aligned) at any time. Each of `engines` threads
 * owns a stream and up to `max_active` slots, a slot being the resident state
 * of one system in flight: its Krylov vectors (allocated from the server's own
 * stream-ordered memory pool at admission, freed at retirement), its device
 * scalars and its dot scratch. An engine advances in steps. A step admits
 * pending requests in arrival order into free slots while the vector memory of
 * the systems in flight stays within `budget_bytes` (one request is always
 * admitted when none is in flight), runs their structure check, Jacobi and
 * solver set-up, then one iteration (Fig. 2 or Fig. 4) of every system in
 * flight: one launch per phase for all of them, each system on blocks of
 * `rows_per_block` rows (0: sized per step from the rows in flight, about four
 * waves of blocks), classic and pipelined systems on two streams. Stopped systems (converged, breakdown, NaN,
 * invalid, or maxit iterations) are retired a step or two later. A request that
 * arrives while others iterate joins them at the next step. Every answer is
 * bitwise the one rbs_solve gives for that system alone (the same element
 * functions, exact dots and scalar tails). The caller keeps a submitted
 * system's buffers alive until its request is done. Latency = submission to
 * retirement; queue = submission to admission. Handles and outputs are host.
 * Errors: bad arguments at submission, or a system that fails its device-side
 * structure or diagonal check, end the request with RBS_EINVAL (poll/wait
 * report it in info->status, rbs_last_error() gives the reason); a CUDA error
 * ends every request in flight with RBS_ECUDA. */
typedef struct rbs_server rbs_server;
int rbs_server_create(int32_t engines, int32_t max_active, int64_t budget_bytes, int64_t rows_per_block,
                      rbs_server **out);
int rbs_server_submit(rbs_server *srv, const rbs_system *system, int64_t *ticket);
int rbs_server_poll(rbs_server *srv, int64_t ticket, int32_t *done, rbs_info *info, double *latency_s,
                    double *queue_s);
int rbs_server_wait(rbs_server *srv, int64_t ticket, rbs_info *info, double *latency_s, double *queue_s);
/* Where a request ran: the engine step that admitted it and the step whose
 * scalars retired it (-1 before that), and how many systems were already in
 * flight on its engine when it joined. */
typedef struct {
    int64_t admit_step, finish_step;
    int32_t active_at_admit, done;
} rbs_request_stats;
int rbs_server_request_stats(rbs_server *srv, int64_t ticket, rbs_request_stats *out);
/* Server counters: steps run, requests completed, most systems in flight at
 * once, requests pending, vector bytes of the systems in flight (the budgeted
 * quantity), and the memory pool's reserved bytes now and at its peak. */
typedef struct {
    int64_t steps, completed, peak_active, pending, budget_in_use, pool_reserved, pool_reserved_peak;
} rbs_server_counters;
int rbs_server_stats(rbs_server *srv, rbs_server_counters *out);
int rbs_server_destroy(rbs_server *srv);

/* ---- library control ---------------------------------------------------------- */
/* Synchronise `stream`, then return and clear the workspace error word:
 * RBS_OK, or RBS_EINVAL if a kernel met an out-of-range CSR index. */
int rbs_stream_status(void *stream);
/* Free every workspace of the calling process (all devices and streams). */
int rbs_release(void);
/* Launch-shape knobs for tuning and for configuration-independence tests.
 * Names: "exdot.grid", "exdot.block", "exdot.window" (0 = auto),
 * "spmv.block" (short rows; long rows run in their own 4-warp blocks),
 * "spmv.mode" (0 auto: warp-staged rows, the long-row schedule when rows average
 * more than 8 nonzeros -- one staging buffer per warp, each row's values and x
 * entries moved to registers; 1 one thread per row; 2 short; 3 long rows),
 * "vec.grid", "vec.block", "solve.check_every", "smem.carveout" (percent of
 * L1/shared storage for the staging kernels; default 75, -1 = driver default);
 * "test.stall_staging" (1: a test mode of the bounded device-side wait --
 * the staged SpMV announces its bulk copies without issuing them and gives up
 * after 64 polls, reads those rows from global memory instead, and the call
 * reports RBS_ETIMEOUT; results do not change).
 * Results never depend on them. */
int rbs_set_param(const char *name, int64_t value);
int64_t rbs_get_param(const char *name);
const char *rbs_last_error(void);
const char *rbs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RBS_H */
