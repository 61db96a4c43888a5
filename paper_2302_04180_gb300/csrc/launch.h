// Host-side interface between the C ABI (capi.cu) and the kernel translation
// units. Plain C++; no kernel code here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rbs.h"

namespace rbs {

struct DotScratch;
struct SolverState;

struct CSRArgs {
    int64_t n, nnz;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
};

// SpMV row schedules (Cfg::mode): one thread per row, warp-staged chunks of
// up to SPMV_CAP_SHORT or SPMV_CAP_LONG nonzeros.
// Bit SPMV_TEST_STALL above the schedule bits selects the staged SpMV's test
// mode of its bounded wait (kernels.cuh).
enum : int { SPMV_MODE_ROW = 1, SPMV_MODE_SHORT = 2, SPMV_MODE_LONG = 3, SPMV_MODE_MASK = 0xff, SPMV_TEST_STALL = 0x100 };
// Long rows run register-staged in blocks of SPMV_REG_WARPS warps: the
// standalone SpMV, and the classic loop's fused K1/K3.
constexpr int SPMV_REG_WARPS = 4;

struct Cfg {
    int grid = 0;
    int block = 256;
    int mode = 2;       // SpMV row schedule (SPMV_MODE_*)
    int carveout = -1;  // shared-memory carveout percent, -1 = driver default
};

// Set the calling thread's rbs_last_error() message and return `code`.
int set_error(int code, const char *msg);
// Free the workspace of stream `s` on the current device (before the stream is destroyed).
void release_stream_workspace(cudaStream_t s);

// ---- standalone kernels (kernels_dot.cu: exact dots, limbs, FPE-8;
// kernels_spmv.cu: SpMV, Jacobi, CSR check) ----
cudaError_t launch_exdot(int k, const double *const *xs, const double *const *ys, int64_t n,
                         DotScratch *g, double *out, int window, Cfg cfg, cudaStream_t s);
cudaError_t launch_exdot_partial(const double *x, const double *y, int64_t n, DotScratch *g,
                                 int64_t *limbs, int32_t *flags, int window, Cfg cfg, cudaStream_t s);
cudaError_t launch_fpe_dot(const double *x, const double *y, int64_t n, DotScratch *g, double *out,
                           unsigned *lost, Cfg cfg, cudaStream_t s);
// Resident blocks per SM of the k-output exact-dot kernel (window Q) at this
// block size, for dots of length n (the kernel variant depends on it): the
// persistent grid is a whole number of waves of it.
int exdot_blocks_per_sm(int k, int window, int block, int64_t n);
// The same kernels with 1- and 2-limb register windows (kernels_exdot_w1.cu,
// kernels_exdot_w2.cu): launch and resident blocks per SM (smem: the
// shared-memory-window reducer of long one- and two-output dots).
cudaError_t launch_exdot_w1(int k, const double *const *xs, const double *const *ys, int64_t n, DotScratch *g,
                            double *out, Cfg cfg, cudaStream_t s);
cudaError_t launch_exdot_w2(int k, const double *const *xs, const double *const *ys, int64_t n, DotScratch *g,
                            double *out, Cfg cfg, cudaStream_t s);
int exdot_occ_w1(int k, int block, bool smem);
int exdot_occ_w2(int k, int block, bool smem);
int fpe_blocks_per_sm(int block);
cudaError_t launch_round_limbs(const int64_t *limbs, const int32_t *flags, double *out, cudaStream_t s);
// y = A x. Without a solver state every index is checked (ERR_INDEX on a bad
// one); with one, the solver has validated the structure and the kernel skips
// the checks (and does nothing once the solver has stopped).
cudaError_t launch_spmv(const CSRArgs &A, const double *x, double *y, const SolverState *st,
                        unsigned *err, Cfg cfg, cudaStream_t s);
cudaError_t launch_jacobi_invd(const CSRArgs &A, const double *diag, double *invd, unsigned *err,
                               Cfg cfg, cudaStream_t s);
cudaError_t launch_jacobi_apply(int64_t n, const double *invd, const double *p, double *phat, Cfg cfg,
                                cudaStream_t s);
cudaError_t launch_csr_check(const CSRArgs &A, unsigned *err, Cfg cfg, cudaStream_t s);

// ---- solver kernels (kernels_solver.cu) ----
struct SolverVecs {
    double *x, *r, *r0, *p, *ph, *s, *q, *qh, *y, *invd;  // classic (x, r, r0, q, qh, y, invd shared)
    double *rh, *w, *wh, *t, *sh, *z, *zh, *v;            // pipelined
};

struct SolverArgs {
    CSRArgs A;
    SolverVecs v;
    const double *b, *x0;
    SolverState *st;
    DotScratch *g;
    double *hist;
    unsigned *err;
    int dot_mode;
    int carveout;  // shared-memory carveout percent for staging kernels, -1 = driver default
    Cfg vec, spmv;
    Cfg p3;  // the pipelined P3 kernel, sized from its own occupancy
    Cfg k3;  // the classic K3 kernel (SpMV + two dots), sized from its own occupancy
};

// Kernel kinds for profiling (rbs_prof.kinds).
enum ProfKind { PK_K1 = 0, PK_VEC = 1, PK_SETUP = 2, PK_SPMV = 3, PK_VEC_DOT = 4, PK_K3 = 5, PK_K4 = 6 };

struct KernelTimer {
    virtual void before(int kind) = 0;
    virtual void after(int kind) = 0;
    virtual void gap() {}  // other work was enqueued since the last after()
    virtual ~KernelTimer() {}
};

cudaError_t solver_setup(const SolverArgs &a, int variant, cudaStream_t s, KernelTimer *t);
cudaError_t solver_iteration(const SolverArgs &a, int variant, cudaStream_t s, KernelTimer *t);

// Last node of the graph loop body: keeps the WHILE loop going while the stop
// flag is clear, and at most maxit + 1 bodies in any case.
cudaError_t launch_set_cond(cudaGraphConditionalHandle h, SolverState *st, cudaStream_t s);

// ---- batched solver (kernels_batch.cu) ----
struct BatchSys {
    CSRArgs A;
    const double *b, *x0, *diag;
    double *x;       // solution (device)
    double *work;    // 17 vector slots of `stride` doubles (9 for classic)
    int64_t stride;  // elements per slot
    double tol;
    int32_t maxit, variant;
    double *hist;    // device history records (hist_cap of them), may be null
    int32_t hist_cap, pad;
};
struct BatchOut {
    int32_t iters, converged, status;
    unsigned err;  // bit 0 invalid CSR, bit 1 zero/NaN/missing diagonal
    double tau0, tau_final, rho0, tau_max, alpha0, mu0;
};
cudaError_t launch_batch_prepare(const BatchSys *d_sys, int nsys, BatchOut *d_out, cudaStream_t s);
// Schedule of one batched launch: `clusters` clusters of `cluster` CTAs; a
// queued system with at least `split` unknowns is solved by a whole cluster,
// smaller ones by one CTA each.
struct BatchSchedule {
    int cluster, clusters;
    int64_t split;
};
cudaError_t launch_batch(const BatchSys *d_sys, const int32_t *d_order, const int64_t *d_sizes, int nsys,
                         unsigned *d_queue, BatchOut *d_out, BatchSchedule sched, cudaStream_t s);
// Clusters of `csize` CTAs that fit on the device at once (0 if none).
int batch_max_clusters(int csize);

// ---- per-step kernels of the serving engine (kernels_step.cu) ----
// One block of a per-step launch: rows [lo, hi) of the system in slot `sys`
// (lo even), which has nblk blocks in the launch.
struct StepTask {
    int32_t sys, nblk;
    int64_t lo, hi;
};
// Size of the device-side view of one system, and that view written to `out`
// (host memory, step_ctx_bytes() bytes): matrix, vectors (v.x is the caller's
// solution buffer, 16-byte aligned), right-hand side, optional x0 and Jacobi
// diagonal, the system's own state and dot scratch (zero at rest), and its
// device history records (nullable; state->hist_cap of them).
size_t step_ctx_bytes();
void step_ctx_make(void *out, const CSRArgs &A, const SolverVecs &v, const double *b, const double *x0,
                   const double *diag, SolverState *st, DotScratch *g, double *hist);
// Admission of new systems (all of one variant): structure check and Jacobi,
// then the set-up of Fig. 2 or Fig. 4; a system that fails its checks ends with
// status RBS_EINVAL and its error bits in its scratch's err word.
cudaError_t step_admit(const void *ctxs, const StepTask *tasks, int ntasks, int variant, cudaStream_t s);
// One iteration of every listed system (all of one variant); stopped systems skip it.
cudaError_t step_iteration(const void *ctxs, const StepTask *tasks, int ntasks, int variant, cudaStream_t s);

// occupancy-derived persistent grid for the kernels of one kind: which = 0 the
// SpMV kernels (classic K1, pipelined S10/S18), 1 the vector kernels, 2 the
// pipelined P3 kernel, 3 the classic K3 kernel
int solver_blocks_per_sm(int variant, int dot_mode, int which, int block, int carveout, int spmv_mode);
// Resident blocks per SM of the standalone SpMV kernel at this block size and
// shared-memory carveout (applies the carveout first).
int spmv_blocks_per_sm(int block, int carveout, int mode);

}  // namespace rbs
