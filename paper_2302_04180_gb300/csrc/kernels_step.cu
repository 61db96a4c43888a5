// Per-step kernels of the serving engine: one launch runs one phase of one
// iteration (Fig. 2 classic K1..K5, Fig. 4 pipelined P1..P4) for every system
// that is in flight at once. A launch is a list of tasks, one per block: a
// system (its Ctx in device memory) and a segment of its rows. Each block runs
// the same per-element functions as the per-solve kernels (solver_elem.cuh)
// over its segment; the exact dots of a system are reduced over that system's
// blocks only (its own scratch and ticket, nblk arrivals), and the system's
// last block runs the scalar tail on the system's own device state. Every
// system therefore gets the bits a solve of it alone gives, whatever else
// shares the launch, and a system that has stopped skips every later phase.
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "launch.h"
#include "solver_elem.cuh"
#include "tails.cuh"

namespace rbs {

namespace {

// The rows of a segment [lo, hi) as element pairs (2j, 2j+1) with 16-byte
// accesses (lo is even), then an odd last element in thread 0.
template <class F>
__device__ __forceinline__ void seg_pairs(int64_t lo, int64_t hi, F &&f) {
    for (int64_t i = lo + 2 * (int64_t)threadIdx.x; i + 1 < hi; i += 2 * (int64_t)blockDim.x) f(i, true);
    if (((hi - lo) & 1) && threadIdx.x == 0) f(hi - 1, false);
}

// y = A x over the block's segment with the warp-staged SpMV (structure
// validated at admission), epilogue fn(row, y_row, z_row).
template <class F>
__device__ __forceinline__ void seg_spmv(const Ctx &c, const StepTask &t, const double *x, const double *z,
                                         unsigned &err, F &&fn) {
    spmv_rows<false, SPMV_CAP_SHORT, false>(c.A, t.lo, t.hi, threadIdx.x >> 5, blockDim.x >> 5, x, z, true, false,
                                            err, fn);
}

constexpr int SCR = SpmvLayout<SPMV_CAP_SHORT>::SCRATCH;

// ---- admission ------------------------------------------------------------------

// Structure check and Jacobi set-up of the segment's rows: rowptr within
// [0, nnz] and non-decreasing, rowptr[0] = 0 and rowptr[n] = nnz, columns in
// [0, n) (error bit 1); invd_i = RN(1 / d_i) with d the given diagonal or the
// first stored (i, i) entry, a zero, NaN or missing one sets error bit 2 (the
// checks of the per-solve path).
__global__ void __launch_bounds__(256) k_step_prepare(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    const CSRView A = c.A;
    bool bad = false, bad_diag = false;
    if (threadIdx.x == 0 && t.lo == 0 && A.rowptr[0] != 0) bad = true;
    if (threadIdx.x == 0 && t.hi == A.n && A.rowptr[A.n] != A.nnz) bad = true;
    for (int64_t i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) {
        const int64_t b = A.rowptr[i], e = A.rowptr[i + 1];
        double d = 0.0;
        bool found = false;
        if (b < 0 || e < b || e > A.nnz) {
            bad = true;
        } else {
            for (int64_t k = b; k < e; k++) {
                const int32_t col = A.col[k];
                if ((uint64_t)(int64_t)col >= (uint64_t)A.n) bad = true;
                else if (!found && col == i) {
                    d = A.val[k];
                    found = true;
                }
            }
        }
        if (c.diag) {
            d = c.diag[i];
            found = true;
        }
        if (!found || d == 0.0 || d != d) {
            bad_diag = true;
            c.invd[i] = 0.0;
        } else {
            c.invd[i] = __ddiv_rn(1.0, d);
        }
    }
    if (bad) atomicOr(c.err, 1u);
    if (bad_diag) atomicOr(c.err, 2u);
}

// A system that failed its checks stops before its set-up (one thread per
// system: the one of its first task).
__global__ void k_step_validate(const Ctx *ctxs, const StepTask *tasks, int ntasks) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ntasks || tasks[j].lo != 0) return;
    const Ctx c = ctxs[tasks[j].sys];
    if (*c.err) {
        c.st->status = RBS_EINVAL;
        c.st->done = 1;
    }
}

// ---- classic (Fig. 2) -----------------------------------------------------------

template <class R>
__global__ void __launch_bounds__(256) k_step_cls_setup(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    bool bad = false;
    for (int64_t i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) red.add_sq(0, cls_setup_elem(c, i, bad));
    if (bad) atomicOr(c.err, 1u);
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals, t.nblk) && threadIdx.x == 0) tail_cls_setup(c.st, vals);
}

template <class R>
__global__ void __launch_bounds__(256, 3) k_step_cls_k1(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    unsigned eb = 0u;
    seg_spmv(c, t, c.ph, c.r0, eb, [&](int64_t i, double si, double r0) {
        c.s[i] = si;
        red.add(0, r0, si);
    });
    if (eb) atomicOr(c.err, eb);
    __shared__ double vals[R::K];
    if (red.template finish<SCR>(c.g, vals, t.nblk, !(eb & ERR_TIMEOUT)) && threadIdx.x == 0) tail_cls_alpha(c.st, vals);
}

__global__ void __launch_bounds__(256) k_step_cls_k2(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    const double na = -c.st->alpha;
    seg_pairs(t.lo, t.hi, [&](int64_t i, bool pair) {
        if (pair) {
            const double2 s = ld2(c.s, i), r = ld2(c.r, i), d = ld2(c.invd, i);
            const VPair u0 = cls_k2(na, s.x, r.x, d.x), u1 = cls_k2(na, s.y, r.y, d.y);
            st2(c.q, i, make_double2(u0.a, u1.a));
            st2(c.qh, i, make_double2(u0.b, u1.b));
        } else {
            const VPair u = cls_k2(na, c.s[i], c.r[i], c.invd[i]);
            c.q[i] = u.a;
            c.qh[i] = u.b;
        }
    });
}

template <class R>
__global__ void __launch_bounds__(256, 3) k_step_cls_k3(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    unsigned eb = 0u;
    seg_spmv(c, t, c.qh, c.q, eb, [&](int64_t i, double yi, double qi) {
        c.y[i] = yi;
        red.add(0, qi, yi);
        red.add_sq(1, yi);
    });
    if (eb) atomicOr(c.err, eb);
    __shared__ double vals[R::K];
    if (red.template finish<SCR>(c.g, vals, t.nblk, !(eb & ERR_TIMEOUT)) && threadIdx.x == 0) tail_cls_omega(c.st, vals);
}

template <class R>
__global__ void __launch_bounds__(256, 4) k_step_cls_k4(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    const double al = c.st->alpha, om = c.st->omega, nom = -om;
    seg_pairs(t.lo, t.hi, [&](int64_t i, bool pair) {
        if (pair) {
            const double2 qh = ld2(c.qh, i), ph = ld2(c.ph, i), y = ld2(c.y, i), q = ld2(c.q, i),
                          r0 = ld2(c.r0, i), x = ld2(c.x, i);
            const VPair u0 = cls_k4(al, om, nom, qh.x, ph.x, x.x, y.x, q.x);
            const VPair u1 = cls_k4(al, om, nom, qh.y, ph.y, x.y, y.y, q.y);
            st2(c.x, i, make_double2(u0.a, u1.a));
            st2(c.r, i, make_double2(u0.b, u1.b));
            red.add(0, r0.x, u0.b);
            red.add(0, r0.y, u1.b);
            red.add_sq(1, u0.b);
            red.add_sq(1, u1.b);
        } else {
            const VPair u = cls_k4(al, om, nom, c.qh[i], c.ph[i], c.x[i], c.y[i], c.q[i]);
            c.x[i] = u.a;
            c.r[i] = u.b;
            red.add(0, c.r0[i], u.b);
            red.add_sq(1, u.b);
        }
    });
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals, t.nblk) && threadIdx.x == 0) tail_cls_beta(c.st, vals, c.hist);
}

__global__ void __launch_bounds__(256) k_step_cls_k5(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    const double be = c.st->beta, nom = -c.st->omega;
    seg_pairs(t.lo, t.hi, [&](int64_t i, bool pair) {
        if (pair) {
            const double2 s = ld2(c.s, i), r = ld2(c.r, i), d = ld2(c.invd, i), p = ld2(c.p, i);
            const VPair u0 = cls_k5(be, nom, s.x, p.x, r.x, d.x), u1 = cls_k5(be, nom, s.y, p.y, r.y, d.y);
            st2(c.p, i, make_double2(u0.a, u1.a));
            st2(c.ph, i, make_double2(u0.b, u1.b));
        } else {
            const VPair u = cls_k5(be, nom, c.s[i], c.p[i], c.r[i], c.invd[i]);
            c.p[i] = u.a;
            c.ph[i] = u.b;
        }
    });
}

// ---- pipelined (Fig. 4) ---------------------------------------------------------

__global__ void __launch_bounds__(256) k_step_pipe_setup1(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    bool bad = false;
    for (int64_t i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) pipe_setup1_elem(c, i, bad);
    if (bad) atomicOr(c.err, 1u);
}

template <class R>
__global__ void __launch_bounds__(256, 3) k_step_pipe_setup2(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    unsigned eb = 0u;
    seg_spmv(c, t, c.rh, c.r0, eb, [&](int64_t i, double wi, double r0) {
        c.w[i] = wi;
        c.wh[i] = __dmul_rn(wi, c.invd[i]);
        red.add_sq(0, r0);  // r = r0 at set-up
        red.add(1, r0, wi);
    });
    if (eb) atomicOr(c.err, eb);
    __shared__ double vals[R::K];
    if (red.template finish<SCR>(c.g, vals, t.nblk, !(eb & ERR_TIMEOUT)) && threadIdx.x == 0) tail_pipe_setup(c.st, vals);
}

// y = A x without a dot: the pipelined S10 (v = A zhat) and S18 / set-up (t = A what)
template <bool TO_V>
__global__ void __launch_bounds__(256, 3) k_step_spmv(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    unsigned eb = 0u;
    double *y = TO_V ? c.v : c.t;
    seg_spmv(c, t, TO_V ? c.zh : c.wh, nullptr, eb, [&](int64_t i, double yi, double) { y[i] = yi; });
    if (eb) atomicOr(c.err, eb);
}

template <class R>
__global__ void __launch_bounds__(256, 3) k_step_pipe_p1(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    const double al = c.st->alpha, nal = -al, be = c.st->beta, nom = -c.st->omega;
    const bool first = c.st->iter == 0;
    for (int64_t i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x)
        p1_store(c, i, p1_elem(p1_load(c, i, first), first, nal, be, nom, red));
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals, t.nblk) && threadIdx.x == 0) tail_pipe_omega(c.st, vals);
}

template <class R>
__global__ void __launch_bounds__(256, 2) k_step_pipe_p3(const Ctx *ctxs, const StepTask *tasks) {
    const StepTask t = tasks[blockIdx.x];
    const Ctx c = ctxs[t.sys];
    if (c.st->done) return;
    R red;
    red.init();
    const double al = c.st->alpha, nal = -al, om = c.st->omega, nom = -om;
    for (int64_t i = t.lo + threadIdx.x; i < t.hi; i += blockDim.x) {
        const P3Out o = p3_elem(P3In{c.qh[i], c.y[i], c.q[i], c.ph[i], c.x[i], c.zh[i], c.wh[i], c.v[i], c.t[i],
                                     c.invd[i], c.r0[i], c.s[i], c.z[i]},
                                al, nal, om, nom, red);
        c.x[i] = o.x;
        c.r[i] = o.r;
        c.rh[i] = o.rh;
        c.w[i] = o.w;
        c.wh[i] = o.wh;
    }
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals, t.nblk) && threadIdx.x == 0) tail_pipe_beta(c.st, vals, c.hist);
}

using R1 = ExactR<1, SQ>;
using R2 = ExactR<2, SQ>;
using R5 = ExactR<5, SQ>;

void step_carveout() {
    static std::once_flag once;
    std::call_once(once, [] {
        const int c = 75;  // as the per-solve staging kernels: three blocks per SM, L1 left for the gathers
        cudaFuncSetAttribute(k_step_cls_k1<R1>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        cudaFuncSetAttribute(k_step_cls_k3<R2>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        cudaFuncSetAttribute(k_step_pipe_setup2<R2>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        cudaFuncSetAttribute(k_step_spmv<true>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        cudaFuncSetAttribute(k_step_spmv<false>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        cudaGetLastError();
    });
}

}  // namespace

void step_ctx_make(void *out, const CSRArgs &A, const SolverVecs &v, const double *b, const double *x0,
                   const double *diag, SolverState *st, DotScratch *g, double *hist) {
    Ctx c;
    memset(&c, 0, sizeof c);
    c.A = CSRView{A.n, A.nnz, A.rowptr, A.col, A.val};
    c.n = A.n;
    c.x = v.x; c.r = v.r; c.r0 = v.r0; c.p = v.p; c.ph = v.ph; c.s = v.s; c.q = v.q; c.qh = v.qh;
    c.y = v.y; c.invd = v.invd; c.rh = v.rh; c.w = v.w; c.wh = v.wh; c.t = v.t; c.sh = v.sh;
    c.z = v.z; c.zh = v.zh; c.v = v.v;
    c.b = b;
    c.x0 = x0;
    c.diag = diag;
    c.st = st;
    c.g = g;
    c.hist = hist;
    c.err = &g->err;
    c.spmv_mode = SPMV_MODE_SHORT;
    memcpy(out, &c, sizeof c);
}

size_t step_ctx_bytes() { return sizeof(Ctx); }

cudaError_t step_admit(const void *ctxs, const StepTask *tasks, int ntasks, int variant, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    step_carveout();
    const Ctx *c = static_cast<const Ctx *>(ctxs);
    k_step_prepare<<<ntasks, 256, 0, s>>>(c, tasks);
    k_step_validate<<<(ntasks + 255) / 256, 256, 0, s>>>(c, tasks, ntasks);
    if (variant == RBS_CLASSIC) {
        k_step_cls_setup<R1><<<ntasks, 256, 0, s>>>(c, tasks);
    } else {
        k_step_pipe_setup1<<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_pipe_setup2<R2><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_spmv<false><<<ntasks, 256, 0, s>>>(c, tasks);
    }
    return cudaGetLastError();
}

cudaError_t step_iteration(const void *ctxs, const StepTask *tasks, int ntasks, int variant, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    step_carveout();
    const Ctx *c = static_cast<const Ctx *>(ctxs);
    if (variant == RBS_CLASSIC) {
        k_step_cls_k1<R1><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_cls_k2<<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_cls_k3<R2><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_cls_k4<R2><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_cls_k5<<<ntasks, 256, 0, s>>>(c, tasks);
    } else {
        k_step_pipe_p1<R2><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_spmv<true><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_pipe_p3<R5><<<ntasks, 256, 0, s>>>(c, tasks);
        k_step_spmv<false><<<ntasks, 256, 0, s>>>(c, tasks);
    }
    return cudaGetLastError();
}

}  // namespace rbs
