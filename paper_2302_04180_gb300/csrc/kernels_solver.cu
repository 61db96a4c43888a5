// Fused kernels of the classic (Fig. 2) and pipelined (Fig. 4) PBiCGStab
// loops, with device-resident scalars. Every dot rides in the epilogue of the
// kernel that produces its operands, and the block that finishes a reduction
// last computes the scalar recurrence (alpha, omega, beta, tau, stop test) in
// place, so the host never sits between two steps.
//
// Classic iteration (5 launches):
//   K1  s = A phat, <r0,s>                      -> alpha          (S2, S3)
//   K2  q = fma(-alpha, s, r), qhat = q*invd                        (S4, S5)
//   K3  y = A qhat, <q,y>, <y,y>                -> omega          (S6, S7)
//   K4  x = fma(omega, qhat, fma(alpha, phat, x)), r = fma(-omega, y, q),
//       <r0,r>, <r,r>                           -> tau, stop, beta (S8-S11, S10)
//   K5  p = fma(beta, fma(-omega, s, p), r), phat = p*invd        (S12, S1)
// Pipelined iteration (4 launches):
//   P1  S1-S7 and S9 element-wise, <q,y>, <y,y>  -> omega          (S1-S9, S11)
//   P2  v = A zhat                                                  (S10)
//   P3  S12-S15 and S17 element-wise, <r0,r>, <r0,w>, <r0,s>, <r0,z>, <r,r>
//                                                -> tau, stop, beta, alpha (S16, S19)
//   P4  t = A what                                                  (S18)
// Once the stop flag is set, every later kernel returns at once.
#include <mutex>

#include "kernels.cuh"

#include "launch.h"
#include "solver_elem.cuh"
#include "tails.cuh"

namespace rbs {

// ---- classic kernels -------------------------------------------------------------

// set-up: r = b - A x0 (or b), x = x0 (or +0), r0 = p = r, phat = r*invd, <r0,r0>
template <class R>
__global__ void __launch_bounds__(256) k_cls_setup(Ctx c) {
    R red;
    red.init();
    bool bad = false;
    for (int64_t i = gtid(); i < c.n; i += gstride()) {
        const double ri = cls_setup_elem(c, i, bad);
        red.add_sq(0, ri);
    }
    if (bad) atomicOr(c.err, 1u);
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals) && threadIdx.x == 0) tail_cls_setup(c.st, vals);
}

// SpMV rows of the fused K1/K3 with epilogue fn(row, y_row, z_row): short
// rows warp-staged (or one thread per row, mode 1) in 256-thread blocks; long
// rows (CAP = SPMV_CAP_LONG) register-staged in blocks of SPMV_REG_WARPS warps.
// Finish the kernel's reducer with finish<FusedScratch<CAP>::BYTES,
// FusedScratch<CAP>::WARPS>, so that its flush reuses the staging buffer.
template <int CAP>
struct FusedScratch {
    static constexpr bool REG = CAP > SPMV_CAP_SHORT;
    static constexpr int BYTES = REG ? SpmvLayout<CAP>::BUF : SpmvLayout<CAP>::SCRATCH;
    static constexpr int WARPS = REG ? SPMV_REG_WARPS : MAX_WARPS;
    static constexpr int THREADS = WARPS * 32;
};
template <int CAP, class F>
__device__ __forceinline__ void fused_spmv(const Ctx &c, const double *x, const double *z, unsigned &eb, F &&fn) {
    if (FusedScratch<CAP>::REG)
        spmv_rows_reg<false, CAP, false>(c.A, 0, c.A.n, (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                                         (int64_t)gridDim.x * (blockDim.x >> 5), x, z, true,
                                         (c.spmv_mode & SPMV_TEST_STALL) != 0, eb, fn);
    else
        spmv_each<false, CAP>(c.A, x, z, c.spmv_mode, eb, fn);
}

// K1: s = A phat, <r0, s>
template <class R, int CAP>
__global__ void __launch_bounds__(FusedScratch<CAP>::THREADS, 3) k_cls_k1(Ctx c) {
    if (c.st->done) return;
    R red;
    red.init();
    unsigned eb = 0u;
    fused_spmv<CAP>(c, c.ph, c.r0, eb, [&](int64_t i, double si, double r0) {
        c.s[i] = si;
        red.add(0, r0, si);
    });
    if (eb) atomicOr(c.err, eb);
    __shared__ double vals[R::K];
    if (red.template finish<FusedScratch<CAP>::BYTES, FusedScratch<CAP>::WARPS>(c.g, vals, 0u,
                                                                               !(eb & ERR_TIMEOUT)) &&
        threadIdx.x == 0)
        tail_cls_alpha(c.st, vals);
}

// K2: q = fma(-alpha, s, r), qhat = q * invd. Four blocks per SM, like K4, whose
// occupancy sizes the vector grid: left free, the compiler took 80 registers, three
// blocks fit and the grid ran in 1.33 waves.
__global__ void __launch_bounds__(256, 4) k_cls_k2(Ctx c) {
    if (c.st->done) return;
    const double na = -c.st->alpha;
    for_pairs(c.n, [&](int64_t i, bool pair) {
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

// K3: y = A qhat, <q, y>, <y, y>
template <class R, int CAP>
__global__ void __launch_bounds__(FusedScratch<CAP>::THREADS, 3) k_cls_k3(Ctx c) {
    if (c.st->done) return;
    R red;
    red.init();
    unsigned eb = 0u;
    fused_spmv<CAP>(c, c.qh, c.q, eb, [&](int64_t i, double yi, double qi) {
        c.y[i] = yi;
        red.add(0, qi, yi);
        red.add_sq(1, yi);
    });
    if (eb) atomicOr(c.err, eb);
    __shared__ double vals[R::K];
    if (red.template finish<FusedScratch<CAP>::BYTES, FusedScratch<CAP>::WARPS>(c.g, vals, 0u,
                                                                               !(eb & ERR_TIMEOUT)) &&
        threadIdx.x == 0)
        tail_cls_omega(c.st, vals);
}

// K4: x = fma(omega, qhat, fma(alpha, phat, x)), r = fma(-omega, y, q), <r0,r>, <r,r>
template <class R>
__global__ void __launch_bounds__(256) k_cls_k4(Ctx c) {
    if (c.st->done) return;
    R red;
    red.init();
    const double al = c.st->alpha, om = c.st->omega, nom = -om;
    for_pairs(c.n, [&](int64_t i, bool pair) {
        if (pair) {
            const double2 qh = ld2(c.qh, i), ph = ld2(c.ph, i), y = ld2(c.y, i), q = ld2(c.q, i),
                          r0 = ld2(c.r0, i);
            const double2 x = ld2(c.x, i);
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
    if (red.finish(c.g, vals) && threadIdx.x == 0) tail_cls_beta(c.st, vals, c.hist);
}

// K5: p = fma(beta, fma(-omega, s, p), r), phat = p * invd
__global__ void __launch_bounds__(256) k_cls_k5(Ctx c) {
    if (c.st->done) return;
    const double be = c.st->beta, nom = -c.st->omega;
    for_pairs(c.n, [&](int64_t i, bool pair) {
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

// ---- pipelined kernels -------------------------------------------------------------

// set-up 1: r = b - A x0 (or b), x, r0 = r, rhat = r * invd
__global__ void __launch_bounds__(256) k_pipe_setup1(Ctx c) {
    bool bad = false;
    for (int64_t i = gtid(); i < c.n; i += gstride()) pipe_setup1_elem(c, i, bad);
    if (bad) atomicOr(c.err, 1u);
}

// set-up 2: w = A rhat, what = w * invd, <r0,r>, <r0,w> -> alpha0
template <class R, int CAP>
__global__ void __launch_bounds__(256, CAP > SPMV_CAP_SHORT ? 1 : 3) k_pipe_setup2(Ctx c) {
    R red;
    red.init();
    unsigned eb = 0u;
    spmv_each<false, CAP>(c.A, c.rh, c.r0, c.spmv_mode, eb, [&](int64_t i, double wi, double r0) {
        c.w[i] = wi;
        c.wh[i] = __dmul_rn(wi, c.invd[i]);
        red.add_sq(0, r0);  // r = r0 at set-up
        red.add(1, r0, wi);
    });
    if (eb) atomicOr(c.err, eb);
    __shared__ double vals[R::K];
    if (red.template finish<SpmvLayout<CAP>::SCRATCH>(c.g, vals, 0u, !(eb & ERR_TIMEOUT)) && threadIdx.x == 0)
        tail_pipe_setup(c.st, vals);
}

// Launch shape of P1 and P3 per reducer (blocks per SM; two elements per thread
// with 16-byte accesses or one), the fastest measured on Poisson 256^3. With the
// exact reducer, pairs issue twice the loads per thread and lower occupancy
// keeps the dot windows in registers: P3 at two blocks uses 121 registers, no
// spills, where four blocks spilled the five windows; P1 is best at three.
template <class R> struct P1Cfg { static constexpr int blocks = 3, pairs = 1; };
template <int K> struct P1Cfg<PlainR<K>> { static constexpr int blocks = 4, pairs = 0; };

// P1: S1-S4 (copies at iteration 0), S5-S7, S9; <q,y>, <y,y> -> omega.
// Every operand of an element is loaded before its first store (the vectors are
// not restrict-qualified, so later loads could not be issued early).
template <class R>
__global__ void __launch_bounds__(256, P1Cfg<R>::blocks) k_pipe_p1(Ctx c) {
    if (c.st->done) return;
    R red;
    red.init();
    const double al = c.st->alpha, nal = -al, be = c.st->beta, nom = -c.st->omega;
    const bool first = c.st->iter == 0;
    if (P1Cfg<R>::pairs) {
        for_pairs(c.n, [&](int64_t i, bool pair) {
            if (pair) {
                const double2 rh = ld2(c.rh, i), w = ld2(c.w, i), wh = ld2(c.wh, i), t = ld2(c.t, i),
                              r = ld2(c.r, i), d = ld2(c.invd, i);
                double2 ph{0.0, 0.0}, s{0.0, 0.0}, sh{0.0, 0.0}, z{0.0, 0.0}, zh{0.0, 0.0}, v{0.0, 0.0};
                if (!first) {
                    ph = ld2(c.ph, i);
                    s = ld2(c.s, i);
                    sh = ld2(c.sh, i);
                    z = ld2(c.z, i);
                    zh = ld2(c.zh, i);
                    v = ld2(c.v, i);
                }
                const P1Out o0 = p1_elem(P1In{rh.x, w.x, wh.x, t.x, r.x, d.x, ph.x, s.x, sh.x, z.x, zh.x, v.x}, first,
                                         nal, be, nom, red);
                const P1Out o1 = p1_elem(P1In{rh.y, w.y, wh.y, t.y, r.y, d.y, ph.y, s.y, sh.y, z.y, zh.y, v.y}, first,
                                         nal, be, nom, red);
                st2(c.ph, i, make_double2(o0.ph, o1.ph));
                st2(c.s, i, make_double2(o0.s, o1.s));
                st2(c.sh, i, make_double2(o0.sh, o1.sh));
                st2(c.z, i, make_double2(o0.z, o1.z));
                st2(c.q, i, make_double2(o0.q, o1.q));
                st2(c.qh, i, make_double2(o0.qh, o1.qh));
                st2(c.y, i, make_double2(o0.y, o1.y));
                st2(c.zh, i, make_double2(o0.zh, o1.zh));
            } else {
                p1_store(c, i, p1_elem(p1_load(c, i, first), first, nal, be, nom, red));
            }
        });
    } else {
        for (int64_t i = gtid(); i < c.n; i += gstride())
            p1_store(c, i, p1_elem(p1_load(c, i, first), first, nal, be, nom, red));
    }
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals) && threadIdx.x == 0) tail_pipe_omega(c.st, vals);
}

// (P3's launch shape: see P1Cfg.)
template <class R> struct P3Cfg { static constexpr int blocks = 2, pairs = 1; };
template <int K> struct P3Cfg<PlainR<K>> { static constexpr int blocks = 3, pairs = 0; };

// P3: S12-S15, S17; <r0,r>, <r0,w>, <r0,s>, <r0,z>, <r,r> -> tau, beta, alpha.
// Every operand of an element is loaded before its first store (the vectors are
// not restrict-qualified, so later loads could not be issued early).
template <class R>
__global__ void __launch_bounds__(256, P3Cfg<R>::blocks) k_pipe_p3(Ctx c) {
    if (c.st->done) return;
    R red;
    red.init();
    const double al = c.st->alpha, nal = -al, om = c.st->omega, nom = -om;
    if (P3Cfg<R>::pairs) {
        for_pairs(c.n, [&](int64_t i, bool pair) {
            if (pair) {
                const double2 qh = ld2(c.qh, i), y = ld2(c.y, i), q = ld2(c.q, i), ph = ld2(c.ph, i),
                              x = ld2(c.x, i), zh = ld2(c.zh, i), wh = ld2(c.wh, i), v = ld2(c.v, i),
                              t = ld2(c.t, i), d = ld2(c.invd, i), r0 = ld2(c.r0, i), s = ld2(c.s, i),
                              z = ld2(c.z, i);
                const P3Out o0 = p3_elem(P3In{qh.x, y.x, q.x, ph.x, x.x, zh.x, wh.x, v.x, t.x, d.x, r0.x, s.x, z.x},
                                         al, nal, om, nom, red);
                const P3Out o1 = p3_elem(P3In{qh.y, y.y, q.y, ph.y, x.y, zh.y, wh.y, v.y, t.y, d.y, r0.y, s.y, z.y},
                                         al, nal, om, nom, red);
                st2(c.x, i, make_double2(o0.x, o1.x));
                st2(c.r, i, make_double2(o0.r, o1.r));
                st2(c.rh, i, make_double2(o0.rh, o1.rh));
                st2(c.w, i, make_double2(o0.w, o1.w));
                st2(c.wh, i, make_double2(o0.wh, o1.wh));
            } else {
                const P3Out o = p3_elem(P3In{c.qh[i], c.y[i], c.q[i], c.ph[i], c.x[i], c.zh[i], c.wh[i], c.v[i],
                                             c.t[i], c.invd[i], c.r0[i], c.s[i], c.z[i]},
                                        al, nal, om, nom, red);
                c.x[i] = o.x;
                c.r[i] = o.r;
                c.rh[i] = o.rh;
                c.w[i] = o.w;
                c.wh[i] = o.wh;
            }
        });
    } else {
        for (int64_t i = gtid(); i < c.n; i += gstride()) {
            const P3Out o = p3_elem(P3In{c.qh[i], c.y[i], c.q[i], c.ph[i], c.x[i], c.zh[i], c.wh[i], c.v[i], c.t[i],
                                         c.invd[i], c.r0[i], c.s[i], c.z[i]},
                                    al, nal, om, nom, red);
            c.x[i] = o.x;
            c.r[i] = o.r;
            c.rh[i] = o.rh;
            c.w[i] = o.w;
            c.wh[i] = o.wh;
        }
    }
    __shared__ double vals[R::K];
    if (red.finish(c.g, vals) && threadIdx.x == 0) tail_pipe_beta(c.st, vals, c.hist);
}

// ---- launch -----------------------------------------------------------------------

static Ctx make_ctx(const SolverArgs &a) {
    Ctx c;
    c.A = CSRView{a.A.n, a.A.nnz, a.A.rowptr, a.A.col, a.A.val};
    c.n = a.A.n;
    c.x = a.v.x; c.r = a.v.r; c.r0 = a.v.r0; c.p = a.v.p; c.ph = a.v.ph; c.s = a.v.s;
    c.q = a.v.q; c.qh = a.v.qh; c.y = a.v.y; c.invd = a.v.invd;
    c.rh = a.v.rh; c.w = a.v.w; c.wh = a.v.wh; c.t = a.v.t; c.sh = a.v.sh; c.z = a.v.z;
    c.zh = a.v.zh; c.v = a.v.v;
    c.b = a.b; c.x0 = a.x0; c.diag = nullptr; c.st = a.st; c.g = a.g; c.hist = a.hist; c.err = a.err;
    c.spmv_mode = a.spmv.mode;
    return c;
}

#define TIMED(kind, launch)             \
    do {                                \
        if (tm) tm->before(kind);       \
        launch;                         \
        if (tm) tm->after(kind);        \
    } while (0)

template <class R1, class R2, class R5>
static cudaError_t setup_t(const SolverArgs &a, int variant, cudaStream_t s, KernelTimer *tm) {
    Ctx c = make_ctx(a);
    if (variant == RBS_CLASSIC) {
        TIMED(PK_SETUP, (k_cls_setup<R1><<<a.vec.grid, a.vec.block, 0, s>>>(c)));
    } else {
        TIMED(PK_SETUP, (k_pipe_setup1<<<a.vec.grid, a.vec.block, 0, s>>>(c)));
        if ((a.spmv.mode & SPMV_MODE_MASK) == SPMV_MODE_LONG)
            TIMED(PK_SETUP, (k_pipe_setup2<R2, SPMV_CAP_LONG><<<a.spmv.grid, a.spmv.block, 0, s>>>(c)));
        else
            TIMED(PK_SETUP, (k_pipe_setup2<R2, SPMV_CAP_SHORT><<<a.spmv.grid, a.spmv.block, 0, s>>>(c)));
        TIMED(PK_SETUP, (launch_spmv(a.A, a.v.wh, a.v.t, a.st, a.err, a.spmv, s)));
    }
    return cudaGetLastError();
}

template <class R1, class R2, class R5>
static cudaError_t iter_t(const SolverArgs &a, int variant, cudaStream_t s, KernelTimer *tm) {
    Ctx c = make_ctx(a);
    if (variant == RBS_CLASSIC) {
        const bool lng = (a.spmv.mode & SPMV_MODE_MASK) == SPMV_MODE_LONG;
        if (lng) TIMED(PK_K1, (k_cls_k1<R1, SPMV_CAP_LONG><<<a.spmv.grid, a.spmv.block, 0, s>>>(c)));
        else TIMED(PK_K1, (k_cls_k1<R1, SPMV_CAP_SHORT><<<a.spmv.grid, a.spmv.block, 0, s>>>(c)));
        TIMED(PK_VEC, (k_cls_k2<<<a.vec.grid, a.vec.block, 0, s>>>(c)));
        if (lng) TIMED(PK_K3, (k_cls_k3<R2, SPMV_CAP_LONG><<<a.k3.grid, a.k3.block, 0, s>>>(c)));
        else TIMED(PK_K3, (k_cls_k3<R2, SPMV_CAP_SHORT><<<a.k3.grid, a.k3.block, 0, s>>>(c)));
        TIMED(PK_K4, (k_cls_k4<R2><<<a.vec.grid, a.vec.block, 0, s>>>(c)));
        TIMED(PK_VEC, (k_cls_k5<<<a.vec.grid, a.vec.block, 0, s>>>(c)));
    } else {
        TIMED(PK_VEC_DOT, (k_pipe_p1<R2><<<a.vec.grid, a.vec.block, 0, s>>>(c)));
        TIMED(PK_SPMV, (launch_spmv(a.A, a.v.zh, a.v.v, a.st, a.err, a.spmv, s)));
        TIMED(PK_VEC_DOT, (k_pipe_p3<R5><<<a.p3.grid, a.p3.block, 0, s>>>(c)));
        TIMED(PK_SPMV, (launch_spmv(a.A, a.v.wh, a.v.t, a.st, a.err, a.spmv, s)));
    }
    return cudaGetLastError();
}

// Shared-memory carveout (percent of the unified L1/shared storage, -1 = the
// driver's choice) of the kernels that stage data per warp. The x gathers of
// the SpMV live on L1 hits, so the split is a tuning knob, not a maximum.
template <class R1, class R2, class R5>
static void prefer_shared(int c) {
    cudaFuncSetAttribute(k_cls_k1<R1, SPMV_CAP_SHORT>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
    cudaFuncSetAttribute(k_cls_k3<R2, SPMV_CAP_SHORT>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
    cudaFuncSetAttribute(k_cls_k4<R2>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
    cudaFuncSetAttribute(k_pipe_setup2<R2, SPMV_CAP_SHORT>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
    // the long-row kernels need (nearly) all of it for their staging buffers
    const int cl = c < 0 ? c : 100;
    cudaFuncSetAttribute(k_cls_k1<R1, SPMV_CAP_LONG>, cudaFuncAttributePreferredSharedMemoryCarveout, cl);
    cudaFuncSetAttribute(k_cls_k3<R2, SPMV_CAP_LONG>, cudaFuncAttributePreferredSharedMemoryCarveout, cl);
    cudaFuncSetAttribute(k_pipe_setup2<R2, SPMV_CAP_LONG>, cudaFuncAttributePreferredSharedMemoryCarveout, cl);
    cudaFuncSetAttribute(k_pipe_p1<R2>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
    cudaFuncSetAttribute(k_pipe_p3<R5>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
    cudaGetLastError();
}

// Apply the carveout to this device's kernels once per value. It must come
// before any occupancy query, which depends on it.
static void apply_carveout(int dot_mode, int c) {
    static std::mutex mu;
    static int applied_exact[64], applied_plain[64];
    static bool init = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!init) {
        for (int i = 0; i < 64; i++) applied_exact[i] = applied_plain[i] = -2;
        init = true;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    if (dot_mode == RBS_DOT_PLAIN && applied_plain[dev] != c) {
        prefer_shared<PlainR<1>, PlainR<2>, PlainR<5>>(c);
        applied_plain[dev] = c;
    } else if (dot_mode != RBS_DOT_PLAIN && applied_exact[dev] != c) {
        prefer_shared<ExactR<1, SQ>, ExactR<2, SQ>, ExactR<5, SQ>>(c);
        applied_exact[dev] = c;
    }
}

cudaError_t solver_setup(const SolverArgs &a, int variant, cudaStream_t s, KernelTimer *t) {
    apply_carveout(a.dot_mode, a.carveout);
    if (a.dot_mode == RBS_DOT_PLAIN) return setup_t<PlainR<1>, PlainR<2>, PlainR<5>>(a, variant, s, t);
    return setup_t<ExactR<1, SQ>, ExactR<2, SQ>, ExactR<5, SQ>>(a, variant, s, t);
}

cudaError_t solver_iteration(const SolverArgs &a, int variant, cudaStream_t s, KernelTimer *t) {
    if (a.dot_mode == RBS_DOT_PLAIN) return iter_t<PlainR<1>, PlainR<2>, PlainR<5>>(a, variant, s, t);
    return iter_t<ExactR<1, SQ>, ExactR<2, SQ>, ExactR<5, SQ>>(a, variant, s, t);
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, SolverState *st) {
    const int loops = st->loops + 1;
    st->loops = loops;
    cudaGraphSetConditional(h, (!st->done && loops <= st->maxit + 1) ? 1u : 0u);
}

cudaError_t launch_set_cond(cudaGraphConditionalHandle h, SolverState *st, cudaStream_t s) {
    k_set_cond<<<1, 1, 0, s>>>(h, st);
    return cudaGetLastError();
}

int solver_blocks_per_sm(int variant, int dot_mode, int which, int block, int carveout, int spmv_mode) {
    apply_carveout(dot_mode, carveout);
    if (which == 0 && variant == RBS_PIPELINED) return spmv_blocks_per_sm(block, carveout, spmv_mode);
    const bool lng = spmv_mode == SPMV_MODE_LONG;
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (dot_mode == RBS_DOT_PLAIN) {
        using R1 = PlainR<1>;
        using R2 = PlainR<2>;
        if (which == 0) {
            e = lng ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k1<R1, SPMV_CAP_LONG>, block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k1<R1, SPMV_CAP_SHORT>, block, 0);
        } else if (which == 3) {
            e = lng ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k3<R2, SPMV_CAP_LONG>, block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k3<R2, SPMV_CAP_SHORT>, block, 0);
        } else if (variant == RBS_PIPELINED) {
            e = which == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pipe_p3<PlainR<5>>, block, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pipe_p1<R2>, block, 0);
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k4<R2>, block, 0);
        }
    } else {
        using R1 = ExactR<1, SQ>;
        using R2 = ExactR<2, SQ>;
        if (which == 0) {
            e = lng ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k1<R1, SPMV_CAP_LONG>, block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k1<R1, SPMV_CAP_SHORT>, block, 0);
        } else if (which == 3) {
            e = lng ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k3<R2, SPMV_CAP_LONG>, block, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k3<R2, SPMV_CAP_SHORT>, block, 0);
        } else if (variant == RBS_PIPELINED) {
            e = which == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pipe_p3<ExactR<5, SQ>>, block, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pipe_p1<R2>, block, 0);
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cls_k4<R2>, block, 0);
        }
    }
    if (e != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

}  // namespace rbs
