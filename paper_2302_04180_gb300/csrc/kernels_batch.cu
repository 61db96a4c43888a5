// Batched solver: many independent systems in one persistent launch.
//
// The launch is made of thread-block clusters of C CTAs (C chosen at launch:
// 1, 2, 4, 8 or 16). Systems come from a queue ordered largest first. While
// the next system has at least `split` unknowns, a whole cluster solves it:
// the rows are split across the cluster's CTAs, element-wise steps touch only a
// CTA's own rows, the SpMV gathers x from the whole vector, and every exact dot
// is reduced across the cluster through distributed shared memory. From the
// first smaller system on, the cluster's CTAs work alone, each taking its own
// systems from the queue and solving them with CTA barriers only, so small
// systems do not pay for cluster barriers and every SM stays busy to the end.
// Every group (cluster or CTA) rounds the group-summed integers itself and
// runs the same scalar recurrence on the same bits, so all its CTAs take the
// same decisions and meet the same barriers; no CTA ever spins on a flag.
// Arithmetic, fma forms and readings are those of the per-step kernels, so a
// system's result is bitwise the one rbs_solve gives, whatever the schedule.
#include <cooperative_groups.h>
#include <mutex>

#include "kernels.cuh"
#include "launch.h"
#include "tails.cuh"

namespace cg = cooperative_groups;

namespace rbs {

constexpr int BMAX = 16;  // most CTAs per cluster (non-portable size)
constexpr int BQ = 4;  // exact-dot window placements

enum Slot { S_R, S_R0, S_P, S_PH, S_S, S_Q, S_QH, S_Y, S_INVD, S_RH, S_W, S_WH, S_T, S_SH, S_Z, S_ZH, S_V };

// y_i for row i, fma chain in stored order from +0.0 (as spmv_row), with x
// read through L2: other CTAs of the cluster wrote it inside this kernel.
__device__ __forceinline__ double spmv_row_l2(const CSRView &A, int64_t i, const double *x, bool &bad) {
    const int64_t b = A.rowptr[i], e = A.rowptr[i + 1];
    double acc = 0.0;
    if (b < 0 || e < b || e > A.nnz) {
        bad = true;
        return acc;
    }
    for (int64_t k0 = b; k0 < e; k0 += 8) {
        double xv[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            xv[j] = 0.0;
            if (k0 + j < e) {
                const int32_t c = A.col[k0 + j];
                if ((uint64_t)(int64_t)c < (uint64_t)A.n) xv[j] = __ldcg(x + c);
                else bad = true;
            }
        }
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (k0 + j < e && (uint64_t)(int64_t)A.col[k0 + j] < (uint64_t)A.n)
                acc = fma(A.val[k0 + j], xv[j], acc);
    }
    return acc;
}

struct ClusterRed {
    unsigned long long (*acc)[NL];  // this CTA's accumulators (shared)
    long long (*red)[NL];           // group sums (shared)
    uint32_t *flags, *rflags;
    double *vals;
};

// The CTAs that solve one system together: the whole cluster, or one CTA.
struct Grp {
    cg::cluster_group *cl;  // null for a CTA working alone
    unsigned rank, size;
    __device__ __forceinline__ void sync() const {
        if (cl) cl->sync();
        else __syncthreads();
    }
};

// Reduce K exact dots across the group; afterwards vals[0..K-1] hold the
// rounded dots in every CTA of the group and the accumulators are zero again.
template <int K>
__device__ __forceinline__ void group_reduce(const Grp &g, Win<BQ> (&win)[K], uint32_t (&fl)[K],
                                             const ClusterRed &R) {
#pragma unroll
    for (int k = 0; k < K; k++) {
        warp_flush<BQ, FLUSH_SCRATCH>(win[k], R.acc[k]);
        if (fl[k]) atomicOr(&R.flags[k], fl[k]);
        fl[k] = 0u;
    }
    g.sync();
    for (int idx = threadIdx.x; idx < K * NL; idx += blockDim.x) {
        long long sum = 0;
        if (g.cl) {
            for (unsigned r = 0; r < g.size; r++) sum += (long long)*g.cl->map_shared_rank(&R.acc[0][0] + idx, r);
        } else {
            sum = (long long)(&R.acc[0][0])[idx];
        }
        (&R.red[0][0])[idx] = sum;
    }
    if (threadIdx.x < K) {
        uint32_t f = 0u;
        if (g.cl) {
            for (unsigned r = 0; r < g.size; r++) f |= *g.cl->map_shared_rank(R.flags + threadIdx.x, r);
        } else {
            f = R.flags[threadIdx.x];
        }
        R.rflags[threadIdx.x] = f;
    }
    g.sync();
    for (int idx = threadIdx.x; idx < K * NL; idx += blockDim.x) (&R.acc[0][0])[idx] = 0ull;
    if (threadIdx.x < K) {
        R.flags[threadIdx.x] = 0u;
        R.vals[threadIdx.x] = round_limbs_thread(R.red[threadIdx.x], R.rflags[threadIdx.x]);
    }
    __syncthreads();
}

struct SysView {
    CSRView A;
    int64_t n, lo, hi;
    double *v[17];
    double *x;
    const double *b, *x0;
    double *hist;
};

__device__ __forceinline__ void sys_view(const BatchSys &S, const Grp &g, SysView &V) {
    V.A = CSRView{S.A.n, S.A.nnz, S.A.rowptr, S.A.col, S.A.val};
    V.n = S.A.n;
    V.lo = V.n * (int64_t)g.rank / g.size;
    V.hi = V.n * (int64_t)(g.rank + 1) / g.size;
    for (int k = 0; k < 17; k++) V.v[k] = S.work + (int64_t)k * S.stride;
    V.x = S.x;
    V.b = S.b;
    V.x0 = S.x0;
    V.hist = S.hist;
}

#define OWN_ROWS(i) for (int64_t i = V.lo + threadIdx.x; i < V.hi; i += blockDim.x)

template <int N>
struct Vals {
    double v[N];
};

// This CTA's rows, two per thread per pass: ld(i) returns the values row i
// needs and st(i, vals) computes and stores; both rows' loads are issued
// before the first store, so twice the bytes are in flight per thread.
template <class LD, class ST>
__device__ __forceinline__ void own_rows2(const SysView &V, LD &&ld, ST &&st) {
    const int64_t bd = blockDim.x;
    for (int64_t i0 = V.lo + threadIdx.x; i0 < V.hi; i0 += 2 * bd) {
        const int64_t i1 = i0 + bd;
        const bool h1 = i1 < V.hi;
        const auto a = ld(i0);
        decltype(ld(i0)) b{};
        if (h1) b = ld(i1);
        st(i0, a);
        if (h1) st(i1, b);
    }
}

// The same, one row per thread per pass (the pipelined kernels' phases read up
// to 13 vectors: two rows of them would not fit in registers).
template <class LD, class ST>
__device__ __forceinline__ void own_rows1(const SysView &V, LD &&ld, ST &&st) {
    for (int64_t i = V.lo + threadIdx.x; i < V.hi; i += blockDim.x) st(i, ld(i));
}

// y = A x over this CTA's rows with the warp-staged SpMV: x through L2 (other
// CTAs of the group wrote it in this kernel), z (nullable) staged by the lanes
// (written earlier in this kernel), col and val by bulk copies.
// fn(row, y_row, z_row) runs in the lane that owns the row.
template <class F>
__device__ __forceinline__ void group_spmv(const SysView &V, const double *x, const double *z, bool &bad,
                                           F &&fn) {
    unsigned eb = 0u;
    spmv_rows<true, SPMV_CAP_SHORT, true>(V.A, V.lo, V.hi, threadIdx.x >> 5, blockDim.x >> 5, x, z, false, false, eb,
                                          fn);
    if (eb) bad = true;
}

__device__ void solve_classic(const Grp &cl, const SysView &V, SolverState *st, const ClusterRed &R,
                              bool &bad) {
    double *r = V.v[S_R], *r0 = V.v[S_R0], *p = V.v[S_P], *ph = V.v[S_PH], *s = V.v[S_S], *q = V.v[S_Q],
           *qh = V.v[S_QH], *y = V.v[S_Y], *invd = V.v[S_INVD], *x = V.x;
    Win<BQ> w1[1], w2[2];
    uint32_t f1[1] = {0u}, f2[2] = {0u, 0u};
    w1[0].init();
    w2[0].init();
    w2[1].init();
    OWN_ROWS(i) {
        double ri;
        if (V.x0) {
            ri = __dsub_rn(V.b[i], spmv_row_l2(V.A, i, V.x0, bad));
            x[i] = V.x0[i];
        } else {
            ri = V.b[i];
            x[i] = 0.0;
        }
        r[i] = ri;
        r0[i] = ri;
        p[i] = ri;
        ph[i] = __dmul_rn(ri, invd[i]);
        exact_add<BQ, true>(w1[0], f1[0], R.acc[0], ri, ri);
    }
    group_reduce<1>(cl, w1, f1, R);
    if (threadIdx.x == 0) tail_cls_setup(st, R.vals);
    __syncthreads();
    for (int guard = 0; !st->done && guard <= st->maxit; guard++) {
        group_spmv(V, ph, r0, bad, [&](int64_t i, double si, double r0i) {  // K1
            s[i] = si;
            exact_add<BQ>(w1[0], f1[0], R.acc[0], r0i, si);
        });
        group_reduce<1>(cl, w1, f1, R);
        if (threadIdx.x == 0) tail_cls_alpha(st, R.vals);
        __syncthreads();
        if (st->done) break;
        const double na = -st->alpha;
        own_rows2(
            V, [&](int64_t i) { return Vals<3>{{s[i], r[i], invd[i]}}; },
            [&](int64_t i, const Vals<3> &a) {  // K2
                const double qi = fma(na, a.v[0], a.v[1]);
                q[i] = qi;
                qh[i] = __dmul_rn(qi, a.v[2]);
            });
        cl.sync();
        group_spmv(V, qh, q, bad, [&](int64_t i, double yi, double qi) {  // K3
            y[i] = yi;
            exact_add<BQ>(w2[0], f2[0], R.acc[0], qi, yi);
            exact_add<BQ, true>(w2[1], f2[1], R.acc[1], yi, yi);
        });
        group_reduce<2>(cl, w2, f2, R);
        if (threadIdx.x == 0) tail_cls_omega(st, R.vals);
        __syncthreads();
        const double al = st->alpha, om = st->omega, nom = -om;
        own_rows2(
            V, [&](int64_t i) { return Vals<6>{{qh[i], ph[i], x[i], y[i], q[i], r0[i]}}; },
            [&](int64_t i, const Vals<6> &a) {  // K4
                x[i] = fma(om, a.v[0], fma(al, a.v[1], a.v[2]));
                const double ri = fma(nom, a.v[3], a.v[4]);
                r[i] = ri;
                exact_add<BQ>(w2[0], f2[0], R.acc[0], a.v[5], ri);
                exact_add<BQ, true>(w2[1], f2[1], R.acc[1], ri, ri);
            });
        group_reduce<2>(cl, w2, f2, R);
        if (threadIdx.x == 0) tail_cls_beta(st, R.vals, V.hist);
        __syncthreads();
        if (st->done) break;
        const double be = st->beta;
        own_rows2(
            V, [&](int64_t i) { return Vals<4>{{s[i], p[i], r[i], invd[i]}}; },
            [&](int64_t i, const Vals<4> &a) {  // K5
                const double pi = fma(be, fma(nom, a.v[0], a.v[1]), a.v[2]);
                p[i] = pi;
                ph[i] = __dmul_rn(pi, a.v[3]);
            });
        cl.sync();
    }
}

__device__ void solve_pipelined(const Grp &cl, const SysView &V, SolverState *st, const ClusterRed &R,
                                bool &bad) {
    double *r = V.v[S_R], *r0 = V.v[S_R0], *rh = V.v[S_RH], *w = V.v[S_W], *wh = V.v[S_WH], *t = V.v[S_T],
           *ph = V.v[S_PH], *s = V.v[S_S], *sh = V.v[S_SH], *z = V.v[S_Z], *zh = V.v[S_ZH], *v = V.v[S_V],
           *q = V.v[S_Q], *qh = V.v[S_QH], *y = V.v[S_Y], *invd = V.v[S_INVD], *x = V.x;
    Win<BQ> w2[2], w5[5];
    uint32_t f2[2] = {0u, 0u}, f5[5] = {0u, 0u, 0u, 0u, 0u};
    for (int k = 0; k < 2; k++) w2[k].init();
    for (int k = 0; k < 5; k++) w5[k].init();
    OWN_ROWS(i) {
        double ri;
        if (V.x0) {
            ri = __dsub_rn(V.b[i], spmv_row_l2(V.A, i, V.x0, bad));
            x[i] = V.x0[i];
        } else {
            ri = V.b[i];
            x[i] = 0.0;
        }
        r[i] = ri;
        r0[i] = ri;
        rh[i] = __dmul_rn(ri, invd[i]);
    }
    cl.sync();
    group_spmv(V, rh, r0, bad, [&](int64_t i, double wi, double r0i) {
        w[i] = wi;
        wh[i] = __dmul_rn(wi, invd[i]);
        exact_add<BQ, true>(w2[0], f2[0], R.acc[0], r0i, r0i);
        exact_add<BQ>(w2[1], f2[1], R.acc[1], r0i, wi);
    });
    group_reduce<2>(cl, w2, f2, R);
    if (threadIdx.x == 0) tail_pipe_setup(st, R.vals);
    __syncthreads();
    if (!st->done) {
        group_spmv(V, wh, nullptr, bad, [&](int64_t i, double ti, double) { t[i] = ti; });
        cl.sync();
    }
    for (int guard = 0; !st->done && guard <= st->maxit; guard++) {
        const double al = st->alpha, nal = -al, be = st->beta, nom = -st->omega;
        const bool first = st->iter == 0;
        own_rows1(
            V,
            [&](int64_t i) {
                Vals<12> a;
                a.v[0] = rh[i];
                a.v[1] = w[i];
                a.v[2] = wh[i];
                a.v[3] = t[i];
                a.v[4] = r[i];
                a.v[5] = invd[i];
                if (!first) {
                    a.v[6] = ph[i];
                    a.v[7] = s[i];
                    a.v[8] = sh[i];
                    a.v[9] = z[i];
                    a.v[10] = zh[i];
                    a.v[11] = v[i];
                }
                return a;
            },
            [&](int64_t i, const Vals<12> &a) {  // P1: S1-S7, S9
                const double rhi = a.v[0], wi = a.v[1], whi = a.v[2], ti = a.v[3];
                double phi, si, shi, zi;
                if (first) {
                    phi = rhi;
                    si = wi;
                    shi = whi;
                    zi = ti;
                } else {
                    const double ph0 = a.v[6], s0 = a.v[7], sh0 = a.v[8], z0 = a.v[9], zh0 = a.v[10],
                                 v0 = a.v[11];
                    phi = fma(be, fma(nom, sh0, ph0), rhi);
                    si = fma(be, fma(nom, z0, s0), wi);
                    shi = fma(be, fma(nom, zh0, sh0), whi);
                    zi = fma(be, fma(nom, v0, z0), ti);
                }
                const double qi = fma(nal, si, a.v[4]);
                const double qhi = fma(nal, shi, rhi);
                const double yi = fma(nal, zi, wi);
                ph[i] = phi;
                s[i] = si;
                sh[i] = shi;
                z[i] = zi;
                q[i] = qi;
                qh[i] = qhi;
                y[i] = yi;
                zh[i] = __dmul_rn(zi, a.v[5]);
                exact_add<BQ>(w2[0], f2[0], R.acc[0], qi, yi);
                exact_add<BQ, true>(w2[1], f2[1], R.acc[1], yi, yi);
            });
        group_reduce<2>(cl, w2, f2, R);  // also orders zhat for P2's gathers
        if (threadIdx.x == 0) tail_pipe_omega(st, R.vals);
        __syncthreads();
        group_spmv(V, zh, nullptr, bad, [&](int64_t i, double vi, double) { v[i] = vi; });  // P2
        cl.sync();
        const double om = st->omega, nom2 = -om;
        own_rows1(
            V,
            [&](int64_t i) {
                return Vals<13>{{qh[i], y[i], q[i], x[i], ph[i], zh[i], wh[i], v[i], t[i], invd[i], r0[i], s[i],
                                 z[i]}};
            },
            [&](int64_t i, const Vals<13> &a) {  // P3: S12-S15, S17
                const double qhi = a.v[0], yi = a.v[1], qi = a.v[2];
                x[i] = fma(om, qhi, fma(al, a.v[4], a.v[3]));
                const double ri = fma(nom2, yi, qi);
                const double rhi = fma(nom2, fma(nal, a.v[5], a.v[6]), qhi);
                const double wi = fma(nom2, fma(nal, a.v[7], a.v[8]), yi);
                r[i] = ri;
                rh[i] = rhi;
                w[i] = wi;
                wh[i] = __dmul_rn(wi, a.v[9]);
                const double r0i = a.v[10];
                exact_add<BQ>(w5[0], f5[0], R.acc[0], r0i, ri);
                exact_add<BQ>(w5[1], f5[1], R.acc[1], r0i, wi);
                exact_add<BQ>(w5[2], f5[2], R.acc[2], r0i, a.v[11]);
                exact_add<BQ>(w5[3], f5[3], R.acc[3], r0i, a.v[12]);
                exact_add<BQ, true>(w5[4], f5[4], R.acc[4], ri, ri);
            });
        group_reduce<5>(cl, w5, f5, R);  // also orders what for P4's gathers
        if (threadIdx.x == 0) tail_pipe_beta(st, R.vals, V.hist);
        __syncthreads();
        if (st->done) break;
        group_spmv(V, wh, nullptr, bad, [&](int64_t i, double ti, double) { t[i] = ti; });  // P4
        cl.sync();
    }
}

// Solve one queued system (index qi of the order) as group g; rank 0 of the
// group writes the outcome.
__device__ __noinline__ void batch_solve_one(const Grp &g, const BatchSys *__restrict__ sys, const int32_t *__restrict__ order,
                                int qi, BatchOut *out, SolverState &st, const ClusterRed &R, int &s_bad) {
    const int si = order[qi];
    const BatchSys &S = sys[si];
    if (out[si].err) return;  // failed the structure check: same for every CTA of the group
    if (threadIdx.x == 0) {
        memset(&st, 0, sizeof st);
        st.tol = S.tol;
        st.maxit = S.maxit;
        st.variant = S.variant;
        st.hist_cap = g.rank == 0 ? S.hist_cap : 0;
        s_bad = 0;
    }
    __syncthreads();
    SysView V;
    sys_view(S, g, V);
    bool bad = false;
    if (S.variant == RBS_PIPELINED) solve_pipelined(g, V, &st, R, bad);
    else solve_classic(g, V, &st, R, bad);
    if (bad) atomicOr(reinterpret_cast<unsigned *>(&s_bad), 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_bad) atomicOr(&out[si].err, 1u);
        if (g.rank == 0) {
            out[si].iters = st.iter;
            out[si].status = st.status;
            out[si].converged = (st.status == RBS_OK && !(st.tau > st.tau_max)) ? 1 : 0;
            out[si].tau0 = st.tau0;
            out[si].tau_final = st.tau;
            out[si].rho0 = st.rho0;
            out[si].tau_max = st.tau_max;
            out[si].alpha0 = st.alpha0;
            out[si].mu0 = st.mu0;
        }
    }
}

// sizes[q]: unknowns of the q-th queued system (non-increasing).
__global__ void __launch_bounds__(256, 2)
    k_batch(const BatchSys *__restrict__ sys, const int32_t *__restrict__ order, const int64_t *__restrict__ sizes,
            int nsys, int64_t split, unsigned *queue, BatchOut *out) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
    __shared__ int s_next;
    __shared__ SolverState st;
    __shared__ unsigned long long s_acc[5][NL];
    __shared__ long long s_red[5][NL];
    __shared__ uint32_t s_flags[5], s_rflags[5];
    __shared__ double s_vals[5];
    __shared__ int s_bad;
    for (int idx = threadIdx.x; idx < 5 * NL; idx += blockDim.x) (&s_acc[0][0])[idx] = 0ull;
    if (threadIdx.x < 5) s_flags[threadIdx.x] = 0u;
    ClusterRed R{s_acc, s_red, s_flags, s_rflags, s_vals};
    cl.sync();  // every CTA of the cluster runs before any shared memory is touched remotely
    int first_small = -1;  // a small system the cluster pulled, solved by rank 0 alone
    if (csize > 1) {
        const Grp g{&cl, rank, csize};
        for (int guard = 0; guard <= nsys; guard++) {
            if (rank == 0 && threadIdx.x == 0) {
                const int q = (int)atomicAdd(queue, 1u);
                for (unsigned r = 0; r < csize; r++) *cl.map_shared_rank(&s_next, r) = q;
            }
            cl.sync();
            const int qi = s_next;
            cl.sync();  // no remote access of the cluster's shared memory after this in the phase
            if (qi >= nsys) break;
            if (sizes[qi] < split) {
                first_small = rank == 0 ? qi : -1;
                break;
            }
            batch_solve_one(g, sys, order, qi, out, st, R, s_bad);
        }
    }
    // the CTAs now work alone: each takes its own systems from the queue
    const Grp g1{nullptr, 0u, 1u};
    if (first_small >= 0) batch_solve_one(g1, sys, order, first_small, out, st, R, s_bad);
    for (int guard = 0; guard <= nsys; guard++) {
        if (threadIdx.x == 0) s_next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int qi = s_next;
        __syncthreads();
        if (qi >= nsys) break;
        batch_solve_one(g1, sys, order, qi, out, st, R, s_bad);
    }
}

// Per-system structure check and Jacobi set-up: one block per system.
__global__ void __launch_bounds__(256) k_batch_prepare(const BatchSys *__restrict__ sys, int nsys, BatchOut *out) {
    const int si = blockIdx.x;
    if (si >= nsys) return;
    const BatchSys &S = sys[si];
    const CSRView A{S.A.n, S.A.nnz, S.A.rowptr, S.A.col, S.A.val};
    double *invd = S.work + (int64_t)S_INVD * S.stride;
    bool bad = false, bad_diag = false;
    if (threadIdx.x == 0 && (A.rowptr[0] != 0 || A.rowptr[A.n] != A.nnz)) bad = true;
    for (int64_t i = threadIdx.x; i < A.n; i += blockDim.x) {
        const int64_t b = A.rowptr[i], e = A.rowptr[i + 1];
        double d = 0.0;
        bool found = false;
        if (b < 0 || e < b || e > A.nnz) {
            bad = true;
        } else {
            for (int64_t k = b; k < e; k++) {
                const int32_t c = A.col[k];
                if ((uint64_t)(int64_t)c >= (uint64_t)A.n) bad = true;
                else if (!found && c == i) {
                    d = A.val[k];
                    found = true;
                }
            }
        }
        if (S.diag) {
            d = S.diag[i];
            found = true;
        }
        if (!found || d == 0.0 || d != d) {
            bad_diag = true;
            invd[i] = 0.0;
        } else {
            invd[i] = __ddiv_rn(1.0, d);
        }
    }
    if (bad) atomicOr(&out[si].err, 1u);
    if (bad_diag) atomicOr(&out[si].err, 2u);
}

cudaError_t launch_batch_prepare(const BatchSys *d_sys, int nsys, BatchOut *d_out, cudaStream_t s) {
    k_batch_prepare<<<nsys, 256, 0, s>>>(d_sys, nsys, d_out);
    return cudaGetLastError();
}

static cudaLaunchConfig_t batch_cfg(int clusters, int csize, cudaStream_t s, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * csize), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = (unsigned)csize;
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

static void allow_large_clusters() {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        // the SpMV staging buffers take most of a CTA's shared memory
        cudaFuncSetAttribute(k_batch, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaGetLastError();
    });
}

cudaError_t launch_batch(const BatchSys *d_sys, const int32_t *d_order, const int64_t *d_sizes, int nsys,
                         unsigned *d_queue, BatchOut *d_out, BatchSchedule sched, cudaStream_t s) {
    if (sched.cluster < 1 || sched.cluster > BMAX || (sched.cluster & (sched.cluster - 1)))
        return cudaErrorInvalidValue;
    allow_large_clusters();
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = batch_cfg(sched.clusters, sched.cluster, s, &attr);
    return cudaLaunchKernelEx(&cfg, k_batch, d_sys, d_order, d_sizes, nsys, (int64_t)sched.split, d_queue, d_out);
}

int batch_max_clusters(int csize) {
    allow_large_clusters();
    cudaLaunchAttribute attr;
    cudaLaunchConfig_t cfg = batch_cfg(1, csize, nullptr, &attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)k_batch, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 0;
    }
    return n;
}

}  // namespace rbs
