// Per-element steps of the classic (Fig. 2) and pipelined (Fig. 4) loops and
// the solver's view of one system (Ctx). The per-solve kernels
// (kernels_solver.cu) and the per-step kernels of the serving engine
// (kernels_step.cu) both compute every element through these functions, so
// the two paths take the same fma forms and give the same bits.
#pragma once

#include "kernels.cuh"

namespace rbs {

constexpr int SQ = 4;  // window placements used by the solver kernels

struct Ctx {
    CSRView A;
    int64_t n;
    double *x, *r, *r0, *p, *ph, *s, *q, *qh, *y, *invd;
    double *rh, *w, *wh, *t, *sh, *z, *zh, *v;
    const double *b, *x0;
    const double *diag;  // the caller's Jacobi diagonal (per-step path only; null: diag(A))
    SolverState *st;
    DotScratch *g;
    double *hist;
    unsigned *err;
    int spmv_mode;
};

// Two outputs of one element step.
struct VPair {
    double a, b;
};

// set-up, classic: r = RN(b - A x0) (or b), x = x0 (or +0), r0 = p = r,
// phat = RN(r * invd); returns r_i
__device__ __forceinline__ double cls_setup_elem(const Ctx &c, int64_t i, bool &bad) {
    double ri;
    if (c.x0) {
        const double ax = spmv_row(c.A, i, c.x0, bad);
        ri = __dsub_rn(c.b[i], ax);
        c.x[i] = c.x0[i];
    } else {
        ri = c.b[i];
        c.x[i] = 0.0;
    }
    c.r[i] = ri;
    c.r0[i] = ri;
    c.p[i] = ri;
    c.ph[i] = __dmul_rn(ri, c.invd[i]);
    return ri;
}

// S4, S5: q = fma(-alpha, s, r), qhat = RN(q * invd)  -> (q, qhat)
__device__ __forceinline__ VPair cls_k2(double na, double s, double r, double d) {
    const double q = fma(na, s, r);
    return VPair{q, __dmul_rn(q, d)};
}

// S8, S9: x = fma(omega, qhat, fma(alpha, phat, x)), r = fma(-omega, y, q)  -> (x, r)
__device__ __forceinline__ VPair cls_k4(double al, double om, double nom, double qh, double ph, double x, double y,
                                        double q) {
    return VPair{fma(om, qh, fma(al, ph, x)), fma(nom, y, q)};
}

// S12, S1: p = fma(beta, fma(-omega, s, p), r), phat = RN(p * invd)  -> (p, phat)
__device__ __forceinline__ VPair cls_k5(double be, double nom, double s, double p, double r, double d) {
    const double pn = fma(be, fma(nom, s, p), r);
    return VPair{pn, __dmul_rn(pn, d)};
}

// set-up 1, pipelined: r = RN(b - A x0) (or b), x, r0 = r, rhat = RN(r * invd)
__device__ __forceinline__ void pipe_setup1_elem(const Ctx &c, int64_t i, bool &bad) {
    double ri;
    if (c.x0) {
        const double ax = spmv_row(c.A, i, c.x0, bad);
        ri = __dsub_rn(c.b[i], ax);
        c.x[i] = c.x0[i];
    } else {
        ri = c.b[i];
        c.x[i] = 0.0;
    }
    c.r[i] = ri;
    c.r0[i] = ri;
    c.rh[i] = __dmul_rn(ri, c.invd[i]);
}

// P1 for one element: in[0..5] = rh, w, wh, t, r, invd and, after iteration 0,
// in[6..11] = ph, s, sh, z, zh, v (all loaded by the caller before any store);
// out = ph, s, sh, z, q, qh, y, zh.
struct P1In {
    double rh, w, wh, t, r, d, ph, s, sh, z, zh, v;
};
struct P1Out {
    double ph, s, sh, z, q, qh, y, zh;
};
template <class R>
__device__ __forceinline__ P1Out p1_elem(const P1In &a, bool first, double nal, double be, double nom, R &red) {
    P1Out o;
    if (first) {
        o.ph = a.rh;
        o.s = a.w;
        o.sh = a.wh;
        o.z = a.t;
    } else {
        o.ph = fma(be, fma(nom, a.sh, a.ph), a.rh);
        o.s = fma(be, fma(nom, a.z, a.s), a.w);
        o.sh = fma(be, fma(nom, a.zh, a.sh), a.wh);
        o.z = fma(be, fma(nom, a.v, a.z), a.t);
    }
    o.q = fma(nal, o.s, a.r);
    o.qh = fma(nal, o.sh, a.rh);
    o.y = fma(nal, o.z, a.w);
    o.zh = __dmul_rn(o.z, a.d);
    red.add(0, o.q, o.y);
    red.add_sq(1, o.y);
    return o;
}

__device__ __forceinline__ P1In p1_load(const Ctx &c, int64_t i, bool first) {
    P1In a{c.rh[i], c.w[i], c.wh[i], c.t[i], c.r[i], c.invd[i], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (!first) {
        a.ph = c.ph[i];
        a.s = c.s[i];
        a.sh = c.sh[i];
        a.z = c.z[i];
        a.zh = c.zh[i];
        a.v = c.v[i];
    }
    return a;
}

__device__ __forceinline__ void p1_store(const Ctx &c, int64_t i, const P1Out &o) {
    c.ph[i] = o.ph;
    c.s[i] = o.s;
    c.sh[i] = o.sh;
    c.z[i] = o.z;
    c.q[i] = o.q;
    c.qh[i] = o.qh;
    c.y[i] = o.y;
    c.zh[i] = o.zh;
}

// P3 for one element, from its thirteen operands (loaded by the caller before
// any store): x, r, rhat, w and what, and the five dots' products.
struct P3In {
    double qh, y, q, ph, x, zh, wh, v, t, d, r0, s, z;
};
struct P3Out {
    double x, r, rh, w, wh;
};
template <class R>
__device__ __forceinline__ P3Out p3_elem(const P3In &a, double al, double nal, double om, double nom, R &red) {
    P3Out o;
    o.x = fma(om, a.qh, fma(al, a.ph, a.x));
    o.r = fma(nom, a.y, a.q);
    o.rh = fma(nom, fma(nal, a.zh, a.wh), a.qh);
    o.w = fma(nom, fma(nal, a.v, a.t), a.y);
    o.wh = __dmul_rn(o.w, a.d);
    red.add(0, a.r0, o.r);
    red.add(1, a.r0, o.w);
    red.add(2, a.r0, a.s);
    red.add(3, a.r0, a.z);
    red.add_sq(4, o.r);
    return o;
}

}  // namespace rbs
