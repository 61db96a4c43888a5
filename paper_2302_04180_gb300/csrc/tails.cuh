// Scalar recurrences of Fig. 2 and Fig. 4 (the device-side "tails"): run by
// one thread once the dots of a step are rounded. Shared by the per-step
// kernels and the batched cluster solver, so both take the same decisions on
// the same bits. `st` may live in global or shared memory.
#pragma once

#include "common.cuh"

namespace rbs {

__device__ __forceinline__ void rec_begin(SolverState *st) {
    for (int f = 0; f < RBS_HIST_W; f++) st->rec[f] = qnan();
}
__device__ __forceinline__ void rec_commit(SolverState *st, double *hist) {
    const int j = st->iter - 1;
    if (j >= 0 && j < st->hist_cap)
        for (int f = 0; f < RBS_HIST_W; f++) hist[(int64_t)j * RBS_HIST_W + f] = st->rec[f];
}
__device__ __forceinline__ void stop(SolverState *st, int status) {
    st->status = status;
    st->done = 1;
}

// set-up, classic: rho = <r0,r0>, tau0 = sqrt(rho), tau_max = tol * tau0
__device__ __forceinline__ void tail_cls_setup(SolverState *st, const double *v) {
    const double rho = v[0];
    const double tau = __dsqrt_rn(rho);
    st->rho = rho;
    st->rho0 = rho;
    st->tau = tau;
    st->tau0 = tau;
    st->tau_max = __dmul_rn(st->tol, tau);
    st->iter = 0;
    st->status = RBS_OK;
    st->done = 0;
    if (!finite_d(tau)) stop(st, RBS_ENAN);
    else if (!(tau > st->tau_max) || st->maxit <= 0) st->done = 1;
}

// S3: alpha = rho / <r0, s>
__device__ __forceinline__ void tail_cls_alpha(SolverState *st, const double *v) {
    rec_begin(st);
    const double sigma = v[0];
    st->rec[0] = sigma;
    if (sigma == 0.0) { stop(st, RBS_EBREAKDOWN); return; }
    const double alpha = __ddiv_rn(st->rho, sigma);
    st->rec[1] = alpha;
    if (!finite_d(alpha)) { stop(st, RBS_ENAN); return; }
    st->alpha = alpha;
}

// S7: omega = <q,y> / <y,y> (0 when y == 0)
__device__ __forceinline__ void tail_cls_omega(SolverState *st, const double *v) {
    const double gamma = v[0], delta = v[1];
    const double omega = (delta == 0.0) ? 0.0 : __ddiv_rn(gamma, delta);
    st->rec[2] = gamma;
    st->rec[3] = delta;
    st->rec[4] = omega;
    st->omega = omega;
}

// S10, S11 and the while test
__device__ __forceinline__ void tail_cls_beta(SolverState *st, const double *v, double *hist) {
    const double rho1 = v[0], theta = v[1];
    const double tau = __dsqrt_rn(theta);
    st->rec[5] = rho1;
    st->rec[6] = theta;
    st->rec[7] = tau;
    st->iter += 1;
    st->tau = tau;
    const double gamma = st->rec[2], delta = st->rec[3], omega = st->omega;
    if (!finite_d(gamma) || !finite_d(delta) || !finite_d(omega) || !finite_d(rho1) || !finite_d(theta) ||
        !finite_d(tau)) {
        rec_commit(st, hist);
        stop(st, RBS_ENAN);
        return;
    }
    if (!(tau > st->tau_max)) { rec_commit(st, hist); st->done = 1; return; }
    if (omega == 0.0 || rho1 == 0.0) { rec_commit(st, hist); stop(st, RBS_EBREAKDOWN); return; }
    const double beta = __dmul_rn(__ddiv_rn(rho1, st->rho), __ddiv_rn(st->alpha, omega));
    st->rec[8] = beta;
    rec_commit(st, hist);
    if (!finite_d(beta)) { stop(st, RBS_ENAN); return; }
    st->beta = beta;
    st->rho = rho1;
    if (st->iter >= st->maxit) st->done = 1;
}

// set-up, pipelined: rho = <r0,r0>, mu = <r0,w0>, alpha0 = rho / mu
__device__ __forceinline__ void tail_pipe_setup(SolverState *st, const double *v) {
    const double rho = v[0], mu = v[1];
    const double tau = __dsqrt_rn(rho);
    st->rho = rho;
    st->rho0 = rho;
    st->mu0 = mu;
    st->tau = tau;
    st->tau0 = tau;
    st->tau_max = __dmul_rn(st->tol, tau);
    st->alpha0 = qnan();
    st->beta = 0.0;
    st->omega = 0.0;
    st->iter = 0;
    st->status = RBS_OK;
    st->done = 0;
    if (!finite_d(tau) || !finite_d(mu)) { stop(st, RBS_ENAN); return; }
    if (!(tau > st->tau_max) || st->maxit <= 0) { st->done = 1; return; }
    if (mu == 0.0) { stop(st, RBS_EBREAKDOWN); return; }
    const double alpha = __ddiv_rn(rho, mu);
    st->alpha = alpha;
    st->alpha0 = alpha;
    if (!finite_d(alpha)) stop(st, RBS_ENAN);
}

// S8 + S11: omega = <q,y> / <y,y>
__device__ __forceinline__ void tail_pipe_omega(SolverState *st, const double *v) {
    rec_begin(st);
    const double gamma = v[0], delta = v[1];
    const double omega = (delta == 0.0) ? 0.0 : __ddiv_rn(gamma, delta);
    st->rec[0] = gamma;
    st->rec[1] = delta;
    st->rec[2] = omega;
    st->omega = omega;
}

// S16 + S19 and the while test
__device__ __forceinline__ void tail_pipe_beta(SolverState *st, const double *v, double *hist) {
    const double rho1 = v[0], a = v[1], c = v[2], e = v[3], theta = v[4];
    const double tau = __dsqrt_rn(theta);
    st->rec[3] = rho1;
    st->rec[4] = a;
    st->rec[5] = c;
    st->rec[6] = e;
    st->rec[7] = theta;
    st->rec[8] = tau;
    st->iter += 1;
    st->tau = tau;
    const double gamma = st->rec[0], delta = st->rec[1], omega = st->omega;
    if (!finite_d(gamma) || !finite_d(delta) || !finite_d(omega) || !finite_d(rho1) || !finite_d(a) ||
        !finite_d(c) || !finite_d(e) || !finite_d(theta) || !finite_d(tau)) {
        rec_commit(st, hist);
        stop(st, RBS_ENAN);
        return;
    }
    if (!(tau > st->tau_max)) { rec_commit(st, hist); st->done = 1; return; }
    if (omega == 0.0 || rho1 == 0.0) { rec_commit(st, hist); stop(st, RBS_EBREAKDOWN); return; }
    const double beta = __dmul_rn(__ddiv_rn(rho1, st->rho), __ddiv_rn(st->alpha, omega));
    const double bw = __dmul_rn(beta, omega);
    const double den = fma(-bw, e, fma(beta, c, a));
    st->rec[9] = beta;
    st->rec[10] = den;
    if (den == 0.0) { rec_commit(st, hist); stop(st, RBS_EBREAKDOWN); return; }
    const double alpha = __ddiv_rn(rho1, den);
    st->rec[11] = alpha;
    rec_commit(st, hist);
    if (!finite_d(beta) || !finite_d(den) || !finite_d(alpha)) { stop(st, RBS_ENAN); return; }
    st->beta = beta;
    st->alpha = alpha;
    st->rho = rho1;
    if (st->iter >= st->maxit) st->done = 1;
}

}  // namespace rbs
