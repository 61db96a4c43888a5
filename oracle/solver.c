/*
 * CPU oracle, part 2: fma SpMV, Jacobi and the two PBiCGStab loops.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Every vector step is written element by element with explicit fma() where
 * the paper's axpy-like forms are fused (Sec. 3.3, Sec. 4.1 "axpy-like vector
 * updates"); every dot is the exact, once-rounded orc_exdot. The steps follow
 * Fig. 2 (classic) and Fig. 4 (pipelined) in their order and notation.
 *
 * Readings where the paper is silent or leaves a choice (each one is listed in
 * the project design notes):
 *  - SpMV row chain starts at +0.0: y_i = fma(a_last, x_last, ... fma(a_0, x_0, +0)).
 *  - Jacobi multiplies by the rounded reciprocal: invd_i = RN(1/d_i),
 *    phat_i = RN(p_i * invd_i). d is the given diagonal, else the first stored
 *    entry (i, i) of row i; a missing or zero entry is an input error.
 *  - r0 = RN(b - A x0) element-wise; with no x0, x0 = +0 and r0 = b.
 *  - tau = RN(sqrt(<r,r>)), tau_max = RN(tol * tau0); the loop runs while
 *    tau > tau_max and fewer than maxit iterations have run.
 *  - Fused forms: S8/S12 x = fma(omega, qhat, fma(alpha, phat, x));
 *    S12 (classic) p = fma(beta, fma(-omega, s, p), r);
 *    beta = RN(RN(rho'/rho) * RN(alpha/omega)) in the order printed;
 *    pipelined alpha denominator = fma(-RN(beta*omega), e, fma(beta, c, a)).
 *  - Pipelined: tau comes from a fifth dot <r, r> taken with the four of S16;
 *    iteration 0 replaces S1-S4 (beta = 0, zero old vectors) by copies.
 *  - <y,y> == 0 means y = 0, so omega := 0 (the half step solved the system).
 *  - The stop test is taken as soon as tau is known; beta, p (classic) and
 *    S17-S19 (pipelined) are computed only when the loop continues.
 *  - Breakdown (status ORC_EBREAKDOWN, history kept): <r0,s> == 0 (classic
 *    S3), <r0,w0> == 0 (pipelined set-up), and, when the loop would continue,
 *    omega == 0, rho' == 0 or the pipelined alpha denominator == 0.
 *  - A non-finite scalar stops the loop with ORC_ENAN.
 *
 * History record per executed iteration (ORC_HIST_W doubles; fields not
 * computed in that iteration hold the quiet NaN 0x7ff8000000000000):
 *  classic:   0 sigma=<r0,s> 1 alpha 2 gamma=<q,y> 3 delta=<y,y> 4 omega
 *             5 rho'=<r0,r> 6 theta=<r,r> 7 tau 8 beta
 *  pipelined: 0 gamma=<q,y> 1 delta=<y,y> 2 omega 3 rho'=<r0,r> 4 a=<r0,w>
 *             5 c=<r0,s> 6 e=<r0,z> 7 theta=<r,r> 8 tau 9 beta 10 den
 *             11 alpha (next)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static double orc_qnan(void) {
    uint64_t b = 0x7ff8000000000000ull;
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *col,
              const double *val, const double *x, double *y) {
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double acc = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++)
            acc = fma(val[k], x[col[k]], acc);
        y[i] = acc;
    }
}

void orc_fma_vec(int64_t n, double a, const double *x, const double *y, double *out) {
    for (int64_t i = 0; i < n; i++) out[i] = fma(a, x[i], y[i]);
}

int orc_jacobi_invd(int64_t n, const int64_t *rowptr, const int32_t *col,
                    const double *val, const double *diag, double *invd) {
    for (int64_t i = 0; i < n; i++) {
        double d = 0.0;
        int found = 0;
        if (diag) {
            d = diag[i];
            found = 1;
        } else {
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++)
                if (col[k] == i) {
                    d = val[k];
                    found = 1;
                    break;
                }
        }
        if (!found || d == 0.0 || isnan(d)) return ORC_EINVAL;
        invd[i] = 1.0 / d;
    }
    return ORC_OK;
}

void orc_jacobi_apply(int64_t n, const double *invd, const double *p,
                      double *phat) {
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
    for (int64_t i = 0; i < n; i++) phat[i] = p[i] * invd[i];
}

static int csr_valid(int64_t n, const int64_t *rowptr, const int32_t *col) {
    if (n < 0 || !rowptr) return 0;
    if (rowptr[0] != 0) return 0;
    for (int64_t i = 0; i < n; i++)
        if (rowptr[i + 1] < rowptr[i]) return 0;
    for (int64_t k = 0; k < rowptr[n]; k++)
        if (col[k] < 0 || col[k] >= n) return 0;
    return 1;
}

static int finite3(double a, double b, double c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

#define VEC(name) double *name = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double))

static int solve_classic(int64_t n, const int64_t *rowptr, const int32_t *col,
                         const double *val, const double *b, const double *x0,
                         const double *invd, double tol, int32_t maxit,
                         double *x, orc_info *info, double *hist) {
    VEC(r); VEC(r0); VEC(p); VEC(ph); VEC(s); VEC(q); VEC(qh); VEC(y);
    int status = ORC_OK;
    /* set-up (Fig. 2, first rows) */
    if (x0) {
        orc_spmv(n, rowptr, col, val, x0, y);
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) { x[i] = x0[i]; r[i] = b[i] - y[i]; }
    } else {
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
    }
    memcpy(r0, r, (size_t)n * sizeof(double));
    memcpy(p, r, (size_t)n * sizeof(double));
    double rho = orc_exdot(r0, r, n);
    double tau = sqrt(rho);
    double tau_max = tol * tau;
    info->rho0 = rho;
    info->tau0 = tau;
    info->tau_max = tau_max;
    int32_t j = 0;
    if (!isfinite(tau)) status = ORC_ENAN;
    while (status == ORC_OK && tau > tau_max && j < maxit) {
        double *h = hist ? hist + (size_t)j * ORC_HIST_W : NULL;
        double rec[ORC_HIST_W];
        for (int k = 0; k < ORC_HIST_W; k++) rec[k] = orc_qnan();
        /* S1, S2 */
        orc_jacobi_apply(n, invd, p, ph);
        orc_spmv(n, rowptr, col, val, ph, s);
        /* S3 */
        double sigma = orc_exdot(r0, s, n);
        if (sigma == 0.0) { status = ORC_EBREAKDOWN; break; }
        double alpha = rho / sigma;
        if (!isfinite(alpha)) { status = ORC_ENAN; break; }
        /* S4, S5, S6 */
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) q[i] = fma(-alpha, s[i], r[i]);
        orc_jacobi_apply(n, invd, q, qh);
        orc_spmv(n, rowptr, col, val, qh, y);
        /* S7 */
        double gamma = orc_exdot(q, y, n);
        double delta = orc_exdot(y, y, n);
        double omega = (delta == 0.0) ? 0.0 : gamma / delta;
        /* S8, S9 */
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) {
            x[i] = fma(omega, qh[i], fma(alpha, ph[i], x[i]));
            r[i] = fma(-omega, y[i], q[i]);
        }
        /* S10 dot and S11 */
        double rho1 = orc_exdot(r0, r, n);
        double theta = orc_exdot(r, r, n);
        tau = sqrt(theta);
        j++;
        rec[0] = sigma; rec[1] = alpha; rec[2] = gamma; rec[3] = delta;
        rec[4] = omega; rec[5] = rho1; rec[6] = theta; rec[7] = tau;
        if (!finite3(gamma, delta, omega) || !finite3(rho1, theta, tau)) {
            if (h) memcpy(h, rec, sizeof rec);
            status = ORC_ENAN;
            break;
        }
        if (!(tau > tau_max)) { if (h) memcpy(h, rec, sizeof rec); break; }
        if (omega == 0.0 || rho1 == 0.0) {
            if (h) memcpy(h, rec, sizeof rec);
            status = ORC_EBREAKDOWN;
            break;
        }
        /* S10 scalar, S12 */
        double beta = (rho1 / rho) * (alpha / omega);
        rec[8] = beta;
        if (h) memcpy(h, rec, sizeof rec);
        if (!isfinite(beta)) { status = ORC_ENAN; break; }
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double t = fma(-omega, s[i], p[i]);
            p[i] = fma(beta, t, r[i]);
        }
        rho = rho1;
    }
    info->iters = j;
    info->tau_final = tau;
    info->converged = (status == ORC_OK && !(tau > tau_max)) ? 1 : 0;
    info->status = status;
    free(r); free(r0); free(p); free(ph); free(s); free(q); free(qh); free(y);
    return status;
}

static int solve_pipelined(int64_t n, const int64_t *rowptr, const int32_t *col,
                           const double *val, const double *b, const double *x0,
                           const double *invd, double tol, int32_t maxit,
                           double *x, orc_info *info, double *hist) {
    VEC(r); VEC(r0); VEC(rh); VEC(w); VEC(wh); VEC(t); VEC(ph); VEC(s);
    VEC(sh); VEC(z); VEC(zh); VEC(v); VEC(q); VEC(qh); VEC(y);
    int status = ORC_OK;
    /* set-up (Fig. 4, first rows) */
    if (x0) {
        orc_spmv(n, rowptr, col, val, x0, y);
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) { x[i] = x0[i]; r[i] = b[i] - y[i]; }
    } else {
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
    }
    memcpy(r0, r, (size_t)n * sizeof(double));
    orc_jacobi_apply(n, invd, r, rh);
    orc_spmv(n, rowptr, col, val, rh, w);
    orc_jacobi_apply(n, invd, w, wh);
    orc_spmv(n, rowptr, col, val, wh, t);
    double rho = orc_exdot(r0, r, n);
    double mu = orc_exdot(r0, w, n);
    double tau = sqrt(rho);
    double tau_max = tol * tau;
    double alpha = 0.0, beta = 0.0, omega = 0.0;
    info->rho0 = rho;
    info->mu0 = mu;
    info->tau0 = tau;
    info->tau_max = tau_max;
    info->alpha0 = orc_qnan();
    int32_t j = 0;
    if (!isfinite(tau) || !isfinite(mu)) status = ORC_ENAN;
    if (status == ORC_OK && tau > tau_max && maxit > 0) {
        if (mu == 0.0) status = ORC_EBREAKDOWN;
        else {
            alpha = rho / mu;
            info->alpha0 = alpha;
            if (!isfinite(alpha)) status = ORC_ENAN;
        }
    }
    while (status == ORC_OK && tau > tau_max && j < maxit) {
        double *h = hist ? hist + (size_t)j * ORC_HIST_W : NULL;
        double rec[ORC_HIST_W];
        for (int k = 0; k < ORC_HIST_W; k++) rec[k] = orc_qnan();
        /* S1-S4 (copies at j = 0), S5-S7 */
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) {
            if (j == 0) {
                ph[i] = rh[i]; s[i] = w[i]; sh[i] = wh[i]; z[i] = t[i];
            } else {
                double ph_new = fma(beta, fma(-omega, sh[i], ph[i]), rh[i]);
                double s_new = fma(beta, fma(-omega, z[i], s[i]), w[i]);
                double sh_new = fma(beta, fma(-omega, zh[i], sh[i]), wh[i]);
                double z_new = fma(beta, fma(-omega, v[i], z[i]), t[i]);
                ph[i] = ph_new; s[i] = s_new; sh[i] = sh_new; z[i] = z_new;
            }
            q[i] = fma(-alpha, s[i], r[i]);
            qh[i] = fma(-alpha, sh[i], rh[i]);
            y[i] = fma(-alpha, z[i], w[i]);
        }
        /* S8 */
        double gamma = orc_exdot(q, y, n);
        double delta = orc_exdot(y, y, n);
        /* S9, S10 */
        orc_jacobi_apply(n, invd, z, zh);
        orc_spmv(n, rowptr, col, val, zh, v);
        /* S11 */
        omega = (delta == 0.0) ? 0.0 : gamma / delta;
        /* S12-S15 */
#pragma omp parallel for if (orc_get_threads() > 1) num_threads(orc_get_threads()) schedule(static)
        for (int64_t i = 0; i < n; i++) {
            x[i] = fma(omega, qh[i], fma(alpha, ph[i], x[i]));
            r[i] = fma(-omega, y[i], q[i]);
            rh[i] = fma(-omega, fma(-alpha, zh[i], wh[i]), qh[i]);
            w[i] = fma(-omega, fma(-alpha, v[i], t[i]), y[i]);
        }
        /* S16, with <r,r> as the fifth dot */
        double rho1 = orc_exdot(r0, r, n);
        double a = orc_exdot(r0, w, n);
        double c = orc_exdot(r0, s, n);
        double e = orc_exdot(r0, z, n);
        double theta = orc_exdot(r, r, n);
        tau = sqrt(theta);
        j++;
        rec[0] = gamma; rec[1] = delta; rec[2] = omega; rec[3] = rho1;
        rec[4] = a; rec[5] = c; rec[6] = e; rec[7] = theta; rec[8] = tau;
        if (!finite3(gamma, delta, omega) || !finite3(rho1, a, c) ||
            !finite3(e, theta, tau)) {
            if (h) memcpy(h, rec, sizeof rec);
            status = ORC_ENAN;
            break;
        }
        if (!(tau > tau_max)) { if (h) memcpy(h, rec, sizeof rec); break; }
        if (omega == 0.0 || rho1 == 0.0) {
            if (h) memcpy(h, rec, sizeof rec);
            status = ORC_EBREAKDOWN;
            break;
        }
        /* S17, S18 */
        orc_jacobi_apply(n, invd, w, wh);
        orc_spmv(n, rowptr, col, val, wh, t);
        /* S19 */
        beta = (rho1 / rho) * (alpha / omega);
        double bw = beta * omega;
        double den = fma(-bw, e, fma(beta, c, a));
        rec[9] = beta;
        rec[10] = den;
        if (den == 0.0) {
            if (h) memcpy(h, rec, sizeof rec);
            status = ORC_EBREAKDOWN;
            break;
        }
        alpha = rho1 / den;
        rec[11] = alpha;
        if (h) memcpy(h, rec, sizeof rec);
        if (!isfinite(beta) || !isfinite(den) || !isfinite(alpha)) {
            status = ORC_ENAN;
            break;
        }
        rho = rho1;
    }
    info->iters = j;
    info->tau_final = tau;
    info->converged = (status == ORC_OK && !(tau > tau_max)) ? 1 : 0;
    info->status = status;
    free(r); free(r0); free(rh); free(w); free(wh); free(t); free(ph); free(s);
    free(sh); free(z); free(zh); free(v); free(q); free(qh); free(y);
    return status;
}

int orc_solve(int64_t n, const int64_t *rowptr, const int32_t *col,
              const double *val, const double *b, const double *x0,
              const double *diag, double tol, int32_t maxit, int32_t variant,
              double *x_out, orc_info *info, double *hist) {
    memset(info, 0, sizeof *info);
    info->status = ORC_EINVAL;
    if (n <= 0 || !b || !x_out || maxit < 0 || !(tol >= 0.0)) return ORC_EINVAL;
    if (variant != 0 && variant != 1) return ORC_EINVAL;
    if (!csr_valid(n, rowptr, col)) return ORC_EINVAL;
    double *invd = (double *)malloc((size_t)n * sizeof(double));
    if (orc_jacobi_invd(n, rowptr, col, val, diag, invd) != ORC_OK) {
        free(invd);
        return ORC_EINVAL;
    }
    int st = variant == 0
                 ? solve_classic(n, rowptr, col, val, b, x0, invd, tol, maxit, x_out, info, hist)
                 : solve_pipelined(n, rowptr, col, val, b, x0, invd, tol, maxit, x_out, info, hist);
    free(invd);
    return st;
}
