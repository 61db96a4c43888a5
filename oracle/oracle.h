/*
 * CPU oracle for the reproducible (pipelined) PBiCGStab hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This library is the plain, slow, obviously correct
 * statement of what the GPU path must compute, bit for bit. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: Iakymchuk & Aliaga, "General framework for re-assuring numerical
 * reliability in parallel Krylov solvers: A case of BiCGStab methods"
 * (arXiv 2302.04180). Citations below name the paper's sections, algorithms
 * and figures.
 *
 * Arithmetic: IEEE-754 binary64, round to nearest even, built with
 * -ffp-contract=off and without fast-math, so every a*b+c written in this file
 * is two roundings and every fused step is an explicit fma() call (Sec. 3.3).
 */
#ifndef RBS_ORACLE_H
#define RBS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes of the oracle (numbered like the public library's, defined here
 * on their own). */
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EBREAKDOWN 4
#define ORC_ENAN 5

/* Kulisch long accumulator (Sec. 2): two's complement fixed-point integer of
 * ORC_DIGITS 32-bit digits; bit 0 weighs 2^-2148, the weight of the least
 * significant bit of the product of two binary64 subnormals. 136 digits are
 * 4352 bits, more than the 4288 bits Kulisch gives for an exact binary64 dot. */
#define ORC_DIGITS 136
#define ORC_LSB_EXP (-2148)

/* flags of non-finite products, kept beside the digits */
#define ORC_F_NAN 1    /* a NaN operand or an inf*0 product */
#define ORC_F_PINF 2   /* some product is +inf */
#define ORC_F_NINF 4   /* some product is -inf */

typedef struct {
    uint32_t d[ORC_DIGITS];
    int32_t flags;
} orc_acc;

/* Alg. 1 (TwoSum) and Alg. 2 (TwoProd): r + s == a + b (resp. a*b) exactly. */
void orc_twosum(double a, double b, double *r, double *s);
void orc_twoprod(double a, double b, double *r, double *s);
/* a*b+c with two roundings: proves the build did not contract (Sec. 3.3). */
double orc_mul_add_unfused(double a, double b, double c);

void orc_acc_zero(orc_acc *a);
void orc_acc_add_product(orc_acc *a, double x, double y);
void orc_acc_add_double(orc_acc *a, double x);
double orc_acc_round(const orc_acc *a);

/* exdot: RN(sum_i x_i*y_i) with the sum taken exactly (Sec. 2, Sec. 3.2). */
double orc_exdot(const double *x, const double *y, int64_t n);
/* exact sum of the x_i, rounded once */
double orc_exsum(const double *x, int64_t n);

/* Distributed form of Sec. 3.2: a rank exports its accumulator as ORC_DIGITS
 * int64 words (each the 32-bit digit value, 0..2^32-1) plus its flags. Ranks
 * add the words as plain integers in any order (an integer Allreduce), OR the
 * flags, and round once with orc_round_limbs. */
void orc_exdot_limbs(const double *x, const double *y, int64_t n,
                     int64_t *limbs, int32_t *flags);
double orc_round_limbs(const int64_t *limbs, int32_t flags);

/* SpMV in CSR with the row's fma chain in stored order, starting at +0.0
 * (Sec. 4.1, "Sparse matrix-vector product"; Sec. 3.3). */
/* Threads the oracle's loops and exact dots use (1, the default: sequential).
 * With more, SpMV rows and element-wise steps are split across threads (each
 * element is computed exactly as before), and each exact dot sums per-thread
 * orc_exdot_limbs integers before its one rounding (orc_round_limbs): the
 * rank-split reduction, so every result is bitwise that of one thread. Built
 * without OpenMP, the count is ignored. */
void orc_set_threads(int n);
int orc_get_threads(void);

/* out_i = fma(a, x_i, y_i), one rounding each (the axpy-like steps of Fig. 2
 * and Fig. 4, for drivers that run the loop outside this library, such as the
 * row-block ranks of the sharded-solve test). */
void orc_fma_vec(int64_t n, double a, const double *x, const double *y, double *out);

void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *col,
              const double *val, const double *x, double *y);

/* Jacobi (Sec. 4): invd_i = RN(1/d_i); phat_i = RN(p_i * invd_i). */
int orc_jacobi_invd(int64_t n, const int64_t *rowptr, const int32_t *col,
                    const double *val, const double *diag, double *invd);
void orc_jacobi_apply(int64_t n, const double *invd, const double *p,
                      double *phat);

/* Solver. variant 0 = classic PBiCGStab (Fig. 2), 1 = pipelined (Fig. 4). */
#define ORC_HIST_W 12
typedef struct {
    int32_t iters;
    int32_t converged;
    int32_t status;
    double tau0;
    double tau_final;
    double rho0;
    double tau_max;
    double alpha0; /* pipelined only */
    double mu0;    /* pipelined only: <r0, w0> */
} orc_info;

/* hist (nullable) receives ORC_HIST_W doubles per executed iteration; its
 * capacity is maxit records. */
int orc_solve(int64_t n, const int64_t *rowptr, const int32_t *col,
              const double *val, const double *b, const double *x0,
              const double *diag, double tol, int32_t maxit, int32_t variant,
              double *x_out, orc_info *info, double *hist);

#ifdef __cplusplus
}
#endif
#endif
