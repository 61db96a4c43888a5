/*
 * CPU oracle, part 1: error-free transformations and the exact dot product.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * exdot is computed by its plain definition: every product x_i*y_i is formed
 * exactly as an integer (53-bit x 53-bit significands) times a power of two,
 * added exactly into a Kulisch long accumulator (Sec. 2; 4288 bits suffice,
 * this one has 4352), and the exact sum is rounded once to nearest even. The
 * ExBLAS method of the paper reaches exactly this value because it is
 * correctly rounded (Sec. 2 on ExBLAS, Sec. 3.2), so the definition is the
 * oracle.
 *
 * Readings where the paper is silent: an exact zero sum is +0.0; a NaN operand,
 * an inf*0 product or products of both infinite signs give NaN; otherwise any
 * infinite product gives that infinity; finite products are summed exactly even
 * when their sum overflows binary64, which then rounds to +-inf.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- Alg. 1 and Alg. 2 --------------------------------------------------- */

void orc_twosum(double a, double b, double *r, double *s) {
    double rr = a + b;
    double z = rr - a;
    *s = (a - (rr - z)) + (b - z);
    *r = rr;
}

void orc_twoprod(double a, double b, double *r, double *s) {
    double rr = a * b;
    *s = fma(a, b, -rr);
    *r = rr;
}

double orc_mul_add_unfused(double a, double b, double c) {
    double t = a * b;
    return t + c;
}

/* ---- binary64 decomposition (IEEE-754 format, Table 1) ---------------------
 * x = (-1)^neg * m * 2^e with m < 2^53 an integer: for a normal number
 * m = 2^52 + fraction and e = biased_exponent - 1075; for a subnormal or zero
 * m = fraction and e = -1074. */
typedef struct {
    int neg;
    int cls; /* 0 finite, 1 infinite, 2 NaN */
    uint64_t m;
    int e;
} orc_parts;

static orc_parts orc_split(double x) {
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    orc_parts p;
    p.neg = (int)(bits >> 63);
    int be = (int)((bits >> 52) & 0x7ff);
    uint64_t frac = bits & 0x000fffffffffffffull;
    if (be == 0x7ff) {
        p.cls = frac ? 2 : 1;
        p.m = 0;
        p.e = 0;
    } else if (be == 0) {
        p.cls = 0;
        p.m = frac;
        p.e = -1074;
    } else {
        p.cls = 0;
        p.m = frac | (1ull << 52);
        p.e = be - 1075;
    }
    return p;
}

/* ---- accumulator ---------------------------------------------------------- */

void orc_acc_zero(orc_acc *a) { memset(a, 0, sizeof *a); }

/* add (or subtract) the nonnegative integer w[0..nw-1] (32-bit words, least
 * significant first) times 2^shift, shift >= 0, modulo 2^(32*ORC_DIGITS). */
static void acc_addsub_words(orc_acc *a, const uint32_t *w, int nw, int shift,
                             int subtract) {
    int q = shift / 32, r = shift % 32;
    uint32_t sh[8];
    int ns = nw + 1;
    for (int k = 0; k < ns; k++) {
        uint64_t lo = (k < nw) ? w[k] : 0;
        uint64_t below = (k >= 1) ? w[k - 1] : 0;
        /* word k of (w << r) */
        uint64_t v = (lo << r) | (r ? (below >> (32 - r)) : 0);
        sh[k] = (uint32_t)v;
    }
    if (!subtract) {
        uint64_t carry = 0;
        int j = q;
        for (int k = 0; k < ns && j < ORC_DIGITS; k++, j++) {
            uint64_t t = (uint64_t)a->d[j] + sh[k] + carry;
            a->d[j] = (uint32_t)t;
            carry = t >> 32;
        }
        for (; carry && j < ORC_DIGITS; j++) {
            uint64_t t = (uint64_t)a->d[j] + carry;
            a->d[j] = (uint32_t)t;
            carry = t >> 32;
        }
    } else {
        uint64_t borrow = 0;
        int j = q;
        for (int k = 0; k < ns && j < ORC_DIGITS; k++, j++) {
            uint64_t sub = (uint64_t)sh[k] + borrow;
            uint64_t cur = a->d[j];
            borrow = cur < sub;
            a->d[j] = (uint32_t)(cur - sub);
        }
        for (; borrow && j < ORC_DIGITS; j++) {
            uint64_t cur = a->d[j];
            borrow = cur < 1;
            a->d[j] = (uint32_t)(cur - 1);
        }
    }
}

void orc_acc_add_product(orc_acc *a, double x, double y) {
    orc_parts px = orc_split(x), py = orc_split(y);
    int neg = px.neg ^ py.neg;
    if (px.cls == 2 || py.cls == 2) {
        a->flags |= ORC_F_NAN;
        return;
    }
    if (px.cls == 1 || py.cls == 1) {
        /* inf * 0 is NaN; inf * finite-nonzero or inf * inf is signed inf */
        int zero = (px.cls == 0 && px.m == 0) || (py.cls == 0 && py.m == 0);
        if (zero)
            a->flags |= ORC_F_NAN;
        else
            a->flags |= neg ? ORC_F_NINF : ORC_F_PINF;
        return;
    }
    if (px.m == 0 || py.m == 0) return;
    unsigned __int128 prod = (unsigned __int128)px.m * py.m; /* < 2^106 */
    uint32_t w[4];
    for (int k = 0; k < 4; k++) w[k] = (uint32_t)(prod >> (32 * k));
    int shift = px.e + py.e - ORC_LSB_EXP; /* >= 0: e >= -1074 each */
    acc_addsub_words(a, w, 4, shift, neg);
}

void orc_acc_add_double(orc_acc *a, double x) { orc_acc_add_product(a, x, 1.0); }

static int acc_bit(const uint32_t *d, int i) { return (int)((d[i / 32] >> (i % 32)) & 1u); }

static double round_digits(const uint32_t *src, int32_t flags) {
    if (flags & ORC_F_NAN) return NAN;
    if ((flags & ORC_F_PINF) && (flags & ORC_F_NINF)) return NAN;
    if (flags & ORC_F_PINF) return INFINITY;
    if (flags & ORC_F_NINF) return -INFINITY;
    uint32_t m[ORC_DIGITS];
    memcpy(m, src, sizeof m);
    int neg = (int)(m[ORC_DIGITS - 1] >> 31);
    if (neg) { /* two's complement negation */
        uint64_t carry = 1;
        for (int j = 0; j < ORC_DIGITS; j++) {
            uint64_t t = (uint64_t)(uint32_t)~m[j] + carry;
            m[j] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    int h = -1;
    for (int i = 32 * ORC_DIGITS - 1; i >= 0; i--)
        if (acc_bit(m, i)) { h = i; break; }
    if (h < 0) return 0.0; /* exact zero: +0.0 */
    /* bit index 1074 weighs 2^-1074, the binary64 subnormal quantum */
    int lsb = h - 52;
    if (lsb < 1074) lsb = 1074;
    uint64_t mant = 0;
    for (int i = h; i >= lsb; i--) mant = (mant << 1) | (uint64_t)acc_bit(m, i);
    int round_bit = (lsb >= 1) ? acc_bit(m, lsb - 1) : 0;
    int sticky = 0;
    for (int i = lsb - 2; i >= 0 && !sticky; i--) sticky = acc_bit(m, i);
    if (round_bit && (sticky || (mant & 1))) mant += 1;
    /* mant <= 2^53 is exact in binary64; the scaling is exact or overflows */
    double v = ldexp((double)mant, lsb + ORC_LSB_EXP);
    return neg ? -v : v;
}

double orc_acc_round(const orc_acc *a) { return round_digits(a->d, a->flags); }

static int orc_threads = 1;

void orc_set_threads(int n) { orc_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return orc_threads; }

/* One exact dot over threads: thread t accumulates its contiguous chunk into
 * its own digit array (orc_exdot_limbs), the integer arrays are summed and the
 * total rounded once (orc_round_limbs). */
static double exdot_threads(const double *x, const double *y, int64_t n, int T) {
    int64_t(*limbs)[ORC_DIGITS] = calloc((size_t)T, sizeof *limbs);
    int32_t *flags = calloc((size_t)T, sizeof *flags);
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; t++) {
        const int64_t lo = n * t / T, hi = n * (t + 1) / T;
        orc_exdot_limbs(x + lo, y + lo, hi - lo, limbs[t], &flags[t]);
    }
    int64_t sum[ORC_DIGITS] = {0};
    int32_t fl = 0;
    for (int t = 0; t < T; t++) {
        for (int d = 0; d < ORC_DIGITS; d++) sum[d] += limbs[t][d];
        fl |= flags[t];
    }
    free(limbs);
    free(flags);
    return orc_round_limbs(sum, fl);
}

double orc_exdot(const double *x, const double *y, int64_t n) {
    if (orc_threads > 1) return exdot_threads(x, y, n, orc_threads);
    orc_acc a;
    orc_acc_zero(&a);
    for (int64_t i = 0; i < n; i++) orc_acc_add_product(&a, x[i], y[i]);
    return orc_acc_round(&a);
}

double orc_exsum(const double *x, int64_t n) {
    orc_acc a;
    orc_acc_zero(&a);
    for (int64_t i = 0; i < n; i++) orc_acc_add_double(&a, x[i]);
    return orc_acc_round(&a);
}

void orc_exdot_limbs(const double *x, const double *y, int64_t n, int64_t *limbs,
                     int32_t *flags) {
    orc_acc a;
    orc_acc_zero(&a);
    for (int64_t i = 0; i < n; i++) orc_acc_add_product(&a, x[i], y[i]);
    for (int j = 0; j < ORC_DIGITS; j++) limbs[j] = (int64_t)a.d[j];
    *flags = a.flags;
}

double orc_round_limbs(const int64_t *limbs, int32_t flags) {
    /* carry-normalise the integer sums modulo 2^(32*ORC_DIGITS) (Sec. 3.2:
     * a normalisation after the integer reduction of long accumulators) */
    uint32_t d[ORC_DIGITS];
    int64_t carry = 0;
    for (int j = 0; j < ORC_DIGITS; j++) {
        /* limbs hold sums of 32-bit digits: nonnegative and far below 2^62 */
        int64_t t = limbs[j] + carry;
        d[j] = (uint32_t)(t & 0xffffffffll);
        carry = t >> 32;
    }
    return round_digits(d, flags);
}
