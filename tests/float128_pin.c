/*
 * float128_pin.c -- an independent check of the oracle's results in binary128
 * (_Float128, 113-bit significand), for the tests.
 *
 * For doubles alpha, x, y: the product alpha*x is exact in binary128 (at most
 * 106 significant bits), and converting it to double rounds once, to nearest
 * even: that is p = RN(alpha*x).  The sum p + y is exact in binary128 when
 * the exponents of p and y differ by at most 59 (the aligned sum needs at most
 * 53 + 59 + 1 = 113 bits, the carry included), and converting it rounds once
 * again: w = RN(p + y).  Cases outside those conditions (non-finite operands
 * or results, a larger exponent gap, products or sums whose rounding leaves
 * the normal range) are counted as skipped, not checked; the exact-rational
 * pins cover them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int exponent_of(double v) {
    int e;
    frexp(v, &e);
    return e;
}

static int normal_or_zero(double v) {
    return v == 0.0 || (isfinite(v) && fabs(v) >= 0x1p-1022);
}

/* Number of w[i] that differ (bitwise) from the binary128 result; *checked and
 * *skipped count the cases. */
int64_t pin_check(int64_t n, double alpha, const double *x, const double *y, const double *w,
                  int64_t *checked, int64_t *skipped) {
    int64_t bad = 0, ok = 0, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(alpha) || !isfinite(x[i]) || !isfinite(y[i])) {
            ++skip;
            continue;
        }
        const _Float128 prod = (_Float128)alpha * (_Float128)x[i];
        const double p = (double)prod;
        if (!normal_or_zero(p) || (p == 0.0 && prod != 0)) {  /* subnormal or underflowed */
            ++skip;
            continue;
        }
        if (p != 0.0 && y[i] != 0.0 && abs(exponent_of(p) - exponent_of(y[i])) > 59) {
            ++skip;
            continue;
        }
        const _Float128 sum = (_Float128)p + (_Float128)y[i];
        const double expect = (double)sum;
        if (!normal_or_zero(expect)) {
            ++skip;
            continue;
        }
        uint64_t a, b;
        memcpy(&a, &expect, 8);
        memcpy(&b, &w[i], 8);
        /* an exact zero sum is +0 in round to nearest, as the conversion gives */
        if (a != b) ++bad;
        ++ok;
    }
    *checked = ok;
    *skipped = skip;
    return bad;
}

/* ---- the sibling operations, step by step ------------------------------------ */

/* RN(a*b) through binary128; *skip set when the result is not a normal double
 * or zero (or an operand is not finite). */
static double rn_prod(double a, double b, int *skip) {
    if (!isfinite(a) || !isfinite(b)) {
        *skip = 1;
        return 0.0;
    }
    const _Float128 e = (_Float128)a * (_Float128)b;
    const double r = (double)e;
    if (!normal_or_zero(r) || (r == 0.0 && e != 0)) *skip = 1;
    return r;
}

/* RN(a+b) through binary128; *skip set unless the sum is exact there (an
 * exponent gap of at most 59) and rounds to a normal double or zero. */
static double rn_sum(double a, double b, int *skip) {
    if (!isfinite(a) || !isfinite(b)) {
        *skip = 1;
        return 0.0;
    }
    if (a != 0.0 && b != 0.0 && abs(exponent_of(a) - exponent_of(b)) > 59) *skip = 1;
    const double r = (double)((_Float128)a + (_Float128)b);
    if (!normal_or_zero(r)) *skip = 1;
    return r;
}

static int same_bits(double a, double b) {
    uint64_t u, v;
    memcpy(&u, &a, 8);
    memcpy(&v, &b, 8);
    return u == v;
}

/* z_out[i] == RN(RN(RN(al*x) + RN(be*y)) + RN(ga*z)) */
int64_t pin_axpbypcz(int64_t n, double al, double be, double ga, const double *x,
                     const double *y, const double *z, const double *z_out, int64_t *checked,
                     int64_t *skipped) {
    int64_t bad = 0, ok = 0, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        int s = 0;
        const double ax = rn_prod(al, x[i], &s), by = rn_prod(be, y[i], &s),
                     cz = rn_prod(ga, z[i], &s);
        const double s1 = rn_sum(ax, by, &s);
        const double s2 = rn_sum(s1, cz, &s);
        if (s) {
            ++skip;
            continue;
        }
        bad += !same_bits(s2, z_out[i]);
        ++ok;
    }
    *checked = ok;
    *skipped = skip;
    return bad;
}

/* y_out[i] == RN(RN(al*x) + RN(be*y)) */
int64_t pin_axpby(int64_t n, double al, double be, const double *x, const double *y,
                  const double *y_out, int64_t *checked, int64_t *skipped) {
    int64_t bad = 0, ok = 0, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        int s = 0;
        const double r = rn_sum(rn_prod(al, x[i], &s), rn_prod(be, y[i], &s), &s);
        if (s) {
            ++skip;
            continue;
        }
        bad += !same_bits(r, y_out[i]);
        ++ok;
    }
    *checked = ok;
    *skipped = skip;
    return bad;
}

/* y_out[i] == y[i] + a[0]*x[0][i] + ... in order, every step rounded; the x
 * vectors are packed one after another (m blocks of n). */
int64_t pin_maxpy(int64_t n, int m, const double *a, const double *xs, const double *y,
                  const double *y_out, int64_t *checked, int64_t *skipped) {
    int64_t bad = 0, ok = 0, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        int s = 0;
        double acc = y[i];
        for (int j = 0; j < m; ++j) acc = rn_sum(acc, rn_prod(a[j], xs[(int64_t)j * n + i], &s), &s);
        if (s) {
            ++skip;
            continue;
        }
        bad += !same_bits(acc, y_out[i]);
        ++ok;
    }
    *checked = ok;
    *skipped = skip;
    return bad;
}

/* w[i] == RN(x[i]*y[i]) */
int64_t pin_pmult(int64_t n, const double *x, const double *y, const double *w,
                  int64_t *checked, int64_t *skipped) {
    int64_t bad = 0, ok = 0, skip = 0;
    for (int64_t i = 0; i < n; ++i) {
        int s = 0;
        const double p = rn_prod(x[i], y[i], &s);
        if (s) {
            ++skip;
            continue;
        }
        bad += !same_bits(p, w[i]);
        ++ok;
    }
    *checked = ok;
    *skipped = skip;
    return bad;
}
