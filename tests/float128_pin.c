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
