/*
 * reduce_oracle.c -- CPU oracle for the fused update-and-reduce operations:
 * the VecWXPY update of the paper (Sec. 3, Fig. 1) followed by a dot product
 * or a squared 2-norm of its result, as a residual update is followed by its
 * norm.
 *
 * TEST INFRASTRUCTURE ONLY, like wxpy_oracle.c: only the tests and the
 * benchmark's CPU legs load it; it shares no code with the CUDA sources.
 *
 * The paper defines no reduction, so the operation is defined here, and
 * fixed, so that its result is reproducible bit for bit whatever runs it:
 *
 *   w[i] = RN(RN(alpha*x[i]) + y[i])                   (the update, as wxpy)
 *   t[i] = RN(w[i]*w[i])        (norm2)   or   RN(w[i]*z[i])   (dot)
 *   result = TREE(t[0 .. n-1])
 *
 * TREE: cut the index range into tiles of T = 8192 consecutive indices
 * (tile k holds indices kT .. kT + T - 1; the last tile is padded with +0
 * past n).  The sum of a tile is the halving tree: for s = T/2, T/4, ..., 1,
 * e[i] = RN(e[i] + e[i + s]) for every i < s; the sum is e[0].  The tile sums
 * p[0 .. P-1] are padded with +0 to the next power of two P' and summed by
 * the same halving tree.  n = 0 gives +0.  Every sum is rounded to
 * nearest-even in binary64 (built with -ffp-contract=off: no fused
 * multiply-add anywhere).
 *
 * Each element of w is computed from x[i] and y[i] before it is stored, so w
 * may be exactly x or y.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__FAST_MATH__)
#error "the oracle must be built without -ffast-math"
#endif

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1
#define ORACLE_NO_MEMORY 2

#define TILE 8192

/* The halving tree over e[0 .. len-1], len a power of two; e is overwritten. */
static double halving_sum(double *e, int64_t len)
{
    int64_t s, i;
    for (s = len / 2; s >= 1; s /= 2)
        for (i = 0; i < s; ++i)
            e[i] = e[i] + e[i + s];
    return e[0];
}

/* TREE over t[0 .. n-1]. */
static int tree_sum(int64_t n, const double *t, double *result)
{
    int64_t ntiles, padded, k, i;
    double *tile, *partial;
    if (n == 0) {
        *result = 0.0;
        return ORACLE_OK;
    }
    ntiles = (n + TILE - 1) / TILE;
    padded = 1;
    while (padded < ntiles)
        padded *= 2;
    tile = (double *)malloc(sizeof(double) * TILE);
    partial = (double *)malloc(sizeof(double) * (size_t)padded);
    if (!tile || !partial) {
        free(tile);
        free(partial);
        return ORACLE_NO_MEMORY;
    }
    for (k = 0; k < ntiles; ++k) {
        for (i = 0; i < TILE; ++i) {
            int64_t g = k * TILE + i;
            tile[i] = g < n ? t[g] : 0.0;
        }
        partial[k] = halving_sum(tile, TILE);
    }
    for (k = ntiles; k < padded; ++k)
        partial[k] = 0.0;
    *result = halving_sum(partial, padded);
    free(tile);
    free(partial);
    return ORACLE_OK;
}

int oracle_wxpy_norm2(int64_t n, double alpha, const double *x, const double *y, double *w,
                      double *result)
{
    int64_t i;
    double *t;
    int rc;
    if (n < 0 || !result || (n > 0 && (!x || !y || !w)))
        return ORACLE_BAD_ARG;
    t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!t)
        return ORACLE_NO_MEMORY;
    for (i = 0; i < n; ++i) {
        double prod = alpha * x[i];
        double sum = prod + y[i];
        w[i] = sum;
        t[i] = sum * sum;
    }
    rc = tree_sum(n, t, result);
    free(t);
    return rc;
}

int oracle_wxpy_dot(int64_t n, double alpha, const double *x, const double *y, double *w,
                    const double *z, double *result)
{
    int64_t i;
    double *t;
    int rc;
    if (n < 0 || !result || (n > 0 && (!x || !y || !w || !z)))
        return ORACLE_BAD_ARG;
    t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!t)
        return ORACLE_NO_MEMORY;
    for (i = 0; i < n; ++i) {
        double prod = alpha * x[i];
        double sum = prod + y[i];
        double zi = z[i]; /* read before w[i] is stored: z may be w */
        w[i] = sum;
        t[i] = sum * zi;
    }
    rc = tree_sum(n, t, result);
    free(t);
    return rc;
}
