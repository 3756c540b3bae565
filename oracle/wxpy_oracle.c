/*
 * wxpy_oracle.c -- CPU oracle for the VecWXPY operation w = alpha*x + y.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  The library's
 * product path never links, loads or calls it, and it shares no code,
 * header or constant with the CUDA sources.
 *
 * What it computes.  The paper autotunes the PETSc-style vector kernel it
 * calls "vecwxpy" (Sec. 3, Fig. 1), and its method (Sec. 2) checks every
 * tuned variant against the outputs of the plain, unannotated reference
 * code.  This file is that plain reference code: for every index i in
 * [0, n) it forms
 *
 *      w[i] = RN( RN(alpha * x[i]) + y[i] )
 *
 * in IEEE-754 binary64 with round-to-nearest-even: a correctly rounded
 * product, then a correctly rounded sum.  The paper never writes the
 * formula (it only names the kernel); w = alpha*x + y is PETSc's VecWXPY.
 * It is also silent on precision and on fused multiply-add; the readings
 * taken here are FP64 and two separate roundings, with no FMA.
 *
 * Build flags that the result depends on: -ffp-contract=off (so that the
 * compiler may not fuse the multiply and the add, which GCC on aarch64
 * would otherwise do) and no -ffast-math (which may flush subnormals).
 *
 * Aliasing: each element is read before it is written and no element is
 * read after another element has been written, so w may be exactly x or
 * exactly y (element-wise in-place update).  Partial overlap is not
 * meaningful for the operation and is not checked here.
 */
#include <stddef.h>
#include <stdint.h>

#if defined(__FAST_MATH__)
#error "the oracle must be built without -ffast-math"
#endif

/* GCC ignores '#pragma STDC FP_CONTRACT'; -ffp-contract=off is what forbids fusion. */

/* Status codes of this file (independent of the library's codes). */
#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1

/*
 * w[i] = RN(RN(alpha*x[i]) + y[i]) for i in [0, n).
 * n < 0, or a null pointer with n > 0, returns ORACLE_BAD_ARG and writes
 * nothing.  n == 0 is a no-op.
 */
int oracle_wxpy(int64_t n, double alpha, const double *x, const double *y,
                double *w)
{
    int64_t i;
    if (n < 0)
        return ORACLE_BAD_ARG;
    if (n > 0 && (x == NULL || y == NULL || w == NULL))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double xi = x[i];
        double yi = y[i];
        double prod = alpha * xi; /* first rounding: RN(alpha * x_i) */
        double sum = prod + yi;   /* second rounding: RN(prod + y_i) */
        w[i] = sum;
    }
    return ORACLE_OK;
}

/*
 * Batched form: segment s computes w_s = alpha_s * x_s + y_s over n[s]
 * elements, in segment order, by calling oracle_wxpy once per segment.
 * Returns the first non-zero status met, or ORACLE_OK.
 */
int oracle_wxpy_batch(int64_t count, const int64_t *n, const double *alpha,
                      const double *const *x, const double *const *y,
                      double *const *w)
{
    int64_t s;
    if (count < 0)
        return ORACLE_BAD_ARG;
    if (count > 0 && (n == NULL || alpha == NULL || x == NULL || y == NULL ||
                      w == NULL))
        return ORACLE_BAD_ARG;
    for (s = 0; s < count; ++s) {
        int rc = oracle_wxpy(n[s], alpha[s], x[s], y[s], w[s]);
        if (rc != ORACLE_OK)
            return rc;
    }
    return ORACLE_OK;
}
