/*
 * vecops_oracle.c -- CPU oracle for the other PETSc-style vector kernels of
 * the library: VecAXPY, VecAYPX, VecAXPBYPCZ, VecMAXPY and VecPointwiseMult.
 *
 * TEST INFRASTRUCTURE ONLY, like wxpy_oracle.c: only the tests and the
 * benchmark's CPU legs load it; it shares no code with the CUDA sources.
 *
 * The paper tunes one kernel of this family, vecwxpy (Sec. 3, Fig. 1); these
 * are its siblings in the same vector library.  The paper defines none of
 * them, so each follows PETSc's definition, with every product and every sum
 * rounded to nearest-even in binary64 and evaluated left to right (no fused
 * multiply-add; built with -ffp-contract=off):
 *
 *   axpy:      y[i] = RN(RN(alpha*x[i]) + y[i])
 *   aypx:      y[i] = RN(x[i] + RN(alpha*y[i]))
 *   axpby:     y[i] = RN(RN(alpha*x[i]) + RN(beta*y[i]))
 *   axpbypcz:  z[i] = RN(RN(RN(alpha*x[i]) + RN(beta*y[i])) + RN(gamma*z[i]))
 *   maxpy:     y[i] = RN(... RN(RN(y[i] + RN(a[0]*x0[i])) + RN(a[1]*x1[i])) ...
 *                        + RN(a[m-1]*x_{m-1}[i]))       (terms added in order j)
 *   pmult:     w[i] = RN(x[i]*y[i])
 *
 * Each element is read before it is written, so the output may be exactly one
 * of the inputs.
 */
#include <stddef.h>
#include <stdint.h>

#if defined(__FAST_MATH__)
#error "the oracle must be built without -ffast-math"
#endif

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1

int oracle_axpy(int64_t n, double alpha, const double *x, double *y)
{
    int64_t i;
    if (n < 0 || (n > 0 && (!x || !y)))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double prod = alpha * x[i];
        double sum = prod + y[i];
        y[i] = sum;
    }
    return ORACLE_OK;
}

int oracle_aypx(int64_t n, double alpha, const double *x, double *y)
{
    int64_t i;
    if (n < 0 || (n > 0 && (!x || !y)))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double prod = alpha * y[i];
        double sum = x[i] + prod;
        y[i] = sum;
    }
    return ORACLE_OK;
}

int oracle_axpby(int64_t n, double alpha, double beta, const double *x, double *y)
{
    int64_t i;
    if (n < 0 || (n > 0 && (!x || !y)))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double ax = alpha * x[i];
        double by = beta * y[i];
        double sum = ax + by;
        y[i] = sum;
    }
    return ORACLE_OK;
}

int oracle_axpbypcz(int64_t n, double alpha, double beta, double gamma, const double *x,
                    const double *y, double *z)
{
    int64_t i;
    if (n < 0 || (n > 0 && (!x || !y || !z)))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double ax = alpha * x[i];
        double by = beta * y[i];
        double cz = gamma * z[i];
        double s1 = ax + by;
        double s2 = s1 + cz;
        z[i] = s2;
    }
    return ORACLE_OK;
}

int oracle_maxpy(int64_t n, int m, const double *alpha, const double *const *x, double *y)
{
    int64_t i;
    int j;
    if (n < 0 || m < 0 || (n > 0 && (!y || (m > 0 && (!alpha || !x)))))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double acc = y[i];
        for (j = 0; j < m; ++j) {
            double prod = alpha[j] * x[j][i];
            acc = acc + prod;
        }
        y[i] = acc;
    }
    return ORACLE_OK;
}

int oracle_pmult(int64_t n, const double *x, const double *y, double *w)
{
    int64_t i;
    if (n < 0 || (n > 0 && (!x || !y || !w)))
        return ORACLE_BAD_ARG;
    for (i = 0; i < n; ++i) {
        double prod = x[i] * y[i];
        w[i] = prod;
    }
    return ORACLE_OK;
}
