/* kernels.c -- the host family of w[i] = RN(RN(alpha*x[i]) + y[i]) loops, the
 * paper's own experiment (Sec. 3, Fig. 1) on this machine's CPU cores.
 *
 * The paper tunes vecwxpy on a CPU by generating variants of its loop with SIMD
 * and unrolling pragmas and compiling each with the production compiler; the
 * baseline is the plain loop at -O3, vectorised by the compiler alone.  Here a
 * variant is one of 13 loops compiled under one of a few flag sets
 * ("flavours"; this file is compiled once per flavour, FLAVOUR_TABLE naming
 * the exported table):
 *
 *   0       the plain loop (what the compiler vectorises by itself);
 *   1 .. 12 explicit SIMD: vectors of VW = 1, 2, 4 or 8 doubles (GCC vector
 *           extensions, lowered to whatever the flavour's target has) times
 *           an unroll of U = 1, 2 or 4 vectors per step.
 *
 * Every flavour is compiled with -ffp-contract=off: the product and the sum
 * are rounded separately, never fused, so every variant gives the same bits.
 * A step loads all of its x and y vectors before it stores any w, so exact
 * aliasing (w == x or w == y) is element-wise, as for the GPU kernels.
 */
#include <stdint.h>
#include <string.h>

#include "cpu_internal.h"

#ifndef FLAVOUR_TABLE
#error "FLAVOUR_TABLE must name the exported kernel table"
#endif

typedef double v2d __attribute__((vector_size(16)));
typedef double v4d __attribute__((vector_size(32)));
typedef double v8d __attribute__((vector_size(64)));

static void plain_loop(int64_t n, double a, const double *x, const double *y, double *w) {
    for (int64_t i = 0; i < n; ++i) {
        double p = a * x[i];
        w[i] = p + y[i];
    }
}

static inline void tail(int64_t i, int64_t n, double a, const double *x, const double *y,
                        double *w) {
    for (; i < n; ++i) {
        double p = a * x[i];
        w[i] = p + y[i];
    }
}

/* Scalar (VW = 1) with an unroll of U: loads first, then products, sums, stores. */
#define SCALAR_KERNEL(U)                                                               \
    static void scalar_u##U(int64_t n, double a, const double *x, const double *y,     \
                            double *w) {                                               \
        int64_t i = 0;                                                                 \
        for (; i + (U) <= n; i += (U)) {                                               \
            double xv[U], yv[U];                                                       \
            for (int u = 0; u < (U); ++u) {                                            \
                xv[u] = x[i + u];                                                      \
                yv[u] = y[i + u];                                                      \
            }                                                                          \
            for (int u = 0; u < (U); ++u) {                                            \
                double p = a * xv[u];                                                  \
                w[i + u] = p + yv[u];                                                  \
            }                                                                          \
        }                                                                              \
        tail(i, n, a, x, y, w);                                                        \
    }

/* VW doubles per vector (type VT), U vectors per step; unaligned loads and
 * stores through memcpy, which the compiler turns into vector moves. */
#define VECTOR_KERNEL(VT, VW, U)                                                       \
    static void v##VW##_u##U(int64_t n, double a, const double *x, const double *y,    \
                             double *w) {                                              \
        VT av;                                                                         \
        for (int k = 0; k < (VW); ++k) av[k] = a;                                      \
        const int64_t step = (int64_t)(VW) * (U);                                      \
        int64_t i = 0;                                                                 \
        for (; i + step <= n; i += step) {                                             \
            VT xv[U], yv[U];                                                           \
            for (int u = 0; u < (U); ++u) {                                            \
                memcpy(&xv[u], x + i + u * (VW), sizeof(VT));                          \
                memcpy(&yv[u], y + i + u * (VW), sizeof(VT));                          \
            }                                                                          \
            for (int u = 0; u < (U); ++u) {                                            \
                VT p = av * xv[u];                                                     \
                VT s = p + yv[u];                                                      \
                memcpy(w + i + u * (VW), &s, sizeof(VT));                              \
            }                                                                          \
        }                                                                              \
        tail(i, n, a, x, y, w);                                                        \
    }

SCALAR_KERNEL(1)
SCALAR_KERNEL(2)
SCALAR_KERNEL(4)
VECTOR_KERNEL(v2d, 2, 1)
VECTOR_KERNEL(v2d, 2, 2)
VECTOR_KERNEL(v2d, 2, 4)
VECTOR_KERNEL(v4d, 4, 1)
VECTOR_KERNEL(v4d, 4, 2)
VECTOR_KERNEL(v4d, 4, 4)
VECTOR_KERNEL(v8d, 8, 1)
VECTOR_KERNEL(v8d, 8, 2)
VECTOR_KERNEL(v8d, 8, 4)

const wxc_kernel_fn FLAVOUR_TABLE[WXC_KERNELS] = {
    plain_loop, scalar_u1, scalar_u2, scalar_u4, v2_u1, v2_u2, v2_u4,
    v4_u1,      v4_u2,     v4_u4,     v8_u1,     v8_u2, v8_u4,
};
