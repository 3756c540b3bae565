/* cpu_internal.h -- shared between the host kernel family (kernels.c, compiled
 * once per flavour) and the library around it (wxpy_cpu.c). */
#ifndef WXPY_CPU_INTERNAL_H
#define WXPY_CPU_INTERNAL_H

#include <stdint.h>

typedef void (*wxc_kernel_fn)(int64_t n, double a, const double *x, const double *y, double *w);

/* Kernels per flavour: 0 the plain loop, then VW in {1, 2, 4, 8} x U in {1, 2, 4}. */
#define WXC_KERNELS 13
#define WXC_FLAVOURS 3

extern const wxc_kernel_fn wxc_table_f0[WXC_KERNELS];
extern const wxc_kernel_fn wxc_table_f1[WXC_KERNELS];
extern const wxc_kernel_fn wxc_table_f2[WXC_KERNELS];

#endif
