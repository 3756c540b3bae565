/* wxpy_cpu.h -- C ABI of the host (CPU) VecWXPY family and its search: the
 * paper's own experiment (Sec. 3, Fig. 1: vecwxpy tuned with SIMD pragmas
 * against the plain loop at -O3) on the cores of this machine.
 *
 *   w[i] = RN( RN(alpha * x[i]) + y[i] ),  i = 0 .. n-1,  IEEE binary64, never fused
 *
 * A separate library (libwxpy_cpu.so) from the GPU one: every pointer here is
 * a HOST pointer, and nothing here touches a GPU.  Status codes are those of
 * wxpy.h (WXPY_OK, WXPY_EINVAL, WXPY_EOVERLAP, WXPY_ENOMEM, WXPY_EMISMATCH).
 * Validation and aliasing are those of wxpy(): n >= 0; x, y, w non-null and
 * 8-byte aligned when n > 0; w either disjoint from or exactly equal to x and
 * y (a partial overlap is WXPY_EOVERLAP); x and y may overlap freely.
 *
 * Variants.  A variant is (flavour, kernel, threads):
 *   - flavour: the compiler flags the kernels were built with (0: -O2
 *     -fno-tree-vectorize; 1: -O3; 2: -O3 plus this machine's CPU target,
 *     e.g. -mcpu=neoverse-v2+nosve on Grace), every one with -ffp-contract=off;
 *   - kernel: 0 the plain loop (vectorised by the compiler alone), 1 .. 12
 *     explicit SIMD, VW = 1, 2, 4, 8 doubles per vector x U = 1, 2, 4 vectors
 *     per step;
 *   - threads: 1, 2, 4, .. up to the online CPU count (and that count), each
 *     taking one contiguous chunk of the vector, cut at 64-byte boundaries,
 *     from a persistent pool.
 * Every variant gives the same bits. */
#ifndef WXPY_CPU_H
#define WXPY_CPU_H

#include <stdint.h>

#include "wxpy.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wxpy_cpu_variant_info {
    int32_t id;
    int32_t flavour;     /* 0, 1, 2 */
    int32_t kernel;      /* 0 plain loop, 1 .. 12 explicit SIMD */
    int32_t vec;         /* doubles per vector (0 for the plain loop) */
    int32_t unroll;      /* vectors per step (0 for the plain loop) */
    int32_t threads;
    const char *flags;   /* the flavour's compiler flags (static string) */
} wxpy_cpu_variant_info;

typedef struct wxpy_cpu_tune_result {
    int32_t best;             /* winning variant id */
    int32_t best_single;      /* the fastest one-thread variant */
    int32_t candidates;       /* variants timed */
    int32_t rejected;         /* variants whose output differed from the reference */
    int32_t bucket;           /* floor(log2 n): the table cell written */
    int32_t reserved;
    double best_us;           /* median wall time of a call, n elements */
    double best_single_us;
    double baseline_us;       /* the plain loop at -O3 on one thread (the paper's baseline) */
    double reference_us;      /* the reference variant (plain loop, -O2, no vectoriser) */
} wxpy_cpu_tune_result;

/* w = RN(RN(alpha*x) + y) with the variant tuned for n's size bucket, else
 * the baseline variant.  Synchronous. */
int wxpy_cpu(int64_t n, double alpha, const double *x, const double *y, double *w);

/* The same with variant `id`. */
int wxpy_cpu_run_variant(int id, int64_t n, double alpha, const double *x, const double *y,
                         double *w);

/* Number of variants (3 flavours x 13 kernels x the thread counts of this
 * machine), and the fields of variant `id` (WXPY_EINVAL out of range).  The
 * `flags` string is static. */
int wxpy_cpu_variant_count(void);
int wxpy_cpu_variant_describe(int id, wxpy_cpu_variant_info *out);
/* The paper's baseline (flavour 1, plain loop, one thread) and the reference
 * whose outputs every candidate must match (flavour 0, plain loop, one thread). */
int wxpy_cpu_baseline_variant(void);
int wxpy_cpu_reference_variant(void);

/* The Sec. 2 search for n: inputs from a seeded generator; the reference
 * variant's output is the reference result; stage 1 times every (flavour,
 * kernel) on one thread, stage 2 the thread counts for the best kernel of
 * stage 1 (skipped when flags & WXPY_CPU_TUNE_SINGLE).  A candidate is run
 * once and compared bit for bit with the reference (any difference rejects
 * it), then timed as the median of five samples.  A sample times enough
 * back-to-back calls for about 2^20 elements and divides; before it, a 256
 * MiB buffer is rewritten (when the working set is under 1 GiB) so that no
 * input comes from cache -- unless flags & WXPY_CPU_TUNE_WARM, which times
 * calls on cache-resident inputs (the in-cache sizes of the paper's figure).
 * The winner goes to n's size bucket.  Allocates 4 n doubles (plus the flush
 * buffer) while it runs. */
#define WXPY_CPU_TUNE_SINGLE 1u
#define WXPY_CPU_TUNE_WARM 2u
int wxpy_cpu_tune(int64_t n, unsigned flags, wxpy_cpu_tune_result *out);

/* The tuning table: one variant id per size bucket (0 .. 63), -1 untuned. */
int wxpy_cpu_tune_get(int bucket, int *variant_id);
int wxpy_cpu_tune_set(int bucket, int variant_id);
int wxpy_cpu_tune_clear(void);

/* The table as JSON ("wxpy-cpu-tune-1"), keyed by the machine it was tuned on
 * (architecture, online CPU count, the target flavour's flags): the search's
 * result persisted for later processes.  load applies nothing unless every
 * entry is valid; with check_machine it refuses a file from another machine.
 * Errors: WXPY_EINVAL (unwritable, malformed, other machine), WXPY_ENOTFOUND. */
int wxpy_cpu_tune_cache_save(const char *path);
int wxpy_cpu_tune_cache_load(const char *path, int check_machine);

/* Text of the last error on this thread. */
const char *wxpy_cpu_last_error(void);

#ifdef __cplusplus
}
#endif

#endif
