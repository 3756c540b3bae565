/*
 * wxpy.h -- C ABI of the GB300 (sm_103a) VecWXPY library.
 *
 * The operation.  For FP64 vectors x, y, w of length n and a scalar alpha,
 *
 *     w[i] = RN( RN(alpha * x[i]) + y[i] ),   i = 0 .. n-1,
 *
 * in IEEE-754 binary64, round-to-nearest-even, the product and the sum rounded
 * separately (no fused multiply-add).  This is the PETSc vector kernel that the
 * paper autotunes and names "vecwxpy" (Sec. 3, Fig. 1); the paper does not write
 * the formula, and PETSc's VecWXPY defines it.  Every entry point of this file
 * computes exactly these bits, whatever variant runs.
 *
 * The method.  Following Sec. 2, the kernel exists as a family of parameterised
 * code variants; an empirical search runs them, checks their outputs against a
 * plain reference variant, and keeps the fastest per size bucket.  The search
 * knobs are those of Sec. 3 (threads per block, blocks per grid, number of
 * asynchronous streams, L1 size, unroll factor) plus the vector width and the
 * cache policy of the loads and stores.
 *
 * Conventions for every call:
 *  - Return value: a wxpy_status (0 = success).  No exception or signal
 *    crosses the ABI.  After WXPY_ECUDA, wxpy_last_cuda_error() and
 *    wxpy_last_error_message() give details for the calling thread.
 *  - Pointers named x, y, w, *_dev are DEVICE addresses on the current CUDA
 *    device; the caller owns that memory.  The library never frees them.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls documented "asynchronous" only enqueue work on it.
 *  - Vector arguments must be 8-byte aligned.  Exact aliasing (w == x,
 *    w == y, x == y) is allowed and defined element-wise: each element is
 *    read before it is written.  Any partial overlap of w with x or y is
 *    rejected with WXPY_EOVERLAP (x and y may overlap each other freely,
 *    since both are only read).
 */
#ifndef WXPY_H
#define WXPY_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef enum wxpy_status {
    WXPY_OK = 0,
    WXPY_EINVAL = 1,    /* bad argument: n < 0, null or unaligned pointer, bad id */
    WXPY_EOVERLAP = 2,  /* w partially overlaps x or y */
    WXPY_ENOMEM = 3,    /* a library-owned allocation failed */
    WXPY_EBUDGET = 4,   /* request larger than the server's memory budget */
    WXPY_ECUDA = 5,     /* a CUDA runtime call failed (see wxpy_last_cuda_error) */
    WXPY_ETIMEOUT = 6,  /* a bounded wait ran out */
    WXPY_ENOTFOUND = 7, /* unknown ticket / no such entry */
    WXPY_EBUSY = 8,     /* resource in use (for example a server at its slot limit) */
    WXPY_EMISMATCH = 9  /* a variant's output differed from the reference variant */
} wxpy_status;

/* Static English text of a status code; never NULL. */
const char *wxpy_strerror(int status);

/* The cudaError_t of the calling thread's last failed CUDA call (0 if none). */
int wxpy_last_cuda_error(void);

/* Detail text of the calling thread's last error ("" if none).  The pointer
 * stays valid until the thread's next call into the library. */
const char *wxpy_last_error_message(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int wxpy_version(void);

/* ---- device --------------------------------------------------------------- */
typedef struct wxpy_device_info {
    char name[128];          /* cudaDeviceProp::name */
    int32_t device;          /* device ordinal */
    int32_t sm_count;        /* streaming multiprocessors (152 on GB300) */
    int32_t cc_major, cc_minor;
    int64_t l2_bytes;        /* L2 cache size */
    int64_t global_bytes;    /* device memory size */
    int32_t runtime_version; /* CUDA runtime the library was built against */
    int32_t reserved;
} wxpy_device_info;

/* Fills *out for the current device.  Synchronous; no allocation. */
int wxpy_device_query(wxpy_device_info *out);

/* ---- classification (host only, no CUDA call) ------------------------------ */
enum {
    WXPY_ALIAS_XY = 1,  /* x == y: y is not loaded (16 bytes per element) */
    WXPY_ALIAS_WX = 2,  /* w == x */
    WXPY_ALIAS_WY = 4   /* w == y */
};

typedef struct wxpy_class_info {
    int32_t alias;     /* OR of WXPY_ALIAS_* */
    int32_t align;     /* widest vector width in bytes (32, 16 or 8) at which
                          x, y and w share their offset */
    int32_t head;      /* elements before w reaches `align` bytes (<= 3, <= n) */
    int32_t bucket;    /* size bucket floor(log2 n); -1 when n == 0 */
    int32_t tune_key;  /* index of the (bucket, align, alias group) cell of the
                          tuning table, -1 when n == 0 */
    int32_t reserved;
} wxpy_class_info;

/* Validates (n, x, y, w) exactly as wxpy() does and classifies the call:
 * the step that picks the tuned variant (Sec. 2 selection is per size bucket
 * here, and also per alignment and aliasing class).  Pure host arithmetic on
 * the pointer values; never dereferences them. */
int wxpy_classify(int64_t n, const double *x, const double *y, const double *w,
                  wxpy_class_info *out);

/* ---- the variant space (Sec. 2 variants, Sec. 3 knobs) --------------------- */
typedef struct wxpy_variant_info {
    int32_t id;            /* flat index in [0, wxpy_variant_count()), or -1 */
    int32_t vec_bytes;     /* 8, 16, 32: width of each load and store */
    int32_t unroll;        /* 1, 2, 4, 8: independent vectors per thread per pass */
    int32_t threads;       /* threads per block: 128, 256, 512, 1024 */
    int32_t blocks_per_sm; /* 0: one-shot grid (each thread makes one pass);
                              k > 0: grid-stride loop over k * sm_count blocks */
    int32_t cache;         /* 0: ld/st.global; 1: read-only path for the inputs
                              (ld.global.nc.L1::no_allocate) and evict-first
                              stores; 2: evict-first (.cs) loads and stores.
                              1 becomes 2 when w aliases x or y. */
    int32_t carveout;      /* -1: driver default; else the preferred shared
                              memory carveout in percent (0, 50, 100): the
                              rest of the unified L1/shared array is L1 */
    int32_t streams;       /* 1, 2, 4, 8: the call is cut into this many
                              256-byte-aligned pieces, each on its own stream,
                              forked from and joined back into `stream` */
    int32_t fp64_offload;  /* 0: both roundings on the FP64 pipeline; 1: the sum
                              of every other element of a pass, 2: every sum,
                              computed as an exactly rounded binary64 addition in
                              the integer pipeline; 3: every product computed as
                              an exactly rounded binary64 multiplication in the
                              integer pipelines, the sums on the FP64 pipeline
                              (same bits; the FP64 pipeline is the scarce unit on
                              GB300) */
} wxpy_variant_info;

/* Number of variants in the space (vec_bytes x unroll x threads x grid mode x
 * cache x carveout x streams x fp64_offload). */
int wxpy_variant_count(void);

/* Decodes variant `id` into *out.  WXPY_EINVAL for an id out of range. */
int wxpy_variant_describe(int id, wxpy_variant_info *out);

/* Encodes *v into its flat id (written to *id).  WXPY_EINVAL if a field is
 * not one of the listed values. */
int wxpy_variant_encode(const wxpy_variant_info *v, int *id);

/* Forces every later wxpy() call of the process to use variant `id`
 * (tests, benchmarks); id = -1 restores the normal lookup (tuned entry, else
 * the built-in default).  The environment variable WXPY_FORCE_VARIANT=<id>
 * forces a variant from the process's start, as if this had been called
 * first (read once; a value that is not a valid id is ignored); a later call
 * of this function still wins. */
int wxpy_set_variant(int id);

/* Reports in *out the variant that wxpy(n, ., x, y, w, .) would launch now,
 * after the adjustments to the call's class (vec_bytes capped at the class's
 * alignment, cache 1 -> 2 under aliasing).  `tuned` (may be NULL) receives 1 if
 * it came from the tuning table, 2 if forced by wxpy_set_variant, 0 if the
 * built-in default. */
int wxpy_lookup(int64_t n, const double *x, const double *y, const double *w,
                wxpy_variant_info *out, int *tuned);

/* ---- the operation ----------------------------------------------------------- */

/* w[i] = RN(RN(alpha*x[i]) + y[i]) for i in [0, n) (Sec. 3, Fig. 1 vecwxpy).
 * Asynchronous on `stream`; allocates nothing; may be captured in a CUDA
 * graph.  Runs the variant that wxpy_lookup() reports.  n == 0 is a no-op
 * (pointers may then be NULL).  Errors: WXPY_EINVAL (n < 0, null or
 * non-8-byte-aligned pointer), WXPY_EOVERLAP, WXPY_ECUDA (launch failed). */
int wxpy(int64_t n, double alpha, const double *x, const double *y, double *w,
         void *stream);

/* w = RN(RN(alpha*x[i]) + y[i]) for vectors in HOST memory (Sec. 3, Fig. 1
 * vecwxpy), the same bits as wxpy().  The library copies x and y to device
 * staging buffers in chunks, runs wxpy() on each chunk and copies w back,
 * with the copies in, the kernel and the copies out of different chunks
 * overlapping on internal streams that fork from and join back into
 * `stream`.  Asynchronous on `stream`: the host buffers must stay valid, and
 * hw unread, until the stream reaches the end of the call.  Host buffers
 * should be pinned (cudaHostAlloc / cudaHostRegister); pageable memory works
 * but the copies then do not overlap.  The staging buffers (3 x slots x
 * chunk elements) are allocated on a device's first call and kept; calls on
 * one device are serialised by a mutex while they enqueue.  Validation and
 * aliasing rules are those of wxpy().  Errors: as wxpy(), plus WXPY_ENOMEM. */
int wxpy_host(int64_t n, double alpha, const double *hx, const double *hy, double *hw,
              void *stream);

/* Chunk length (a multiple of 32 in [4096, 2^30]; default 2^22), number of
 * pipeline slots (1..8; default 3) and strategy of later wxpy_host() calls.
 * direct = 1: when all three buffers are mapped pinned memory (the runtime
 * gives them device addresses), the kernel reads x, y and writes w across the
 * host link itself -- no staging, both link directions at once -- with one
 * fixed member of the family chosen for the link (16-byte accesses, a
 * grid-stride grid of four blocks per SM, integer-pipeline products), since
 * the link bounds it; otherwise (direct = 0, or unmapped memory) the staged
 * pipeline above, whose kernels use the tuned cells. */
int wxpy_host_config(int64_t chunk_elems, int slots, int direct);

/* Programmatic dependent launch of the single-call kernels (wxpy, wxpy_host's
 * kernels, wxpy_run_variant, the searches' candidates).  When on (the
 * default; the environment variable WXPY_PDL=0 starts the process with it
 * off), each kernel is launched with programmatic stream serialisation: it
 * may be scheduled while the previous kernel of its stream is still running,
 * waits on the device until that kernel has completed and its writes are
 * visible before touching memory, and lets the next launch be scheduled once
 * all its blocks have started.  Results and stream ordering are unchanged
 * (every call still sees all effects of earlier work on its stream); the
 * launch latency of back-to-back calls overlaps the previous kernel's tail.
 * enable = 1 on, 0 off, -1 leaves it as it is; *previous (if not NULL) gets
 * the setting before the call (0 or 1).  WXPY_EINVAL for another enable.
 * Process-wide; host only. */
int wxpy_launch_pdl(int enable, int *previous);

/* The same operation with variant `id` (the tuner's and the tests' entry).
 * The variant is adjusted to the call's class as described at wxpy_lookup. */
int wxpy_run_variant(int id, int64_t n, double alpha, const double *x,
                     const double *y, double *w, void *stream);

/* The plain reference variant of Sec. 2: one element per thread, scalar
 * loads and stores, one-shot grid.  The tuner compares every candidate's
 * output with this variant's, bit for bit. */
int wxpy_reference(int64_t n, double alpha, const double *x, const double *y,
                   double *w, void *stream);

/* ---- sibling vector kernels of the same library -------------------------------- */

/* The paper tunes vecwxpy (Sec. 3, Fig. 1); these are its PETSc siblings, on
 * the same conventions (device pointers, asynchronous on `stream`, 8-byte
 * alignment, the output either disjoint from or exactly equal to each input,
 * WXPY_EINVAL / WXPY_EOVERLAP / WXPY_ECUDA as for wxpy()).  Each product and
 * each sum is rounded to nearest-even in binary64, left to right, never fused:
 *
 *   wxpy_axpy:           y[i] = RN(RN(alpha*x[i]) + y[i])         (VecAXPY; = wxpy into y)
 *   wxpy_aypx:           y[i] = RN(x[i] + RN(alpha*y[i]))         (VecAYPX; = wxpy(alpha, y, x) into y)
 *   wxpy_axpby:          y[i] = RN(RN(alpha*x[i]) + RN(beta*y[i]))   (VecAXPBY)
 *   wxpy_axpbypcz:       z[i] = RN(RN(RN(alpha*x[i]) + RN(beta*y[i])) + RN(gamma*z[i]))
 *   wxpy_maxpy:          y[i] = RN(..RN(RN(y[i] + RN(a[0]*x[0][i])) + RN(a[1]*x[1][i])).. + RN(a[m-1]*x[m-1][i]))
 *   wxpy_pointwise_mult: w[i] = RN(x[i]*y[i])                     (VecPointwiseMult)
 *
 * axpy and aypx run the tuned wxpy() variants.  When all pointers share their
 * offset mod 32 bytes, axpby, axpbypcz and maxpy stream their inputs through a
 * shared-memory ring filled by bulk asynchronous copies (one producer warp,
 * eight consumer warps per block, persistent grid; see wxpy_vecops_status)
 * and pointwise_mult loads 32 bytes per thread into registers; otherwise all
 * three take one element per thread.  maxpy takes `alpha` (m values) and `x`
 * (m device pointers) as HOST arrays and makes one launch per group of 8
 * terms, in order. */
int wxpy_axpy(int64_t n, double alpha, const double *x, double *y, void *stream);
int wxpy_aypx(int64_t n, double alpha, const double *x, double *y, void *stream);
int wxpy_axpby(int64_t n, double alpha, double beta, const double *x, double *y, void *stream);
int wxpy_axpbypcz(int64_t n, double alpha, double beta, double gamma, const double *x,
                  const double *y, double *z, void *stream);
int wxpy_maxpy(int64_t n, int m, const double *alpha, const double *const *x, double *y,
               void *stream);
int wxpy_pointwise_mult(int64_t n, const double *x, const double *y, double *w, void *stream);

/* Pipe split of the streaming sibling kernels (axpbypcz, maxpy,
 * pointwise_mult): how much of their binary64 arithmetic runs as the exactly
 * rounded integer-pipeline operations instead of FP64 instructions.
 * add_offload: the sums (0 none, 1 every other one, 2 all); mul_sixteenths:
 * the fraction, in sixteenths, of each warp's loop iterations whose products
 * run there (0..16).  -1 in either leaves that part to the operation's
 * searched split (wxpy_vecops_tune) or, when it has none, its default (sums
 * in FP64; products 12/16 for axpby, 14/16 for axpbypcz and for maxpy groups of 2 terms,
 * 16/16 for groups of 3..8, 4/16 for pointwise_mult; a maxpy group of one
 * term runs as wxpy() and its tuned variant).  The bits of every result are
 * the same under every split; only the speed differs.  Process-wide, read at
 * each call.  Errors: WXPY_EINVAL out of range. */
int wxpy_vecops_pipes(int add_offload, int mul_sixteenths);

/* The empirical search of Sec. 2 applied to the pipe split of the streaming
 * sibling kernels.  Classes: */
#define WXPY_VEC_AXPBYPCZ 0 /* axpbypcz */
/* 1 .. 7: a maxpy launch group of (class + 1) terms, 2 .. 8 */
#define WXPY_VEC_PMULT 8    /* pointwise_mult */
#define WXPY_VEC_AXPBY 9    /* axpby (its one sum: add offload 1 and 2 both move it) */
#define WXPY_VEC_CLASSES 10

typedef struct wxpy_vecops_tune_result {
    int32_t op_class;       /* WXPY_VEC_* */
    int32_t add_offload;    /* the winning split */
    int32_t mul_sixteenths;
    int32_t candidates;     /* splits timed */
    int32_t rejected;       /* splits whose output differed from the all-FP64 split's */
    int32_t reserved;
    double best_us;         /* median device time of the winner, L2 flushed */
    double default_us;      /* the built-in default split, same conditions */
    double gbs;             /* algorithmic bytes / best_us */
} wxpy_vecops_tune_result;

/* For each class, on generator inputs of n elements per vector: the all-FP64
 * split's output is the reference result; every candidate split (products:
 * 0, 2, .., 16 sixteenths with the sums in FP64; then the sums every other or
 * all in the integer pipeline at the best product share) is run once from
 * pristine inputs and compared with it bit for bit -- a single differing bit
 * rejects it -- and timed as the median of five runs of three back-to-back
 * calls, each run after an L2 flush.
 * The fastest verified split becomes the class's split for later calls that
 * leave wxpy_vecops_pipes at -1, and is saved and loaded with the tune cache
 * (wxpy_tune_cache_save / _load).  `results` (WXPY_VEC_CLASSES entries) may
 * be NULL.  Allocates about 11 n doubles of scratch while it runs, on the
 * current device.  Errors: WXPY_EINVAL (n <= 0), WXPY_ENOMEM, WXPY_ECUDA,
 * WXPY_EMISMATCH (every candidate of a class rejected). */
int wxpy_vecops_tune(int64_t n, wxpy_vecops_tune_result *results);

/* The searched split of a class (-1, -1 when not searched); set installs one
 * (add 0..2, mul 0..16) or clears it (-1, -1). */
int wxpy_vecops_tuned_get(int op_class, int *add_offload, int *mul_sixteenths);
int wxpy_vecops_tuned_set(int op_class, int add_offload, int mul_sixteenths);

/* axpbypcz, maxpy and pointwise_mult on 32-byte co-aligned pointers stream
 * their inputs into shared memory with bulk asynchronous copies, completed on
 * mbarriers; every wait on those barriers gives up after one second.  This
 * synchronises the current device, then returns WXPY_ETIMEOUT (and clears
 * the record) if a wait of any such kernel on it ran out since the last
 * call -- that kernel's output is then incomplete -- else WXPY_OK. */
int wxpy_vecops_status(void);

/* ---- the update fused with a reduction of its result ---------------------------- */

/* w = RN(RN(alpha*x) + y) (the update of Sec. 3, Fig. 1) and, in the same pass,
 *   wxpy_norm2: *result = TREE(RN(w[i]*w[i]))        (the squared 2-norm of w)
 *   wxpy_dot:   *result = TREE(RN(w[i]*z[i]))        (the dot product of w with z)
 * as a residual update is followed by its norm.  TREE is fixed, so the result
 * is the same bits on every run and every grid: the indices are cut into
 * tiles of 8192; a tile's sum is the halving tree e[i] = RN(e[i] + e[i+s]) for
 * s = 4096, 2048, .., 1 (+0 past n); the tile sums, padded with +0 to a power
 * of two, are summed by the same tree; n = 0 gives +0.  (The paper defines no
 * reduction; this one is chosen for reproducibility, and its depth of 13 +
 * log2(tiles) bounds the rounding error like pairwise summation.)
 *
 * Device pointers, asynchronous on `stream`.  x, y, w (and z) as for wxpy():
 * 8-byte aligned, w either disjoint from or exactly equal to each input (each
 * element is read before it is written); `result` is one device double,
 * written when the call completes.  `workspace` is device memory of at least
 * wxpy_reduce_workspace_bytes(n) bytes, 16-byte aligned, disjoint from the
 * vectors and result, owned by the caller; the call overwrites it, so calls in
 * flight at the same time need separate workspaces.  Nothing is allocated.
 * When x, y, w (and z) are all 32-byte aligned, the kernel of the current
 * configuration (wxpy_reduce_variant) reads them as 32-byte vectors;
 * otherwise every element is read and written on its own (same bits).
 * Errors: WXPY_EINVAL (bad argument, workspace too small), WXPY_EOVERLAP,
 * WXPY_ECUDA. */
int64_t wxpy_reduce_workspace_bytes(int64_t n);
int wxpy_norm2(int64_t n, double alpha, const double *x, const double *y, double *w,
               double *result, void *workspace, int64_t workspace_bytes, void *stream);
int wxpy_dot(int64_t n, double alpha, const double *x, const double *y, double *w,
             const double *z, double *result, void *workspace, int64_t workspace_bytes,
             void *stream);

/* The share, in sixteenths, of the tiles whose two products per element
 * (alpha*x and the term) run as the exactly rounded integer-pipeline product
 * instead of FP64 instructions (a rotation over blocks and tiles): 0..16, -1
 * the searched value (wxpy_reduce_tune) or else the default.  Same bits
 * either way.  Process-wide; the same -1 rule holds for wxpy_reduce_variant
 * and wxpy_reduce_sum_levels. */
int wxpy_reduce_pipes(int mul_sixteenths);

/* wxpy_norm2: how many of the leading tree levels of each tile run as the
 * exactly rounded integer-pipeline sum of two non-negative values instead of
 * FP64 instructions: 0..6, -1 the default.  The register-loaded kernel sums
 * its first three levels inside a thread and applies at most 3; the
 * warp-tiled kernels sum six there and apply all; the staged kernels none.
 * Same bits either way.  Process-wide. */
int wxpy_reduce_sum_levels(int levels);

/* The kernel of wxpy_norm2 / wxpy_dot for 32-byte co-aligned pointers
 * (other alignments always take the element path): 0 register-loaded (a
 * block of 256 threads per tile, 32-byte loads into registers); 1, 2, 3
 * staged through a shared-memory ring of bulk copies with (ring stages,
 * resident blocks per SM) = (4, 2), (3, 3), (2, 3); 4, 5, 6 warp-tiled (one
 * warp per tile, no block barrier; rows loaded together, resident 128-thread
 * blocks per SM) = (2, 5), (4, 4), (4, 3); -1 the default.  Same bits for
 * every variant.  Process-wide. */
int wxpy_reduce_variant(int variant);

typedef struct wxpy_reduce_tune_result {
    int32_t kind;            /* 0 wxpy_norm2, 1 wxpy_dot */
    int32_t variant;         /* the winning configuration (see wxpy_reduce_variant) */
    int32_t mul_sixteenths;
    int32_t sum_levels;      /* norm2 only; 0 for dot */
    int32_t candidates;      /* configurations timed */
    int32_t rejected;        /* configurations whose w or result differed from the reference */
    double best_us;          /* median device time of the winner, L2 flushed */
    double default_us;       /* the built-in default configuration, same conditions */
    double gbs;              /* algorithmic bytes (24 or 32 per element) / best_us */
} wxpy_reduce_tune_result;

/* The empirical search of Sec. 2 for the fused reductions.  For each of
 * wxpy_norm2 and wxpy_dot, on generator inputs of n elements per vector: the
 * register-loaded kernel with every operation in FP64 gives the reference w
 * and result; every candidate configuration (the register-loaded kernel at
 * product shares 0, 4, .., 16 sixteenths; for norm2, 1..3 integer tree
 * levels at the best share and at half of it; the three staged shapes and
 * the three warp-tiled shapes at the best share; for norm2, 2, 4 and 6
 * integer tree levels in the fastest warp-tiled shape) is run once and compared with it bit for bit -- a single
 * differing bit of w or of the result rejects it -- and timed as the median
 * of five runs of three back-to-back calls, each run after an L2 flush.  The fastest verified configuration
 * becomes the operation's configuration for later calls whose knobs are left
 * at -1, and is saved and loaded with the tune cache.  `results` (2 entries)
 * may be NULL.  Allocates about 5 n doubles of scratch while it runs, on the
 * current device.  Errors: WXPY_EINVAL (n <= 0), WXPY_ENOMEM, WXPY_ECUDA,
 * WXPY_EMISMATCH (every configuration rejected). */
int wxpy_reduce_tune(int64_t n, wxpy_reduce_tune_result *results);

/* The searched configuration of a reduction (kind 0 norm2, 1 dot; all -1
 * when not searched); set installs one or clears it (all -1). */
int wxpy_reduce_tuned_get(int kind, int *variant, int *mul_sixteenths, int *sum_levels);
int wxpy_reduce_tuned_set(int kind, int variant, int mul_sixteenths, int sum_levels);

/* Synchronises the current device, then returns WXPY_ETIMEOUT (and clears
 * the record) if a bounded wait of a staged reduction launched since the last
 * call ran out -- its w and result are then not to be used -- else WXPY_OK.
 * WXPY_ECUDA if the synchronisation fails. */
int wxpy_reduce_status(void);

/* ---- batched launch: many independent problems in one launch ----------------- */

/* One problem of a batch: w = RN(RN(alpha*x) + y) over n elements (Sec. 3,
 * Fig. 1 vecwxpy).  40 bytes, no padding.  Pointers are device addresses. */
typedef struct wxpy_desc {
    int64_t n;
    double alpha;
    const double *x;
    const double *y;
    double *w;
} wxpy_desc;

typedef struct wxpy_batch_plan wxpy_batch_plan; /* opaque */

typedef struct wxpy_batch_info {
    int64_t segments;  /* descriptors in the table */
    int64_t tiles;     /* work items of the persistent launch */
    int64_t elements;  /* sum of n */
    int64_t bytes;     /* algorithmic bytes: 24 per element */
    int32_t grid;      /* blocks of the launch */
    int32_t threads;   /* threads per block */
} wxpy_batch_info;

/* Builds a plan for the problems in `host_table` (a HOST copy of the table;
 * only its lengths and pointer values are read, never the vectors).  Every
 * descriptor is validated as wxpy() validates a call, and the problems must be
 * independent: no two write overlapping ranges and none reads a range another
 * writes (WXPY_EOVERLAP).  Validation happens before any CUDA call.  The plan
 * cuts each problem into tiles whose length depends on its size bucket (tuned
 * by wxpy_batch_tune, else built in) and uploads the tile list to device
 * memory that the plan owns.  Synchronous.  *out is NULL on error. */
int wxpy_batch_plan_create(const wxpy_desc *host_table, int64_t count,
                           wxpy_batch_plan **out);

/* Runs every problem of the plan in ONE persistent kernel launch on `stream`
 * (asynchronous).  `dev_table` is a DEVICE copy of the table, owned by the
 * caller, with the same lengths as the host table of the plan; alpha and the
 * pointers are read from it at run time.  A tile that would pass the n of the
 * descriptor it reads is skipped and flagged (wxpy_batch_status).  May be
 * captured in a CUDA graph.  A plan serves one host thread at a time. */
int wxpy_batch_launch(wxpy_batch_plan *plan, const wxpy_desc *dev_table, void *stream);

/* The same launch replayed from a CUDA graph that the plan builds on first use
 * (and re-points, by updating the kernel node, when dev_table changes). */
int wxpy_batch_graph_launch(wxpy_batch_plan *plan, const wxpy_desc *dev_table,
                            void *stream);

/* The plan's shape (segments, elements, tiles, grid; see wxpy_batch_info),
 * read from the host copy; touches no device.  WXPY_EINVAL for null. */
int wxpy_batch_plan_info(const wxpy_batch_plan *plan, wxpy_batch_info *out);

/* Reads (synchronously) the plan's status word: bit 0 set if a launch skipped
 * a tile because the device table's n was smaller than the plan's.  clear != 0
 * resets it. */
int wxpy_batch_status(wxpy_batch_plan *plan, unsigned *status, int clear);

/* Frees the plan and its device memory (the caller must make sure no launch
 * of it is still running).  NULL is a no-op. */
int wxpy_batch_plan_destroy(wxpy_batch_plan *plan);

/* One-shot form: validate, plan and launch in one call.  The tile list lives
 * in stream-ordered scratch (cudaMallocAsync / cudaFreeAsync on `stream`). */
int wxpy_batch(const wxpy_desc *host_table, const wxpy_desc *dev_table, int64_t count,
               void *stream);

/* The batched launch for callers that cannot allocate device memory: code
 * whose device memory all belongs to another allocator (a framework's caching
 * pool, a server's fixed arena) that must not see a cudaMalloc it did not
 * make, and hot loops that cannot afford an allocation call.  The paper has
 * no counterpart; this is a library convenience.
 *
 * Same results as wxpy_batch() for the problems in `dev_table` (a DEVICE
 * table of `count` descriptors, owned by the caller, as are all vectors).  It
 * calls no cudaMalloc, cudaFree or other allocating routine and takes no host
 * table: the tiles are planned on the device, in `stream`, into a fixed
 * scratch array of about 3 MiB that is a static device variable of the
 * library, held by every GPU that loads the library until the process exits.
 * Limit: count <= 65536 (WXPY_EINVAL above it, before anything is launched).
 * The first call on a device looks up the scratch address
 * (cudaGetSymbolAddress) for that device and keeps it once the lookup has
 * succeeded (a failed lookup returns WXPY_ECUDA and is retried by the next
 * call); make that first call before any stream capture.  Every call shares
 * the one scratch array, which keeps the last call's contents (each call
 * rebuilds what it reads): calls that overlap on the GPU -- on different
 * streams, or from different threads -- race on it and must be serialised by
 * the caller.  Descriptors are checked on the device only for n <= 0 and for
 * null or misaligned pointers (such problems are skipped); none of the host
 * checks of wxpy_batch() (no WXPY_EOVERLAP) runs here, so the caller
 * guarantees what they would check: within each descriptor, w equals x, equals
 * y, or overlaps neither of them (a partial overlap races silently), and no
 * descriptor writes a range that another descriptor reads or writes.
 * Asynchronous on `stream`. */
int wxpy_batch_noalloc(const wxpy_desc *dev_table, int64_t count, void *stream);

/* ---- the empirical search (Sec. 2) and its persisted results ------------------ */

/* Which call class wxpy_tune() reproduces (default: x, y, w 32-byte co-aligned
 * and distinct), and how it searches. */
enum {
    WXPY_TUNE_ALIGN16 = 1 << 0,  /* x, y, w share their offset mod 16 bytes only */
    WXPY_TUNE_ALIGN8 = 1 << 1,   /* ... mod 8 bytes only */
    WXPY_TUNE_XY = 1 << 2,       /* x == y */
    WXPY_TUNE_WALIAS = 1 << 3,   /* w == x (in-place update) */
    WXPY_TUNE_QUICK = 1 << 4,    /* only the width x unroll x cache stage, fewer reps */
    WXPY_TUNE_RESIDENT = 1 << 5  /* time back-to-back (L2-resident) runs instead of
                                    flushing the L2 before every timed run */
};

typedef struct wxpy_tune_result {
    wxpy_variant_info best;  /* the variant stored for the cell */
    double best_us;          /* its median device time for n elements */
    double default_us;       /* median time of the built-in default variant */
    double reference_us;     /* median time of the plain reference variant */
    double best_gbs;         /* algorithmic GB/s of `best` (24 bytes per element,
                                16 when x == y) */
    int32_t candidates;      /* variants run */
    int32_t rejected;        /* variants whose output differed from the reference */
    int32_t bucket;          /* floor(log2 n) */
    int32_t tune_key;        /* the cell written */
    int32_t ties;            /* candidates timed within 3 % of the fastest */
    int32_t launch_bound;    /* 1: even the plain reference variant timed within
                                3 % of the fastest, so no kernel shape changes the
                                call's time (launch and completion dominate); the
                                cell then gets a fixed choice -- the first
                                candidate in search order within 3 % -- instead of
                                a pick among ties; saved in the tune cache */
} wxpy_tune_result;

/* Runs the search of Sec. 2 for the cell of size bucket floor(log2 n) and the
 * class selected by `flags`: it allocates its own scratch (about 4 * 8n bytes,
 * a buffer of twice the L2 size, and for calls expected under 200 us an arena
 * of at most 2 GiB of input copies), fills the inputs from the seeded
 * generator, runs the reference variant once, then runs every candidate
 * (coordinate search: width x unroll x cache, then threads x grid mode, then
 * carveout x streams), rejects any whose output differs from the reference
 * results by a single bit, times the rest with CUDA events (median of several
 * runs, L2 flushed before each; a call expected under 200 us is timed as a
 * batch of back-to-back calls on separate copies of the inputs, below the
 * event clock's 2.048 us step), and stores the fastest -- or the default
 * variant, if it re-times faster -- in the tuning table, where every later
 * wxpy() call of that cell finds it.  Synchronous; serialised by a mutex;
 * frees its scratch before returning.  `out` may be NULL.
 * Errors: WXPY_EINVAL (n <= 0, XY with WALIAS), WXPY_ENOMEM, WXPY_ECUDA,
 * WXPY_EMISMATCH (no candidate matched the reference). */
int wxpy_tune(int64_t n, unsigned flags, wxpy_tune_result *out);
/* For this search and the other two (wxpy_vecops_tune, wxpy_reduce_tune), the
 * environment variable WXPY_TUNE_REPS=<1..101> sets the timed runs per
 * candidate, whose median counts (read at every search; other values are
 * ignored). */

/* The tuning table: one variant id per cell (tune_key of wxpy_class_info),
 * -1 for an untuned cell.  get/set/clear touch no device; clear also drops
 * the searched splits of the sibling kernels (wxpy_vecops_tune). */
int wxpy_tune_get(int tune_key, int *variant_id);
int wxpy_tune_set(int tune_key, int variant_id);
int wxpy_tune_clear(void);

/* Writes the tuned cells to a JSON file keyed by the device (name, compute
 * capability, SM count, CUDA runtime): the selected variants of Sec. 2 kept
 * across processes.  Replaces the file atomically. */
int wxpy_tune_cache_save(const char *path);

/* Reads a file written by wxpy_tune_cache_save and stores its cells.  With
 * check_device != 0 a file tuned on another device is rejected (WXPY_EINVAL)
 * and nothing is stored; a malformed file stores nothing either.  When the
 * environment variable WXPY_TUNE_CACHE names a file, the first wxpy() call of
 * the process loads it this way (errors ignored). */
int wxpy_tune_cache_load(const char *path, int check_device);

/* ---- the search for the batched launch (Sec. 2 applied per size bucket) ------- */

typedef struct wxpy_batch_tune_result {
    int32_t tile_elems[64];  /* per bucket: elements per tile, 0 = whole segment */
    int32_t unroll[64];      /* per bucket: 1, 2, 4 (0 where not searched) */
    double us[64];           /* per bucket: median time of the bucket's batch */
    double gbs[64];          /* per bucket: algorithmic GB/s of that batch */
    double mixed_us;         /* mixed batch of buckets min..max, chosen grid */
    double mixed_gbs;
    int32_t blocks_per_sm;   /* chosen grid: blocks_per_sm * sm_count */
    int32_t threads;
    int32_t candidates;      /* batched launches run */
    int32_t rejected;        /* candidates whose output differed from the reference */
    int32_t fp64_offload;    /* chosen: 0 every operation on the FP64 pipeline, 1 half
                                of the sums, 3 every product in the integer pipelines
                                (see wxpy_variant_info) */
    int32_t reserved;
} wxpy_batch_tune_result;

/* For each size bucket b in [bucket_min, bucket_max] (at most 30): builds a
 * synthetic batch whose segments all fall in b, obtains its reference results
 * by running the plain reference variant on every segment, then runs the
 * batched launch with every (tile length, unroll) candidate, rejects any
 * whose output differs by a bit, and keeps the fastest (median time) for b.
 * Finally picks blocks per SM and fp64_offload (0, 1 or 3) on a mixed batch.
 * The results replace the
 * process's batch shape table, used by later plans.  Synchronous; allocates
 * and frees its own scratch.  flags: WXPY_TUNE_QUICK narrows the search. */
int wxpy_batch_tune(int bucket_min, int bucket_max, unsigned flags,
                    wxpy_batch_tune_result *out);

/* The batch shape table: per bucket tile length (0 or a multiple of 32, at
 * most 2^30) and unroll (1, 2, 4: 32-byte vectors of x and of y in flight per
 * lane per pass).  Host only; no device touched. */
int wxpy_batch_shape_get(int bucket, int *tile_elems, int *unroll);
int wxpy_batch_shape_set(int bucket, int tile_elems, int unroll);
int wxpy_batch_shape_reset(void);

/* Whole-launch knobs of the batched launch (and of the server's batches):
 * grid = blocks_per_sm (1..32) * sm_count, and fp64_offload 0, 1 (half of the
 * sums in the integer pipeline) or 3 (every product in the integer pipelines),
 * as for wxpy_variant_info.  Host only. */
int wxpy_batch_launch_get(int *blocks_per_sm, int *fp64_offload);
int wxpy_batch_launch_set(int blocks_per_sm, int fp64_offload);

/* ---- serving: continuous batching of wxpy requests --------------------------- */

/* The paper has no serving layer; this runs the operation of Sec. 3 / Fig. 1
 * for a stream of independent requests.  A seeded request (n, alpha, seed)
 * gets inputs x, y = U(-1,1) streams (seed, WXPY_TAG_X) and (seed, WXPY_TAG_Y)
 * of the seeded generator (wxpy_fill_uniform), written into its resident
 * buffers on the device; a caller-data request (wxpy_server_submit_data) gets
 * the caller's x and y copied into them.  Either way the result is
 * w = RN(RN(alpha*x) + y) -- the same bits whether the request runs alone or
 * batched with any other requests.
 *
 * Modes:
 *   WXPY_SERVE_BATCHED  per batch, the inputs step (one segmented fill launch
 *                       for the seeded requests, copies for the caller-data
 *                       ones) and then ONE launch of the batched segmented
 *                       kernel (the one wxpy_batch runs) over the batch,
 *                       reading x and y from the resident buffers and writing
 *                       w: 24 bytes per element;
 *   WXPY_SERVE_SERIAL   the baseline over the identical data path: per
 *                       request, the inputs step (fill x, fill y, or the
 *                       copies) and one wxpy() call;
 *   WXPY_SERVE_FUSED    seeded requests only: one kernel per batch generates
 *                       x and y in registers and writes x, y and w, reading
 *                       nothing (no load path of wxpy is exercised). */
enum { WXPY_SERVE_BATCHED = 0, WXPY_SERVE_SERIAL = 1, WXPY_SERVE_FUSED = 2 };

/* Where the caller's data of wxpy_server_submit_data lives. */
enum { WXPY_SERVE_DATA_DEVICE = 0, WXPY_SERVE_DATA_HOST = 1 };
enum {
    WXPY_REQ_QUEUED = 0,    /* waiting for memory or a slot */
    WXPY_REQ_ADMITTED = 1,  /* buffers assigned, not yet launched */
    WXPY_REQ_RUNNING = 2,   /* part of a batch in flight */
    WXPY_REQ_DONE = 3,      /* result resident until released */
    WXPY_REQ_FAILED = 4     /* its batch failed to launch or run */
};

typedef struct wxpy_server_config {
    int64_t budget_bytes; /* device memory for request buffers (x, y, w of every
                             resident request: 3 * 8n bytes rounded to 256 each),
                             allocated once at create */
    int32_t max_slots;    /* requests resident at once (admitted, not released) */
    int32_t n_streams;    /* streams the batches run on, 1..16; batches on
                             different streams overlap on the device */
    int32_t max_batch;    /* requests coalesced into one batched launch */
    int32_t max_queue;    /* queued requests beyond which submit refuses (EBUSY) */
    int32_t mode;         /* WXPY_SERVE_BATCHED, WXPY_SERVE_SERIAL (the
                             baseline) or WXPY_SERVE_FUSED; see above */
    int32_t admission;    /* 0: strict arrival order -- a request that does not
                             fit the arena waits, and nothing passes it;
                             > 0: backfill -- while the queue's head does not
                             fit, later requests (up to 64 places back) that fit
                             are admitted, for at most `admission`
                             microseconds of the head's wait; after that nothing
                             passes it until it is admitted */
} wxpy_server_config;

typedef struct wxpy_server wxpy_server; /* opaque */

typedef struct wxpy_server_stats {
    int64_t submitted, rejected, completed, failed;
    int64_t queued_now, resident_now, max_queue;
    int64_t batches, launches, elements_done, arena_used;
    int64_t max_inflight; /* most batches on the device at the same time */
    double mean_batch;   /* requests per batch */
    double window_s;     /* time since the statistics were last reset */
    double p50_s, p99_s, mean_s, max_s; /* submit -> completion, completed requests */
    double head_wait_frag_s;  /* time the queue's head waited although the arena
                                 had enough free bytes in total (fragmentation) */
    double head_wait_full_s;  /* time it waited because the arena was too full */
    int64_t backfilled;       /* requests admitted ahead of a waiting head */
    int64_t reserved;
    double max_launch_host_s; /* longest host time the scheduler spent queueing one
                                 batch's work (tables, copies, launches) */
    double max_batch_s;       /* longest time from queueing a batch to the scheduler
                                 seeing it complete */
} wxpy_server_stats;

/* Allocates the arena (cudaMalloc of budget_bytes), per-stream staging, and
 * starts the scheduler thread on the current device.  It admits requests in
 * arrival order while memory and slots allow; it coalesces the admitted
 * requests into one batch per free stream; it polls completion events.
 * WXPY_EINVAL for a bad configuration, WXPY_ENOMEM, WXPY_ECUDA. */
int wxpy_server_create(const wxpy_server_config *cfg, wxpy_server **out);

/* Queues a request; *ticket identifies it.  Never blocks.  WXPY_EBUDGET if it
 * can never fit the budget, WXPY_EBUSY if the queue is full (counted as a
 * reject), WXPY_EINVAL for n <= 0. */
int wxpy_server_submit(wxpy_server *sv, int64_t n, double alpha, uint64_t seed,
                       uint64_t *ticket);

/* Queues a request on the caller's own data: x and y, n doubles each, in
 * device memory (kind WXPY_SERVE_DATA_DEVICE) or host memory
 * (WXPY_SERVE_DATA_HOST; pinned memory lets the copies run asynchronously,
 * pageable memory works but stalls the scheduler while it copies).  When the
 * request's batch runs, the server copies x and y into the request's resident
 * buffers on that batch's stream, ahead of the batch's kernel.  The caller
 * keeps x and y valid and unchanged until the request is done or failed;
 * the server never writes them.  Errors as wxpy_server_submit, plus
 * WXPY_EINVAL for a bad kind, a null or non-8-byte-aligned pointer, or a
 * server in WXPY_SERVE_FUSED mode. */
int wxpy_server_submit_data(wxpy_server *sv, int64_t n, double alpha, const double *x,
                            const double *y, int kind, uint64_t *ticket);

/* State (WXPY_REQ_*) and, once done or failed, the submit -> completion
 * latency in seconds (-1 before).  WXPY_ENOTFOUND for an unknown or released
 * ticket. */
int wxpy_server_poll(wxpy_server *sv, uint64_t ticket, int *state, double *latency_s);

/* Blocks until the request is done (WXPY_OK), failed (WXPY_ECUDA: a launch
 * or copy of its batch failed, or the segmented kernel's tile bounds check
 * fired) or the timeout passes (WXPY_ETIMEOUT). */
int wxpy_server_wait(wxpy_server *sv, uint64_t ticket, double timeout_s, double *latency_s);

/* Device pointers of a done request's x, y, w and its n; valid until release. */
int wxpy_server_result(wxpy_server *sv, uint64_t ticket, const double **x, const double **y,
                       const double **w, int64_t *n);

/* Frees a done or failed request's buffers and slot (WXPY_EBUSY while in flight). */
int wxpy_server_release(wxpy_server *sv, uint64_t ticket);

/* Counters and latency percentiles since the last reset; reset != 0 starts a
 * new window. */
int wxpy_server_get_stats(wxpy_server *sv, int reset, wxpy_server_stats *out);

/* Stops the scheduler after the batches in flight finish, frees everything.
 * Requests not yet finished are dropped.  NULL is a no-op. */
int wxpy_server_destroy(wxpy_server *sv);

typedef struct wxpy_loadgen_config {
    double rate;            /* Poisson arrival rate, requests per second */
    double duration_s;      /* arrivals stop after this */
    int64_t n_min, n_max;   /* request lengths log-uniform on [n_min, n_max] */
    uint64_t seed;          /* arrival gaps, lengths, alphas and request seeds */
    double drain_timeout_s; /* bound on the wait for accepted requests to finish */
} wxpy_loadgen_config;

typedef struct wxpy_loadgen_result {
    int64_t offered, submitted, rejected, completed, failed;
    int64_t max_queue, backlog_at_end, launches;
    double p50_s, p99_s, mean_s, max_s; /* latency of the completed requests */
    double wall_s;                      /* first arrival -> last completion */
    double arrivals_s;                  /* span of the arrivals */
    double elem_per_s, gbs;             /* completed elements (24 B each) / wall_s */
    double mean_batch;
    int32_t drained, reserved;
} wxpy_loadgen_result;

/* A built-in open-loop client.  It submits requests at Poisson arrival times
 * for duration_s, with lengths and alphas drawn from the seeded generator.
 * Its requests release their buffers as soon as they complete, and requests
 * refused at submit count as rejects.  It then waits, up to drain_timeout_s,
 * for the accepted requests to finish.  Blocking.  Resets the statistics
 * window.  WXPY_ETIMEOUT if the load did not drain (the result still holds
 * what was measured). */
int wxpy_server_loadgen(wxpy_server *sv, const wxpy_loadgen_config *cfg,
                        wxpy_loadgen_result *out);

/* ---- seeded synthetic inputs ----------------------------------------------------- */

/* Stream tags used by the library's own synthetic inputs (server requests). */
enum { WXPY_TAG_X = 1, WXPY_TAG_Y = 2, WXPY_TAG_ALPHA = 3, WXPY_TAG_LEN = 4 };

/* dst[i] = lo + (hi - lo) * u(start + i), i in [0, n), where u(k) =
 * (b(k) >> 11) * 2^-53 and b(k) is output k of splitmix64 (Steele, Lea and
 * Flood, OOPSLA 2014) seeded with the key of stream (seed, tag); that key is
 * output number `tag` of splitmix64 seeded with `seed`.  Output k of the
 * generator seeded with s is mix64(s + (k+1) * 0x9E3779B97F4A7C15).
 * The paper has no counterpart: this only makes synthetic inputs (the server
 * fills request vectors with it).  For (lo, hi) = (-1, 1) or (-2, 2) every
 * value is exact, so a host implementation reproduces it bit for bit.
 * Asynchronous on `stream`; dst is a device pointer, 8-byte aligned.
 * WXPY_EINVAL for n < 0, start < 0, hi <= lo or a bad pointer. */
int wxpy_fill_uniform(int64_t n, uint64_t seed, uint32_t tag, int64_t start,
                      double lo, double hi, double *dst, void *stream);

/* ---- fault injection for host-side failure tests ------------------------------ */

/* The next `count` kernel launches made by the library fail with
 * cudaError_t `cuda_error` (returned as WXPY_ECUDA) without touching the GPU.
 * count = 0 clears it.  Process-wide. */
int wxpy_debug_inject_launch_error(int cuda_error, int count);

/* Staged vector kernels launched after this call stop issuing copies at tile
 * `tile` (in the block that owns it), so that block's consumers' bounded wait
 * runs out and wxpy_vecops_status() reports WXPY_ETIMEOUT; no copy is left in
 * flight.  -1 (the default) turns it off.  Process-wide. */
int wxpy_debug_vecops_drop_tile(int64_t tile);

/* Staged reductions launched after this call stop issuing copies before
 * chunk `chunk` (1024 elements; chunk c of tile t is 8t + c), so the owning
 * block's consumers' bounded waits run out and wxpy_reduce_status() reports
 * WXPY_ETIMEOUT; no copy is left in flight.  -1 (the default) turns it off.
 * Process-wide. */
int wxpy_debug_reduce_drop_chunk(int64_t chunk);

#ifdef __cplusplus
}
#endif

#endif /* WXPY_H */
