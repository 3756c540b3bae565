/* wxpy_cpu.c -- the host VecWXPY family: validation, the variant space, a
 * persistent thread pool, and the empirical search of paper Sec. 2 over
 * (flavour, kernel, threads).  See include/wxpy_cpu.h for the contract. */
#define _GNU_SOURCE
#include <errno.h>
#include <pthread.h>
#include <stdarg.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#include <unistd.h>

#include "cpu_internal.h"
#include "wxpy_cpu.h"

#ifndef WXC_FLAVOUR_FLAGS
#define WXC_FLAVOUR_FLAGS "-O2 -fno-tree-vectorize", "-O3", "-O3 (target flags)"
#endif

static const char *const kFlavourFlags[WXC_FLAVOURS] = {WXC_FLAVOUR_FLAGS};
static const wxc_kernel_fn *const kTables[WXC_FLAVOURS] = {wxc_table_f0, wxc_table_f1,
                                                           wxc_table_f2};
static const int kVec[WXC_KERNELS] = {0, 1, 1, 1, 2, 2, 2, 4, 4, 4, 8, 8, 8};
static const int kUnroll[WXC_KERNELS] = {0, 1, 2, 4, 1, 2, 4, 1, 2, 4, 1, 2, 4};

/* ---- errors ------------------------------------------------------------ */

static __thread char t_err[256];

static int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof t_err, fmt, ap);
    va_end(ap);
    return status;
}

const char *wxpy_cpu_last_error(void) { return t_err; }

/* ---- thread counts: 1, 2, 4, ... below the CPU count, then the count ---- */

#define MAX_THREADS 256
static int g_nthr_opts = 0;
static int g_thr_opts[16];
static pthread_once_t g_thr_once = PTHREAD_ONCE_INIT;

static void init_thread_options(void) {
    long ncpu = sysconf(_SC_NPROCESSORS_ONLN);
    if (ncpu < 1) ncpu = 1;
    if (ncpu > MAX_THREADS) ncpu = MAX_THREADS;
    int k = 0;
    for (long t = 1; t < ncpu && k < 15; t *= 2) g_thr_opts[k++] = (int)t;
    g_thr_opts[k++] = (int)ncpu;
    g_nthr_opts = k;
}

static int thread_options(void) {
    pthread_once(&g_thr_once, init_thread_options);
    return g_nthr_opts;
}

int wxpy_cpu_variant_count(void) { return WXC_FLAVOURS * WXC_KERNELS * thread_options(); }

static int encode(int flavour, int kernel, int t_idx) {
    return (flavour * WXC_KERNELS + kernel) * thread_options() + t_idx;
}

int wxpy_cpu_variant_describe(int id, wxpy_cpu_variant_info *out) {
    const int nt = thread_options();
    if (id < 0 || id >= wxpy_cpu_variant_count()) return fail(WXPY_EINVAL, "bad variant id %d", id);
    if (!out) return fail(WXPY_EINVAL, "null output");
    const int t_idx = id % nt, fk = id / nt;
    out->id = id;
    out->flavour = fk / WXC_KERNELS;
    out->kernel = fk % WXC_KERNELS;
    out->vec = kVec[out->kernel];
    out->unroll = kUnroll[out->kernel];
    out->threads = g_thr_opts[t_idx];
    out->flags = kFlavourFlags[out->flavour];
    return WXPY_OK;
}

int wxpy_cpu_baseline_variant(void) { return encode(1, 0, 0); }
int wxpy_cpu_reference_variant(void) { return encode(0, 0, 0); }

/* ---- validation (the rules of wxpy()) ----------------------------------- */

static int validate(int64_t n, const double *x, const double *y, const double *w) {
    if (n < 0) return fail(WXPY_EINVAL, "n = %lld is negative", (long long)n);
    if (n == 0) return WXPY_OK;
    if (n > ((int64_t)1 << 56)) return fail(WXPY_EINVAL, "n too large");
    if (!x || !y || !w) return fail(WXPY_EINVAL, "null pointer");
    if (((uintptr_t)x | (uintptr_t)y | (uintptr_t)w) & 7u)
        return fail(WXPY_EINVAL, "pointers must be 8-byte aligned");
    const uintptr_t bytes = (uintptr_t)n * 8, pw = (uintptr_t)w;
    const uintptr_t in[2] = {(uintptr_t)x, (uintptr_t)y};
    for (int k = 0; k < 2; ++k)
        if (in[k] != pw && in[k] < pw + bytes && pw < in[k] + bytes)
            return fail(WXPY_EOVERLAP, "w partially overlaps %c", k ? 'y' : 'x');
    return WXPY_OK;
}

/* ---- the pool: workers 1 .. T-1 take chunks 1 .. T-1, the caller chunk 0 -- */

struct job {
    wxc_kernel_fn fn;
    int64_t n;
    double a;
    const double *x, *y;
    double *w;
    int parts;
};

static pthread_mutex_t g_call_mu = PTHREAD_MUTEX_INITIALIZER; /* one pooled call at a time */
static pthread_mutex_t g_mu = PTHREAD_MUTEX_INITIALIZER;
static pthread_cond_t g_work = PTHREAD_COND_INITIALIZER;
static pthread_cond_t g_done = PTHREAD_COND_INITIALIZER;
static struct job g_job;
static uint64_t g_gen = 0;
static int g_pending = 0;
static int g_workers = 0;

static void chunk(const struct job *j, int part, int64_t *lo, int64_t *hi) {
    /* contiguous parts, boundaries rounded to 8 elements (64 bytes) */
    int64_t b0 = (int64_t)((__int128)j->n * part / j->parts);
    int64_t b1 = (int64_t)((__int128)j->n * (part + 1) / j->parts);
    b0 = part == 0 ? 0 : ((b0 + 7) & ~(int64_t)7);
    b1 = part + 1 == j->parts ? j->n : ((b1 + 7) & ~(int64_t)7);
    if (b0 > j->n) b0 = j->n;
    if (b1 > j->n) b1 = j->n;
    *lo = b0;
    *hi = b1 > b0 ? b1 : b0;
}

static void run_part(const struct job *j, int part) {
    int64_t lo, hi;
    chunk(j, part, &lo, &hi);
    if (hi > lo) j->fn(hi - lo, j->a, j->x + lo, j->y + lo, j->w + lo);
}

static void *worker(void *arg) {
    const int id = (int)(intptr_t)arg;
    uint64_t seen = 0;
    pthread_mutex_lock(&g_mu);
    for (;;) {
        while (g_gen == seen) pthread_cond_wait(&g_work, &g_mu);
        seen = g_gen;
        const struct job j = g_job;
        pthread_mutex_unlock(&g_mu);
        if (id < j.parts) run_part(&j, id);
        pthread_mutex_lock(&g_mu);
        if (id < j.parts && --g_pending == 0) pthread_cond_signal(&g_done);
    }
    return NULL;
}

static int ensure_workers(int needed) {
    while (g_workers < needed) {
        pthread_t th;
        pthread_attr_t at;
        pthread_attr_init(&at);
        pthread_attr_setdetachstate(&at, PTHREAD_CREATE_DETACHED);
        const int rc = pthread_create(&th, &at, worker, (void *)(intptr_t)(g_workers + 1));
        pthread_attr_destroy(&at);
        if (rc != 0) return fail(WXPY_ENOMEM, "cannot start a worker thread (%d)", rc);
        ++g_workers;
    }
    return WXPY_OK;
}

static int run_pooled(wxc_kernel_fn fn, int threads, int64_t n, double a, const double *x,
                      const double *y, double *w) {
    if (threads <= 1 || n < 8 * (int64_t)threads) {
        fn(n, a, x, y, w);
        return WXPY_OK;
    }
    pthread_mutex_lock(&g_call_mu);
    pthread_mutex_lock(&g_mu);
    int st = ensure_workers(threads - 1);
    if (st != WXPY_OK) {
        pthread_mutex_unlock(&g_mu);
        pthread_mutex_unlock(&g_call_mu);
        return st;
    }
    g_job = (struct job){fn, n, a, x, y, w, threads};
    g_pending = threads - 1;
    ++g_gen;
    pthread_cond_broadcast(&g_work);
    pthread_mutex_unlock(&g_mu);
    const struct job j = {fn, n, a, x, y, w, threads};
    run_part(&j, 0);
    pthread_mutex_lock(&g_mu);
    while (g_pending > 0) pthread_cond_wait(&g_done, &g_mu);
    pthread_mutex_unlock(&g_mu);
    pthread_mutex_unlock(&g_call_mu);
    return WXPY_OK;
}

/* ---- calls ----------------------------------------------------------------- */

static int run_id(int id, int64_t n, double a, const double *x, const double *y, double *w) {
    wxpy_cpu_variant_info v;
    int st = wxpy_cpu_variant_describe(id, &v);
    if (st != WXPY_OK) return st;
    return run_pooled(kTables[v.flavour][v.kernel], v.threads, n, a, x, y, w);
}

int wxpy_cpu_run_variant(int id, int64_t n, double alpha, const double *x, const double *y,
                         double *w) {
    if (id < 0 || id >= wxpy_cpu_variant_count()) return fail(WXPY_EINVAL, "bad variant id %d", id);
    int st = validate(n, x, y, w);
    if (st != WXPY_OK || n == 0) return st;
    return run_id(id, n, alpha, x, y, w);
}

static _Atomic int g_tuned[64] = {
    -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
    -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
    -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};

static int bucket_of(int64_t n) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
    return b;
}

int wxpy_cpu(int64_t n, double alpha, const double *x, const double *y, double *w) {
    int st = validate(n, x, y, w);
    if (st != WXPY_OK || n == 0) return st;
    int id = atomic_load(&g_tuned[bucket_of(n)]);
    if (id < 0 || id >= wxpy_cpu_variant_count()) id = wxpy_cpu_baseline_variant();
    return run_id(id, n, alpha, x, y, w);
}

int wxpy_cpu_tune_get(int bucket, int *variant_id) {
    if (bucket < 0 || bucket >= 64 || !variant_id) return fail(WXPY_EINVAL, "bad bucket %d", bucket);
    *variant_id = atomic_load(&g_tuned[bucket]);
    return WXPY_OK;
}

int wxpy_cpu_tune_set(int bucket, int variant_id) {
    if (bucket < 0 || bucket >= 64) return fail(WXPY_EINVAL, "bad bucket %d", bucket);
    if (variant_id < -1 || variant_id >= wxpy_cpu_variant_count())
        return fail(WXPY_EINVAL, "bad variant id %d", variant_id);
    atomic_store(&g_tuned[bucket], variant_id);
    return WXPY_OK;
}

int wxpy_cpu_tune_clear(void) {
    for (int b = 0; b < 64; ++b) atomic_store(&g_tuned[b], -1);
    return WXPY_OK;
}

/* ---- the tuning table on disk ------------------------------------------------ */

/* The machine a table is valid for: architecture, online CPU count, and the
 * flags of the target flavour (variant ids index the flavour list). */
static void machine_key(char *buf, size_t len) {
    const char *arch =
#if defined(__aarch64__)
        "aarch64";
#elif defined(__x86_64__)
        "x86_64";
#else
        "other";
#endif
    snprintf(buf, len, "%s|cpus%d|%s", arch, g_thr_opts[thread_options() - 1], kFlavourFlags[2]);
}

int wxpy_cpu_tune_cache_save(const char *path) {
    if (!path) return fail(WXPY_EINVAL, "null path");
    char key[256], tmp[4096];
    machine_key(key, sizeof key);
    snprintf(tmp, sizeof tmp, "%s.tmp", path);
    FILE *f = fopen(tmp, "wb");
    if (!f) return fail(WXPY_EINVAL, "cannot write %s", tmp);
    int ok = fprintf(f, "{\n  \"format\": \"wxpy-cpu-tune-1\",\n  \"machine\": \"%s\",\n"
                        "  \"entries\": [", key) > 0;
    int first = 1;
    for (int b = 0; b < 64 && ok; ++b) {
        const int id = atomic_load(&g_tuned[b]);
        if (id < 0) continue;
        wxpy_cpu_variant_info v;
        if (wxpy_cpu_variant_describe(id, &v) != WXPY_OK) continue;
        ok = fprintf(f, "%s\n    {\"bucket\": %d, \"variant\": %d, \"flavour\": %d, "
                        "\"kernel\": %d, \"threads\": %d}",
                     first ? "" : ",", b, id, v.flavour, v.kernel, v.threads) > 0;
        first = 0;
    }
    ok = ok && fprintf(f, "\n  ]\n}\n") > 0;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp, path) != 0) return fail(WXPY_EINVAL, "cannot write %s", path);
    return WXPY_OK;
}

/* Value of integer field `name` inside [from, to) of s; 0 when absent. */
static int find_int_field(const char *from, const char *to, const char *name, long *out) {
    char pat[64];
    snprintf(pat, sizeof pat, "\"%s\"", name);
    const char *p = strstr(from, pat);
    if (!p || p >= to) return 0;
    p = strchr(p + strlen(pat), ':');
    if (!p || p >= to) return 0;
    char *end = NULL;
    errno = 0;
    const long v = strtol(p + 1, &end, 10);
    if (errno || end == p + 1 || end > to) return 0;
    *out = v;
    return 1;
}

int wxpy_cpu_tune_cache_load(const char *path, int check_machine) {
    if (!path) return fail(WXPY_EINVAL, "null path");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(WXPY_ENOTFOUND, "cannot open %s", path);
    char *s = malloc(1 << 20);
    if (!s) {
        fclose(f);
        return fail(WXPY_ENOMEM, "cache buffer");
    }
    const size_t len = fread(s, 1, (1 << 20) - 1, f);
    fclose(f);
    s[len] = 0;
    int st = WXPY_OK;
    if (!strstr(s, "\"format\": \"wxpy-cpu-tune-1\"")) st = fail(WXPY_EINVAL, "%s: not a cpu tune cache", path);
    if (st == WXPY_OK && check_machine) {
        char key[256], pat[300];
        machine_key(key, sizeof key);
        snprintf(pat, sizeof pat, "\"machine\": \"%s\"", key);
        if (!strstr(s, pat)) st = fail(WXPY_EINVAL, "%s was tuned on another machine", path);
    }
    /* parse every entry first; apply only if all are valid */
    int ids[64];
    for (int b = 0; b < 64; ++b) ids[b] = -2;
    const char *p = st == WXPY_OK ? strstr(s, "\"entries\"") : NULL;
    if (st == WXPY_OK && !p) st = fail(WXPY_EINVAL, "%s: no entries", path);
    const char *end = p ? strchr(p, ']') : NULL;
    if (st == WXPY_OK && !end) st = fail(WXPY_EINVAL, "%s: unterminated entries", path);
    while (st == WXPY_OK && (p = strchr(p + 1, '{')) != NULL && p < end) {
        const char *q = strchr(p, '}');
        long b = -1, id = -1;
        if (!q || q > end || !find_int_field(p, q, "bucket", &b) ||
            !find_int_field(p, q, "variant", &id) || b < 0 || b >= 64 || id < 0 ||
            id >= wxpy_cpu_variant_count())
            st = fail(WXPY_EINVAL, "%s: malformed entry", path);
        else
            ids[b] = (int)id;
        p = q;
    }
    free(s);
    if (st != WXPY_OK) return st;
    for (int b = 0; b < 64; ++b)
        if (ids[b] >= 0) atomic_store(&g_tuned[b], ids[b]);
    return WXPY_OK;
}

/* ---- the search ------------------------------------------------------------ */

static double now_us(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec * 1e6 + (double)ts.tv_nsec * 1e-3;
}

/* Seeded inputs (splitmix64 outputs mapped to [-1, 1) exactly). */
static void fill(double *v, int64_t n, uint64_t seed) {
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = (double)(int64_t)(z >> 11) * 0x1p-52 - 1.0;
    }
}

struct scratch {
    double *x, *y, *w, *ref;
    unsigned char *flush;
    size_t flush_bytes;
};

static void scratch_free(struct scratch *s) {
    free(s->x);
    free(s->y);
    free(s->w);
    free(s->ref);
    free(s->flush);
}

/* Median over five samples of the time of one call; a sample times `calls`
 * back-to-back calls (enough for about 2^20 elements, so that short calls are
 * not lost in timer resolution) and divides. */
static int time_id(int id, int64_t n, double a, struct scratch *s, double *median_us) {
    double t[5];
    const int64_t calls = n >= ((int64_t)1 << 20) ? 1 : ((int64_t)1 << 20) / n;
    for (int r = 0; r < 5; ++r) {
        if (s->flush) {  /* rewrite a buffer larger than the last-level cache */
            memset(s->flush, r + 1, s->flush_bytes);
            (void)*(volatile unsigned char *)(s->flush + (size_t)r * 4096);
        }
        const double t0 = now_us();
        for (int64_t c = 0; c < calls; ++c) {
            int st = run_id(id, n, a, s->x, s->y, s->w);
            if (st != WXPY_OK) return st;
        }
        t[r] = (now_us() - t0) / (double)calls;
    }
    for (int i = 1; i < 5; ++i)
        for (int k = i; k > 0 && t[k] < t[k - 1]; --k) {
            const double tmp = t[k];
            t[k] = t[k - 1];
            t[k - 1] = tmp;
        }
    *median_us = t[2];
    return WXPY_OK;
}

static int verify_id(int id, int64_t n, double a, struct scratch *s, int *bad) {
    memset(s->w, 0xff, (size_t)n * 8);
    int st = run_id(id, n, a, s->x, s->y, s->w);
    if (st != WXPY_OK) return st;
    *bad = memcmp(s->w, s->ref, (size_t)n * 8) != 0;
    return WXPY_OK;
}

int wxpy_cpu_tune(int64_t n, unsigned flags, wxpy_cpu_tune_result *out) {
    if (n <= 0) return fail(WXPY_EINVAL, "tune needs n > 0");
    struct scratch s = {0};
    const size_t bytes = (size_t)n * 8;
    if (posix_memalign((void **)&s.x, 64, bytes) || posix_memalign((void **)&s.y, 64, bytes) ||
        posix_memalign((void **)&s.w, 64, bytes) || posix_memalign((void **)&s.ref, 64, bytes)) {
        scratch_free(&s);
        return fail(WXPY_ENOMEM, "tuner scratch of 4 x %zu bytes", bytes);
    }
    if (!(flags & WXPY_CPU_TUNE_WARM) && 3 * bytes < ((size_t)1 << 30)) {
        s.flush_bytes = (size_t)256 << 20;
        s.flush = malloc(s.flush_bytes);
        if (!s.flush) {
            scratch_free(&s);
            return fail(WXPY_ENOMEM, "tuner flush buffer");
        }
    }
    fill(s.x, n, 20130907u + 1);
    fill(s.y, n, 20130907u + 2);
    const double a = -1.25;
    int st = run_id(wxpy_cpu_reference_variant(), n, a, s.x, s.y, s.ref);
    int candidates = 0, rejected = 0;
    int best = -1, best1 = -1;
    double best_us = 0, best1_us = 0, base_us = 0, ref_us = 0;
    /* stage 1: every (flavour, kernel) on one thread */
    for (int f = 0; f < WXC_FLAVOURS && st == WXPY_OK; ++f)
        for (int k = 0; k < WXC_KERNELS && st == WXPY_OK; ++k) {
            const int id = encode(f, k, 0);
            int bad = 0;
            if ((st = verify_id(id, n, a, &s, &bad)) != WXPY_OK) break;
            ++candidates;
            if (bad) {
                ++rejected;
                continue;
            }
            double us = 0;
            if ((st = time_id(id, n, a, &s, &us)) != WXPY_OK) break;
            if (id == wxpy_cpu_baseline_variant()) base_us = us;
            if (id == wxpy_cpu_reference_variant()) ref_us = us;
            if (best1 < 0 || us < best1_us) {
                best1 = id;
                best1_us = us;
            }
        }
    best = best1;
    best_us = best1_us;
    /* stage 2: thread counts for the best one-thread kernel */
    if (st == WXPY_OK && best1 >= 0 && !(flags & WXPY_CPU_TUNE_SINGLE)) {
        const int fk = best1 / thread_options();
        for (int t = 1; t < thread_options() && st == WXPY_OK; ++t) {
            const int id = fk * thread_options() + t;
            int bad = 0;
            if ((st = verify_id(id, n, a, &s, &bad)) != WXPY_OK) break;
            ++candidates;
            if (bad) {
                ++rejected;
                continue;
            }
            double us = 0;
            if ((st = time_id(id, n, a, &s, &us)) != WXPY_OK) break;
            if (us < best_us) {
                best = id;
                best_us = us;
            }
        }
    }
    scratch_free(&s);
    if (st != WXPY_OK) return st;
    if (best < 0) return fail(WXPY_EMISMATCH, "every candidate differed from the reference");
    const int b = bucket_of(n);
    atomic_store(&g_tuned[b], best);
    if (out) {
        out->best = best;
        out->best_single = best1;
        out->candidates = candidates;
        out->rejected = rejected;
        out->bucket = b;
        out->reserved = 0;
        out->best_us = best_us;
        out->best_single_us = best1_us;
        out->baseline_us = base_us;
        out->reference_us = ref_us;
    }
    return WXPY_OK;
}
