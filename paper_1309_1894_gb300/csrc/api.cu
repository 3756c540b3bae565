// api.cu -- C ABI of the single-call path: errors, device query, validation and
// classification, the variant space, lookup, launch and the stream split.
#include <cuda_runtime.h>

#include <cstdlib>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "internal.h"
#include "mixed_kernel.cuh"
#include "trace.h"

namespace wx {

// ---------------------------------------------------------------- errors
namespace {
thread_local int t_cuda_error = 0;
thread_local std::string t_message;
}  // namespace

int fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_message = buf;
    return status;
}

int fail_cuda(cudaError_t e, const char *what) {
    t_cuda_error = (int)e;
    t_message = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return WXPY_ECUDA;
}

void clear_error() {
    t_cuda_error = 0;
    t_message.clear();
}

// ---------------------------------------------------------------- device
namespace {
constexpr int kMaxDevices = 64;
std::once_flag g_dev_once[kMaxDevices];
DeviceProps g_dev[kMaxDevices];
cudaError_t g_dev_err[kMaxDevices];
}  // namespace

namespace {
// Programmatic dependent launch of the single-call kernels: on unless the
// environment says WXPY_PDL=0; wxpy_launch_pdl() changes it.
std::atomic<int> g_pdl{-1};
}  // namespace

bool pdl_enabled() {
    int v = g_pdl.load(std::memory_order_relaxed);
    if (v < 0) {
        const char *e = std::getenv("WXPY_PDL");
        v = (e && e[0] == '0') ? 0 : 1;
        int expected = -1;
        if (!g_pdl.compare_exchange_strong(expected, v)) v = expected;
    }
    return v != 0;
}

bool trace_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("WXPY_NVTX");
        return v && v[0] == '1';
    }();
    return on;
}

const DeviceProps *current_device(int *status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *status = fail_cuda(e, "cudaGetDevice");
        return nullptr;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *status = fail(WXPY_EINVAL, "device ordinal %d out of range", dev);
        return nullptr;
    }
    std::call_once(g_dev_once[dev], [dev] {
        DeviceProps &p = g_dev[dev];
        cudaDeviceProp prop;
        cudaError_t err = cudaGetDeviceProperties(&prop, dev);
        g_dev_err[dev] = err;
        if (err != cudaSuccess) return;
        p.device = dev;
        p.sm_count = prop.multiProcessorCount;
        p.cc_major = prop.major;
        p.cc_minor = prop.minor;
        p.l2_bytes = prop.l2CacheSize;
        p.global_bytes = (int64_t)prop.totalGlobalMem;
        std::snprintf(p.name, sizeof p.name, "%.127s", prop.name);  // the field holds 127 chars
    });
    if (g_dev_err[dev] != cudaSuccess) {
        *status = fail_cuda(g_dev_err[dev], "cudaGetDeviceProperties");
        return nullptr;
    }
    *status = WXPY_OK;
    return &g_dev[dev];
}

// ---------------------------------------------------------------- variants
namespace {
template <std::size_t N>
int index_of(const int (&arr)[N], int v) {
    for (std::size_t i = 0; i < N; ++i)
        if (arr[i] == v) return (int)i;
    return -1;
}
}  // namespace

// Mixed-radix id; the offload digit is the most significant, so ids with
// offload 0 are the ids of the space without that knob.
bool decode_variant(int id, Variant *v) {
    if (id < 0 || id >= kVariantCount) return false;
    int r = id;
    const int st = r % 4; r /= 4;
    const int co = r % 4; r /= 4;
    const int ca = r % 3; r /= 3;
    const int gr = r % 5; r /= 5;
    const int th = r % 4; r /= 4;
    const int un = r % 4; r /= 4;
    const int vb = r % 3; r /= 3;
    const int of = r;  // < 4
    *v = Variant{kVecBytes[vb], kUnroll[un], kThreads[th], kBlocksPerSm[gr],
                 kCache[ca], kCarveout[co], kStreams[st], kOffload[of]};
    return true;
}

int encode_variant(const Variant &v) {
    const int vb = index_of(kVecBytes, v.vec_bytes), un = index_of(kUnroll, v.unroll),
              th = index_of(kThreads, v.threads), gr = index_of(kBlocksPerSm, v.blocks_per_sm),
              ca = index_of(kCache, v.cache), co = index_of(kCarveout, v.carveout),
              st = index_of(kStreams, v.streams), of = index_of(kOffload, v.offload);
    if (vb < 0 || un < 0 || th < 0 || gr < 0 || ca < 0 || co < 0 || st < 0 || of < 0) return -1;
    return (((((((of * 3 + vb) * 4 + un) * 4 + th) * 5 + gr) * 3 + ca) * 4 + co) * 4 + st);
}

void to_info(const Variant &v, int id, wxpy_variant_info *out) {
    out->id = id;
    out->vec_bytes = v.vec_bytes;
    out->unroll = v.unroll;
    out->threads = v.threads;
    out->blocks_per_sm = v.blocks_per_sm;
    out->cache = v.cache;
    out->carveout = v.carveout;
    out->streams = v.streams;
    out->fp64_offload = v.offload;
}

static Variant from_info(const wxpy_variant_info &i) {
    return Variant{i.vec_bytes, i.unroll, i.threads, i.blocks_per_sm, i.cache, i.carveout,
                   i.streams, i.fp64_offload};
}

// ---------------------------------------------------------------- classification
int tune_key_of(int bucket, int align, int alias) {
    const int ai = align == 32 ? 0 : (align == 16 ? 1 : 2);
    const int group = ((alias & WXPY_ALIAS_XY) ? 1 : 0) |
                      ((alias & (WXPY_ALIAS_WX | WXPY_ALIAS_WY)) ? 2 : 0);
    return (bucket * 3 + ai) * 4 + group;
}

static bool overlap(uintptr_t a, uintptr_t b, uint64_t bytes) {
    return a < b + bytes && b < a + bytes;
}

int classify(int64_t n, const double *x, const double *y, const double *w, CallClass *c) {
    if (n < 0) return fail(WXPY_EINVAL, "n = %lld is negative", (long long)n);
    const uintptr_t px = (uintptr_t)x, py = (uintptr_t)y, pw = (uintptr_t)w;
    if (n == 0) {
        *c = CallClass{0, 32, 0, -1, -1};
        return WXPY_OK;
    }
    if (!x || !y || !w) return fail(WXPY_EINVAL, "null vector pointer with n = %lld", (long long)n);
    if ((px | py | pw) & 7u) return fail(WXPY_EINVAL, "vector pointers must be 8-byte aligned");
    if (n > (int64_t)(UINT64_MAX / 16 / 8)) return fail(WXPY_EINVAL, "n = %lld too large", (long long)n);
    const uint64_t bytes = (uint64_t)n * 8u;
    if (px + bytes < px || py + bytes < py || pw + bytes < pw)
        return fail(WXPY_EINVAL, "vector range wraps the address space");
    if (pw != px && overlap(pw, px, bytes))
        return fail(WXPY_EOVERLAP, "w partially overlaps x");
    if (pw != py && overlap(pw, py, bytes))
        return fail(WXPY_EOVERLAP, "w partially overlaps y");
    int alias = 0;
    if (px == py) alias |= WXPY_ALIAS_XY;
    if (pw == px) alias |= WXPY_ALIAS_WX;
    if (pw == py) alias |= WXPY_ALIAS_WY;
    int align = 8;
    for (int vb : {32, 16}) {
        if ((px % vb) == (pw % vb) && (py % vb) == (pw % vb)) {
            align = vb;
            break;
        }
    }
    const int64_t off = (int64_t)((pw % (uintptr_t)align) / 8);
    const int64_t vw = align / 8;
    const int head = (int)std::min<int64_t>((vw - off) % vw, n);
    int bucket = 63 - __builtin_clzll((unsigned long long)n);
    *c = CallClass{alias, align, head, bucket, tune_key_of(bucket, align, alias)};
    return WXPY_OK;
}

Variant adjust_variant(const Variant &v, const CallClass &c) {
    Variant a = v;
    if (v.vec_bytes == 32 && c.align < 32) {
        // Mixed alignment: 32-byte stores on w and per-input load widths
        // (mixed_kernel.cuh), whose instances cover unroll 1..4, the
        // non-coherent and coherent cache forms and offload 0, 1 and 3
        // (2 runs as 1).
        a.unroll = std::min(v.unroll, 4);
        if (a.cache == 0) a.cache = 1;
        if (a.offload == 2) a.offload = 1;
    } else {
        a.vec_bytes = std::min(v.vec_bytes, c.align);
    }
    if (a.cache == 1 && (c.alias & (WXPY_ALIAS_WX | WXPY_ALIAS_WY))) a.cache = 2;
    return a;
}

Variant default_variant(const CallClass &c, int64_t n) {
    (void)n;
    // 32-byte accesses, half the sums in the integer pipeline: the variant
    // that streams at the HBM limit on GB300 when nothing is tuned.
    Variant v{32, 2, 256, 0, 1, -1, 1, 1};
    return adjust_variant(v, c);
}

std::atomic<int> g_forced_variant{-1};
std::atomic<int> g_tuned[kTuneKeys];
std::atomic<int> g_tuned_launch_bound[kTuneKeys];
namespace {
struct TunedInit {
    TunedInit() {
        for (auto &t : g_tuned) t.store(-1, std::memory_order_relaxed);
        for (auto &t : g_tuned_launch_bound) t.store(0, std::memory_order_relaxed);
    }
} g_tuned_init;
}  // namespace

// ---------------------------------------------------------------- launching
namespace {
std::atomic<int> g_inject_count{0};
std::atomic<int> g_inject_error{0};

std::mutex g_carveout_mu;
std::unordered_map<const void *, int> g_carveout_set[kMaxDevices];

cudaError_t set_carveout(const void *func, int device, int carveout) {
    std::lock_guard<std::mutex> lk(g_carveout_mu);
    auto &m = g_carveout_set[device];
    auto it = m.find(func);
    const int cur = (it == m.end()) ? -1 : it->second;
    if (cur == carveout) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         carveout);
    if (e == cudaSuccess) m[func] = carveout;
    return e;
}

// Streams and events of the split, per device; the mutex keeps the
// record/wait sequence of one call from interleaving with another's.
struct SplitResources {
    std::mutex mu;
    bool ready = false;
    cudaStream_t streams[8] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[8] = {};
};
SplitResources g_split[kMaxDevices];

int split_resources(int device, SplitResources **out) {
    SplitResources &r = g_split[device];
    if (!r.ready) {
        for (auto &s : r.streams) {
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) return fail_cuda(e, "cudaStreamCreateWithFlags");
        }
        cudaError_t e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail_cuda(e, "cudaEventCreateWithFlags");
        for (auto &ev : r.join) {
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return fail_cuda(e, "cudaEventCreateWithFlags");
        }
        r.ready = true;
    }
    *out = &r;
    return WXPY_OK;
}

// Offset of p relative to w modulo 32 bytes: 0, 8, 16 or 24.
int rel32(const void *p, const void *w) {
    return (int)((((uintptr_t)p % 32u) + 32u - ((uintptr_t)w % 32u)) % 32u);
}

// One contiguous piece [x, x+n) with one kernel launch.
int launch_piece(const Variant &v, const DeviceProps &dp, int xy, int64_t n, double alpha,
                 const double *x, const double *y, double *w, cudaStream_t s) {
    if (n == 0) return WXPY_OK;
    const int vw = v.vec_bytes / 8;
    const int64_t vb = v.vec_bytes;
    const int64_t off = (int64_t)(((uintptr_t)w % (uintptr_t)vb) / 8);
    const int64_t head = std::min<int64_t>((vw - off) % vw, n);
    uint64_t ab;
    std::memcpy(&ab, &alpha, 8);
    SingleArgs a{x, y, w, alpha, n, head, (n - head) / vw, mul_coef_of(ab)};
    const int u_idx = v.unroll == 1 ? 0 : v.unroll == 2 ? 1 : v.unroll == 4 ? 2 : 3;
    const int rx = rel32(x, w), ry = rel32(y, w);
    // 32-byte variants on pointers whose offsets disagree modulo 32 bytes run
    // the mixed-alignment kernel (stores aligned on w, per-input load widths).
    const SingleEntry ent =
        (vw == 4 && (rx | ry) != 0)
            ? mixed_entry(mixed_width(rx), mixed_width(ry), std::min(u_idx, 2), v.cache, xy,
                          v.offload)
            : single_entry(vw, v.offload, u_idx, v.blocks_per_sm > 0 ? 1 : 0, v.cache, xy);
    // Instances that keep many registers live per thread have a smaller launch
    // bound; the block size is capped at it.
    const int threads = std::min(v.threads, ent.max_threads);
    const int64_t per_block = (int64_t)threads * v.unroll;
    const int64_t need = std::max<int64_t>(1, (a.nchunks + per_block - 1) / per_block);
    int64_t grid = need;
    if (v.blocks_per_sm > 0) grid = std::min<int64_t>(need, (int64_t)v.blocks_per_sm * dp.sm_count);
    if (grid > 0x7fffffff) return fail(WXPY_EINVAL, "grid too large for n = %lld", (long long)n);
    cudaError_t e = set_carveout(ent.func, dp.device, v.carveout);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute(carveout)");
    e = injected_launch_error();
    if (e != cudaSuccess) return fail_cuda(e, "wxpy kernel launch (injected)");
    e = ent.launch((unsigned)grid, (unsigned)threads, a, s);
    if (e != cudaSuccess) return fail_cuda(e, "wxpy kernel launch");
    return WXPY_OK;
}
}  // namespace

SingleEntry single_entry(int vw, int offload, int u_idx, int gs, int cache, int xy) {
    switch (vw * 4 + offload) {
        case 4 * 4 + 0: return SingleTable<4, 0>::get(u_idx, gs, cache, xy);
        case 4 * 4 + 1: return SingleTable<4, 1>::get(u_idx, gs, cache, xy);
        case 4 * 4 + 2: return SingleTable<4, 2>::get(u_idx, gs, cache, xy);
        case 4 * 4 + 3: return SingleTable<4, 3>::get(u_idx, gs, cache, xy);
        case 2 * 4 + 0: return SingleTable<2, 0>::get(u_idx, gs, cache, xy);
        case 2 * 4 + 1: return SingleTable<2, 1>::get(u_idx, gs, cache, xy);
        case 2 * 4 + 2: return SingleTable<2, 2>::get(u_idx, gs, cache, xy);
        case 2 * 4 + 3: return SingleTable<2, 3>::get(u_idx, gs, cache, xy);
        case 1 * 4 + 1: return SingleTable<1, 1>::get(u_idx, gs, cache, xy);
        case 1 * 4 + 2: return SingleTable<1, 2>::get(u_idx, gs, cache, xy);
        case 1 * 4 + 3: return SingleTable<1, 3>::get(u_idx, gs, cache, xy);
        default: return SingleTable<1, 0>::get(u_idx, gs, cache, xy);
    }
}

SingleEntry mixed_entry(int kx, int ky, int u_idx, int cache, int xy, int offload) {
    const int c = cache == 2 ? 2 : 1;
    return offload == 3   ? MixedTable<3>::get(kx, ky, u_idx, c, xy)
           : offload != 0 ? MixedTable<1>::get(kx, ky, u_idx, c, xy)
                          : MixedTable<0>::get(kx, ky, u_idx, c, xy);
}

cudaError_t injected_launch_error() {
    if (g_inject_count.load(std::memory_order_relaxed) <= 0) return cudaSuccess;
    if (g_inject_count.fetch_sub(1) > 0) return (cudaError_t)g_inject_error.load();
    return cudaSuccess;
}

int run_variant(const Variant &v, const CallClass &c, int64_t n, double alpha, const double *x,
                const double *y, double *w, cudaStream_t s) {
    if (n == 0) return WXPY_OK;
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const int xy = (c.alias & WXPY_ALIAS_XY) ? 1 : 0;
    // Pieces must stay large enough to be worth a launch each.
    int S = v.streams;
    while (S > 1 && n / S < 65536) S /= 2;
    if (S <= 1) return launch_piece(v, *dp, xy, n, alpha, x, y, w, s);

    // Cut [0, n) into S pieces whose boundaries are 256-byte aligned in w.
    const int64_t o = (int64_t)(((uintptr_t)w % 256u) / 8);
    int64_t bounds[9];
    bounds[0] = 0;
    for (int k = 1; k < S; ++k) {
        int64_t b = ((o + (n / S) * k) / 32) * 32 - o;
        bounds[k] = std::min(n, std::max(bounds[k - 1], b));
    }
    bounds[S] = n;
    SplitResources *r = nullptr;
    std::lock_guard<std::mutex> lk(g_split[dp->device].mu);
    if ((st = split_resources(dp->device, &r)) != WXPY_OK) return st;
    cudaError_t e = cudaEventRecord(r->fork, s);
    if (e != cudaSuccess) return fail_cuda(e, "cudaEventRecord(fork)");
    for (int k = 1; k < S; ++k) {
        e = cudaStreamWaitEvent(r->streams[k], r->fork, 0);
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamWaitEvent(fork)");
    }
    int result = WXPY_OK;
    for (int k = 0; k < S && result == WXPY_OK; ++k) {
        const int64_t b0 = bounds[k], len = bounds[k + 1] - b0;
        cudaStream_t sk = (k == 0) ? s : r->streams[k];
        result = launch_piece(v, *dp, xy, len, alpha, x + b0, y + b0, w + b0, sk);
    }
    // Join every forked stream back, even after a failed launch, so that no
    // stream is left forked from a capture.
    for (int k = 1; k < S; ++k) {
        e = cudaEventRecord(r->join[k], r->streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, r->join[k], 0);
        if (e != cudaSuccess && result == WXPY_OK) result = fail_cuda(e, "stream join");
    }
    return result;
}

}  // namespace wx

using namespace wx;

// ================================================================= C ABI
extern "C" {

const char *wxpy_strerror(int status) {
    switch (status) {
        case WXPY_OK: return "success";
        case WXPY_EINVAL: return "invalid argument";
        case WXPY_EOVERLAP: return "w partially overlaps x or y";
        case WXPY_ENOMEM: return "out of memory";
        case WXPY_EBUDGET: return "request exceeds the memory budget";
        case WXPY_ECUDA: return "CUDA runtime error";
        case WXPY_ETIMEOUT: return "bounded wait timed out";
        case WXPY_ENOTFOUND: return "not found";
        case WXPY_EBUSY: return "resource busy";
        case WXPY_EMISMATCH: return "variant output differs from the reference variant";
        default: return "unknown status";
    }
}

int wxpy_last_cuda_error(void) { return t_cuda_error; }

const char *wxpy_last_error_message(void) { return t_message.c_str(); }

int wxpy_version(void) { return 10000; }

int wxpy_device_query(wxpy_device_info *out) {
    if (!out) return fail(WXPY_EINVAL, "null output");
    int st = WXPY_OK;
    const DeviceProps *p = current_device(&st);
    if (!p) return st;
    std::memset(out, 0, sizeof *out);
    std::snprintf(out->name, sizeof out->name, "%s", p->name);
    out->device = p->device;
    out->sm_count = p->sm_count;
    out->cc_major = p->cc_major;
    out->cc_minor = p->cc_minor;
    out->l2_bytes = p->l2_bytes;
    out->global_bytes = p->global_bytes;
    out->runtime_version = CUDART_VERSION;
    return WXPY_OK;
}

int wxpy_classify(int64_t n, const double *x, const double *y, const double *w,
                  wxpy_class_info *out) {
    if (!out) return fail(WXPY_EINVAL, "null output");
    CallClass c;
    int st = classify(n, x, y, w, &c);
    if (st != WXPY_OK) return st;
    out->alias = c.alias;
    out->align = c.align;
    out->head = c.head;
    out->bucket = c.bucket;
    out->tune_key = c.tune_key;
    out->reserved = 0;
    return WXPY_OK;
}

int wxpy_variant_count(void) { return kVariantCount; }

int wxpy_variant_describe(int id, wxpy_variant_info *out) {
    if (!out) return fail(WXPY_EINVAL, "null output");
    Variant v;
    if (!decode_variant(id, &v)) return fail(WXPY_EINVAL, "variant id %d out of range", id);
    to_info(v, id, out);
    return WXPY_OK;
}

int wxpy_variant_encode(const wxpy_variant_info *v, int *id) {
    if (!v || !id) return fail(WXPY_EINVAL, "null argument");
    const int r = encode_variant(from_info(*v));
    if (r < 0) return fail(WXPY_EINVAL, "variant field outside the space");
    *id = r;
    return WXPY_OK;
}

// WXPY_FORCE_VARIANT: a variant id forced from the process's start, as if
// wxpy_set_variant had been called first (read once; a value that is not a
// valid id is ignored).  An explicit wxpy_set_variant call still wins.
static std::once_flag g_force_env_once;

static void read_force_env() {
    std::call_once(g_force_env_once, [] {
        const char *s = std::getenv("WXPY_FORCE_VARIANT");
        if (!s || !*s) return;
        char *end = nullptr;
        const long id = std::strtol(s, &end, 10);
        if (*end != '\0' || id < 0 || id >= kVariantCount) return;
        int expected = -1;
        g_forced_variant.compare_exchange_strong(expected, (int)id);
    });
}

int wxpy_set_variant(int id) {
    if (id != -1 && (id < 0 || id >= kVariantCount))
        return fail(WXPY_EINVAL, "variant id %d out of range", id);
    read_force_env();
    g_forced_variant.store(id);
    return WXPY_OK;
}

static int select_variant(const CallClass &c, int64_t n, Variant *v, int *source) {
    autoload_tune_cache();
    read_force_env();
    const int forced = g_forced_variant.load(std::memory_order_relaxed);
    if (forced >= 0 && decode_variant(forced, v)) {
        *source = 2;
    } else {
        const int t = c.tune_key >= 0 ? g_tuned[c.tune_key].load(std::memory_order_relaxed) : -1;
        if (t >= 0 && decode_variant(t, v)) {
            *source = 1;
        } else {
            *v = default_variant(c, n);
            *source = 0;
        }
    }
    *v = adjust_variant(*v, c);
    return WXPY_OK;
}

int wxpy_lookup(int64_t n, const double *x, const double *y, const double *w,
                wxpy_variant_info *out, int *tuned) {
    if (!out) return fail(WXPY_EINVAL, "null output");
    CallClass c;
    int st = classify(n, x, y, w, &c);
    if (st != WXPY_OK) return st;
    Variant v;
    int source = 0;
    select_variant(c, n, &v, &source);
    to_info(v, encode_variant(v), out);
    if (tuned) *tuned = source;
    return WXPY_OK;
}

int wxpy(int64_t n, double alpha, const double *x, const double *y, double *w, void *stream) {
    CallClass c;
    int st = classify(n, x, y, w, &c);
    if (st != WXPY_OK || n == 0) return st;
    Variant v;
    int source = 0;
    select_variant(c, n, &v, &source);
    return run_variant(v, c, n, alpha, x, y, w, (cudaStream_t)stream);
}

int wxpy_run_variant(int id, int64_t n, double alpha, const double *x, const double *y,
                     double *w, void *stream) {
    Variant v;
    if (!decode_variant(id, &v)) return fail(WXPY_EINVAL, "variant id %d out of range", id);
    CallClass c;
    int st = classify(n, x, y, w, &c);
    if (st != WXPY_OK || n == 0) return st;
    return run_variant(adjust_variant(v, c), c, n, alpha, x, y, w, (cudaStream_t)stream);
}

int wxpy_reference(int64_t n, double alpha, const double *x, const double *y, double *w,
                   void *stream) {
    CallClass c;
    int st = classify(n, x, y, w, &c);
    if (st != WXPY_OK || n == 0) return st;
    const int64_t grid = (n + 255) / 256;
    if (grid > 0x7fffffff) return fail(WXPY_EINVAL, "n too large for the reference variant");
    SingleArgs a{x, y, w, alpha, n, 0, 0, MulCoef{}};
    cudaError_t e = injected_launch_error();
    if (e == cudaSuccess) e = launch_reference((unsigned)grid, 256u, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "reference kernel launch");
    return WXPY_OK;
}

int wxpy_launch_pdl(int enable, int *previous) {
    if (enable < -1 || enable > 1) return fail(WXPY_EINVAL, "enable must be 0, 1 or -1");
    const int prev = pdl_enabled() ? 1 : 0;
    if (enable >= 0) g_pdl.store(enable);
    if (previous) *previous = prev;
    return WXPY_OK;
}

int wxpy_debug_inject_launch_error(int cuda_error, int count) {
    if (count < 0) return fail(WXPY_EINVAL, "negative count");
    g_inject_error.store(cuda_error);
    g_inject_count.store(count);
    return WXPY_OK;
}

}  // extern "C"
