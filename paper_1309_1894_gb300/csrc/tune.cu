// tune.cu -- the empirical search of paper Sec. 2 applied to the WXPY family,
// and the persisted table of its results.
//
// Sec. 2: the annotated code is turned into variants, each variant is compiled
// and run to obtain its performance and its outputs, the outputs are compared
// with the reference results of the unchanged code, and the best-performing
// variant is the result of the tuning.  Here the variants are the members of
// the kernel family (Sec. 3 knobs: threads per block, blocks per grid, number
// of streams, L1 size via the carveout, unroll; plus vector width and cache
// policy), the reference results come from the plain reference variant run on
// the same inputs, and a candidate whose output differs by a single bit is
// rejected.  The winner is stored per (size bucket, alignment class, alias
// group) cell and used by every later wxpy() call that falls in that cell.
//
// Search order (coordinate descent over the knobs, cheapest to tune first):
//   A. vector width x unroll x cache policy at 256 threads, one-shot grid;
//   B. threads per block x grid mode, from the best of A;
//   C. carveout x stream count, from the best of B.
// Each candidate is timed `reps` times; the median counts.  Before every timed
// run the L2 is flushed by reading a buffer of twice its size, and a device
// delay is queued first so that the host's launch latency is not timed.  The
// device's event timestamps advance in steps of 2.048 us on GB300 (every
// elapsed time of the size sweep is a multiple of it), so a call expected to
// take under 200 us is timed as a batch of back-to-back calls, each on its own
// copy of the inputs in an arena laid out like the tuning buffers (same
// alignment class, none of the copies in L2 after the flush), and the batch
// time is divided by its length.
#include <cuda_runtime.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace wx {
namespace {

std::mutex g_tune_mu;

struct Scratch {
    double *x = nullptr, *y = nullptr, *x0 = nullptr, *wref = nullptr, *wcand = nullptr;
    double *arena = nullptr;  // batch copies: `batch` sets of x, y, w, each `set_elems` long
    int64_t set_elems = 0, y_off = 0, w_off = 0;
    int batch = 1;
    void *flush = nullptr;
    int64_t flush_bytes = 0;
    unsigned long long *count = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
        if (s) cudaStreamSynchronize(s);
        for (void *p : {(void *)x, (void *)y, (void *)x0, (void *)wref, (void *)wcand,
                        (void *)arena, flush, (void *)count})
            if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

// One tuning problem: the call class to reproduce and the pointers that do.
struct Problem {
    int64_t n;
    double alpha;
    const double *x, *y;
    double *w;
    bool w_alias;  // w == x: candidate runs overwrite x
    CallClass cls;
};

int alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WXPY_ENOMEM, "tuner scratch allocation of %zu bytes failed", bytes);
    }
    return WXPY_OK;
}

// Median device time (us per call) of `reps` timed runs; each run is one
// call, or sc.batch back-to-back calls launch(0 .. batch-1) divided by batch.
template <class Launch>
int time_calls(Scratch &sc, int reps, bool flush, Launch &&launch, double *median_us) {
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) {
        int st;
        if (flush && (st = launch_l2_flush(sc.flush, sc.flush_bytes, sc.count, sc.s)) != WXPY_OK)
            return st;
        // long enough to cover the host's enqueueing of the whole batch
        launch_device_delay(20000 + 10000ll * sc.batch, sc.s);
        cudaEventRecord(sc.e0, sc.s);
        for (int i = 0; i < sc.batch; ++i)
            if ((st = launch(i)) != WXPY_OK) return st;
        cudaEventRecord(sc.e1, sc.s);
        cudaError_t e = cudaEventSynchronize(sc.e1);
        if (e != cudaSuccess) return fail_cuda(e, "tuner timing");
        cudaEventElapsedTime(&ms[r], sc.e0, sc.e1);
    }
    std::sort(ms.begin(), ms.end());
    *median_us = 1e3 * (double)ms[reps / 2] / sc.batch;
    return WXPY_OK;
}

// The operands of call i of a batch: the tuning buffers themselves for one
// call or resident timing, else copy i in the arena (same offsets within a
// 256-byte-aligned set, so the same alignment and alias class).
void batch_operands(const Problem &p, const Scratch &sc, bool flush, int i, const double **x,
                    const double **y, double **w) {
    if (sc.batch == 1 || !flush) {
        *x = p.x;
        *y = p.y;
        *w = p.w;
        return;
    }
    double *base = sc.arena + (int64_t)i * sc.set_elems;
    const int64_t xo = (const char *)p.x - (const char *)sc.x;  // off_x bytes
    double *xi = (double *)((char *)base + xo);
    *x = xi;
    *y = p.y == p.x ? xi : base + sc.y_off;
    *w = p.w == p.x ? xi : base + sc.w_off;
}

// Median device time (us per call) of `reps` runs of variant v.
int time_variant(const Variant &v, const Problem &p, Scratch &sc, int reps, bool flush,
                 double *median_us) {
    return time_calls(sc, reps, flush, [&](int i) {
        const double *x, *y;
        double *w;
        batch_operands(p, sc, flush, i, &x, &y, &w);
        return run_variant(v, p.cls, p.n, p.alpha, x, y, w, sc.s);
    }, median_us);
}

// Runs v once on pristine inputs and counts bit mismatches against wref.
int verify_variant(const Variant &v, const Problem &p, Scratch &sc, unsigned long long *bad) {
    const size_t bytes = (size_t)p.n * 8;
    cudaError_t e = cudaSuccess;
    double *out = p.w_alias ? (double *)p.x : sc.wcand;
    if (p.w_alias) e = cudaMemcpyAsync((void *)p.x, sc.x0, bytes, cudaMemcpyDeviceToDevice, sc.s);
    else e = cudaMemsetAsync(sc.wcand, 0xff, bytes, sc.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.count, 0, sizeof(unsigned long long), sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "tuner verify setup");
    int st = run_variant(v, p.cls, p.n, p.alpha, p.x, p.y, out, sc.s);
    if (st != WXPY_OK) return st;
    if ((st = launch_count_mismatch(out, sc.wref, p.n, sc.count, sc.s)) != WXPY_OK) return st;
    e = cudaMemcpyAsync(bad, sc.count, sizeof *bad, cudaMemcpyDeviceToHost, sc.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "tuner verify");
    if (p.w_alias) {  // leave x pristine for the timing runs
        e = cudaMemcpyAsync((void *)p.x, sc.x0, bytes, cudaMemcpyDeviceToDevice, sc.s);
        if (e != cudaSuccess) return fail_cuda(e, "tuner restore");
    }
    return WXPY_OK;
}

struct Candidate {
    Variant v;
    double us;
};

}  // namespace

int tune_impl(int64_t n, unsigned flags, wxpy_tune_result *out) {
    TraceRange trace("wxpy_tune");
    if (n <= 0) return fail(WXPY_EINVAL, "tune needs n > 0");
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const bool xy = flags & WXPY_TUNE_XY, walias = flags & WXPY_TUNE_WALIAS;
    const int off_x = (flags & WXPY_TUNE_ALIGN8) ? 8 : ((flags & WXPY_TUNE_ALIGN16) ? 16 : 0);
    const bool quick = flags & WXPY_TUNE_QUICK;
    const bool flush = !(flags & WXPY_TUNE_RESIDENT);
    if (xy && walias) return fail(WXPY_EINVAL, "choose at most one of XY and WALIAS");

    Scratch sc;
    const size_t vbytes = (size_t)n * 8 + 64;
    if ((st = alloc((void **)&sc.x, vbytes)) || (st = alloc((void **)&sc.y, vbytes)) ||
        (st = alloc((void **)&sc.wref, vbytes)) || (st = alloc((void **)&sc.wcand, vbytes)) ||
        (st = alloc((void **)&sc.count, 64)))
        return st;
    if (walias && (st = alloc((void **)&sc.x0, vbytes))) return st;
    sc.flush_bytes = std::max<int64_t>(2 * dp->l2_bytes, 64 << 20);
    if (flush && (st = alloc(&sc.flush, (size_t)sc.flush_bytes))) return st;
    cudaError_t e = cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e1);
    if (e != cudaSuccess) return fail_cuda(e, "tuner stream/events");
    if (flush && (e = cudaMemsetAsync(sc.flush, 0, (size_t)sc.flush_bytes, sc.s)) != cudaSuccess)
        return fail_cuda(e, "tuner flush init");

    // Inputs: x shifted by off_x bytes relative to y and w reproduces the
    // requested alignment class; values from the seeded generator.
    Problem p;
    p.n = n;
    p.alpha = 0.5;  // keeps repeated in-place runs bounded
    double *xs = (double *)((char *)sc.x + off_x);
    p.x = xs;
    p.y = xy ? xs : sc.y;
    p.w = walias ? xs : sc.wcand;
    p.w_alias = walias;
    if ((st = launch_fill_uniform(xs, n, 20130907ull, 1, 0, -1.0, 1.0, sc.s)) ||
        (st = launch_fill_uniform(sc.y, n, 20130907ull, 2, 0, -1.0, 1.0, sc.s)))
        return st;
    if (walias && (e = cudaMemcpyAsync(sc.x0, xs, (size_t)n * 8, cudaMemcpyDeviceToDevice, sc.s)) !=
                      cudaSuccess)
        return fail_cuda(e, "tuner copy");
    if ((st = classify(n, p.x, p.y, p.w, &p.cls)) != WXPY_OK) return st;

    // Reference results of Sec. 2: the plain variant on the same inputs.
    {
        SingleArgs a{p.x, p.y, sc.wref, p.alpha, n, 0, 0, MulCoef{}};
        e = launch_reference((unsigned)((n + 255) / 256), 256u, a, sc.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
        if (e != cudaSuccess) return fail_cuda(e, "tuner reference run");
    }
    // Repetitions: more for short runs, whose times are noisier.
    const double est_us = 24.0 * (double)n / 6.0e6 + 3.0;  // 6 TB/s = 6e6 bytes per us
    int reps = est_us > 2000 ? 5 : (est_us > 200 ? 7 : 11);
    if (quick) reps = std::max(3, reps / 2);
    reps = tune_reps(reps);
    // Batches of back-to-back calls for short ones (at least about 200 us per
    // timed run), within a 2 GiB arena when each call needs its own copy.
    if (est_us < 200.0) {
        const int64_t vb = ((int64_t)n * 8 + 64 + 255) / 256 * 256;
        sc.set_elems = 3 * vb / 8;
        sc.y_off = vb / 8;
        sc.w_off = 2 * vb / 8;
        int b = (int)std::min(64.0, std::ceil(200.0 / est_us));
        if (flush) b = (int)std::min<int64_t>(b, ((int64_t)2 << 30) / (3 * vb));
        sc.batch = std::max(1, b);
        if (flush && sc.batch > 1) {
            if ((st = alloc((void **)&sc.arena, (size_t)(sc.batch * 3 * vb)))) return st;
            if ((st = launch_fill_uniform(sc.arena, sc.batch * sc.set_elems, 20130907ull, 3, 0, -1.0,
                                          1.0, sc.s)))
                return st;
        }
    }

    int candidates = 0, rejected = 0;
    std::vector<Candidate> all;  // every timed candidate, in search order
    auto consider = [&](const Variant &raw, std::vector<Candidate> &pool) -> int {
        const Variant v = adjust_variant(raw, p.cls);
        for (const auto &c : pool)
            if (std::memcmp(&c.v, &v, sizeof v) == 0) return WXPY_OK;  // duplicate after adjust
        unsigned long long bad = 0;
        int s2 = verify_variant(v, p, sc, &bad);
        if (s2 != WXPY_OK) return s2;
        ++candidates;
        if (bad) {
            ++rejected;
            return WXPY_OK;
        }
        double us = 0;
        if ((s2 = time_variant(v, p, sc, reps, flush, &us)) != WXPY_OK) return s2;
        pool.push_back(Candidate{v, us});
        all.push_back(Candidate{v, us});
        return WXPY_OK;
    };
    auto best_of = [](const std::vector<Candidate> &pool) {
        return *std::min_element(pool.begin(), pool.end(),
                                 [](const Candidate &a, const Candidate &b) { return a.us < b.us; });
    };

    // Stage A: width x unroll x cache x FP64 offload.
    std::vector<Candidate> A;
    for (int vb : kVecBytes)
        for (int u : kUnroll) {
            if (quick && u == 1) continue;
            for (int ca : kCache) {
                if (quick && ca == 0) continue;
                for (int of : kOffload)
                    if ((st = consider(Variant{vb, u, 256, 0, ca, -1, 1, of}, A)) != WXPY_OK)
                        return st;
            }
        }
    if (A.empty()) return fail(WXPY_EMISMATCH, "every candidate differed from the reference");
    Candidate best = best_of(A);
    if (!quick) {
        // Stage B: block size x grid mode.
        std::vector<Candidate> B{best};
        for (int t : kThreads)
            for (int g : kBlocksPerSm) {
                Variant v = best.v;
                v.threads = t;
                v.blocks_per_sm = g;
                if ((st = consider(v, B)) != WXPY_OK) return st;
            }
        best = best_of(B);
        // Stage C: carveout x streams (a split needs pieces of >= 65536 elements).
        std::vector<Candidate> C{best};
        for (int co : kCarveout)
            for (int s : kStreams) {
                if (s > 1 && n / s < 65536) continue;
                Variant v = best.v;
                v.carveout = co;
                v.streams = s;
                if ((st = consider(v, C)) != WXPY_OK) return st;
            }
        best = best_of(C);
    }
    // Re-time the winner against the default and the reference variant.
    double best_us = 0, def_us = 0, ref_us = 0;
    if ((st = time_variant(best.v, p, sc, reps, flush, &best_us)) != WXPY_OK) return st;
    const Variant dv = default_variant(p.cls, n);
    if ((st = time_variant(dv, p, sc, reps, flush, &def_us)) != WXPY_OK) return st;
    st = time_calls(sc, reps, flush, [&](int i) {
        const double *x, *y;
        double *w;
        batch_operands(p, sc, flush, i, &x, &y, &w);
        SingleArgs a{x, y, w, p.alpha, n, 0, 0, MulCoef{}};
        const cudaError_t le = launch_reference((unsigned)((n + 255) / 256), 256u, a, sc.s);
        return le == cudaSuccess ? WXPY_OK : fail_cuda(le, "tuner reference timing");
    }, &ref_us);
    if (st != WXPY_OK) return st;
    // Keep whichever of the winner and the default is faster on the re-timing.
    Variant chosen = best.v;
    double chosen_us = best_us;
    if (def_us < best_us) {
        chosen = dv;
        chosen_us = def_us;
    }
    // Launch-bound cells.  When even the plain reference variant (one element
    // per thread, scalar accesses) times within kTieBand of the winner, no
    // kernel shape changes the call's time: it is the cost of launching and
    // finishing a kernel, not of moving its bytes, and the "winner" is a pick
    // among ties that the timing noise decides.  Such a cell gets a fixed
    // choice instead: the first candidate in search order (the plainest
    // shapes come first) whose time is within the band.
    constexpr double kTieBand = 1.03;
    const double floor_us = std::min(chosen_us, best.us);
    int ties = 0;
    for (const auto &c : all)
        if (c.us <= floor_us * kTieBand) ++ties;
    const bool launch_bound = ref_us <= floor_us * kTieBand;
    if (launch_bound) {
        for (const auto &c : all)
            if (c.us <= floor_us * kTieBand) {
                chosen = c.v;
                chosen_us = c.us;
                break;
            }
    }
    const int id = encode_variant(chosen);
    g_tuned[p.cls.tune_key].store(id);
    g_tuned_launch_bound[p.cls.tune_key].store(launch_bound ? 1 : 0);
    if (out) {
        std::memset(out, 0, sizeof *out);
        to_info(chosen, id, &out->best);
        out->best_us = chosen_us;
        out->default_us = def_us;
        out->reference_us = ref_us;
        const double bytes_per_elem = xy ? 16.0 : 24.0;
        out->best_gbs = bytes_per_elem * (double)n / (chosen_us * 1e-6) / 1e9;
        out->candidates = candidates;
        out->rejected = rejected;
        out->bucket = p.cls.bucket;
        out->tune_key = p.cls.tune_key;
        out->ties = ties;
        out->launch_bound = launch_bound ? 1 : 0;
    }
    return WXPY_OK;
}

// ---------------------------------------------------------------- tune cache file
namespace {

std::string device_key(const DeviceProps &d) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|cc%d.%d|sm%d|cudart%d", d.name, d.cc_major, d.cc_minor,
                  d.sm_count, CUDART_VERSION);
    return buf;
}

// Finds the string value of "key": "..." in s (no escapes are written by save).
bool find_string(const std::string &s, const char *key, std::string *val) {
    const std::string pat = std::string("\"") + key + "\"";
    size_t p = s.find(pat);
    if (p == std::string::npos) return false;
    p = s.find('"', s.find(':', p + pat.size()) + 1);
    if (p == std::string::npos) return false;
    const size_t q = s.find('"', p + 1);
    if (q == std::string::npos) return false;
    *val = s.substr(p + 1, q - p - 1);
    return true;
}

bool find_int(const std::string &s, size_t from, size_t to, const char *key, long long *val) {
    const std::string pat = std::string("\"") + key + "\"";
    size_t p = s.find(pat, from);
    if (p == std::string::npos || p >= to) return false;
    p = s.find(':', p + pat.size());
    if (p == std::string::npos || p >= to) return false;
    char *end = nullptr;
    errno = 0;
    const long long v = std::strtoll(s.c_str() + p + 1, &end, 10);
    if (errno || end == s.c_str() + p + 1) return false;
    *val = v;
    return true;
}

}  // namespace

int cache_save(const char *path) {
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    std::string out = "{\n  \"format\": \"wxpy-tune-1\",\n  \"device\": \"" + device_key(*dp) + "\",";
    {
        const BatchShape bs = current_batch_shape();
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "\n  \"batch_launch\": {\"threads\": %d, \"blocks_per_sm\": %d, "
                      "\"fp64_offload\": %d},",
                      bs.threads, bs.blocks_per_sm, bs.offload);
        out += buf;
        out += "\n  \"batch\": [";
        for (int b = 0; b < kBuckets; ++b) {
            std::snprintf(buf, sizeof buf, "%s\n    {\"bucket\": %d, \"tile\": %d, \"unroll_log2\": %d}",
                          b ? "," : "", b, bs.tile_elems[b], (int)bs.unroll_log2[b]);
            out += buf;
        }
        out += "\n  ],";
    }
    {
        out += "\n  \"vecops\": [";
        bool vfirst = true;
        for (int c = 0; c < WXPY_VEC_CLASSES; ++c) {
            VecPipes vp;
            if (!vecops_tuned_load(c, &vp)) continue;
            char buf[120];
            std::snprintf(buf, sizeof buf,
                          "%s\n    {\"class\": %d, \"add_offload\": %d, \"mul_sixteenths\": %d}",
                          vfirst ? "" : ",", c, vp.add, vp.mul);
            out += buf;
            vfirst = false;
        }
        out += "\n  ],";
    }
    {
        out += "\n  \"reduce\": [";
        bool rfirst = true;
        for (int k = 0; k < 2; ++k) {
            ReduceConfig rc;
            if (!reduce_tuned_load(k, &rc)) continue;
            char buf[140];
            std::snprintf(buf, sizeof buf,
                          "%s\n    {\"kind\": %d, \"variant\": %d, \"mul_sixteenths\": %d, "
                          "\"sum_levels\": %d}",
                          rfirst ? "" : ",", k, rc.variant, rc.mul, rc.suml);
            out += buf;
            rfirst = false;
        }
        out += "\n  ],";
    }
    out += "\n  \"entries\": [";
    bool first = true;
    for (int k = 0; k < kTuneKeys; ++k) {
        const int id = g_tuned[k].load();
        if (id < 0) continue;
        Variant v;
        decode_variant(id, &v);
        char buf[400];
        std::snprintf(buf, sizeof buf,
                      "%s\n    {\"key\": %d, \"bucket\": %d, \"align\": %d, \"group\": %d, "
                      "\"variant\": %d, \"vec_bytes\": %d, \"unroll\": %d, \"threads\": %d, "
                      "\"blocks_per_sm\": %d, \"cache\": %d, \"carveout\": %d, \"streams\": %d, "
                      "\"fp64_offload\": %d, \"launch_bound\": %d}",
                      first ? "" : ",", k, k / 12, (k / 4) % 3 == 0 ? 32 : ((k / 4) % 3 == 1 ? 16 : 8),
                      k % 4, id, v.vec_bytes, v.unroll, v.threads, v.blocks_per_sm, v.cache,
                      v.carveout, v.streams, v.offload, g_tuned_launch_bound[k].load());
        out += buf;
        first = false;
    }
    out += "\n  ]\n}\n";
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(WXPY_EINVAL, "cannot write %s", tmp.c_str());
    const bool ok = std::fwrite(out.data(), 1, out.size(), f) == out.size();
    std::fclose(f);
    if (!ok || std::rename(tmp.c_str(), path) != 0)
        return fail(WXPY_EINVAL, "cannot write %s", path);
    return WXPY_OK;
}

int cache_load(const char *path, const char *expect_device) {
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(WXPY_ENOTFOUND, "cannot open %s", path);
    std::string s;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, r);
    std::fclose(f);
    std::string fmt, dev;
    if (!find_string(s, "format", &fmt) || fmt != "wxpy-tune-1")
        return fail(WXPY_EINVAL, "%s: not a wxpy tune cache", path);
    if (!find_string(s, "device", &dev)) return fail(WXPY_EINVAL, "%s: no device key", path);
    if (expect_device && dev != expect_device)
        return fail(WXPY_EINVAL, "%s was tuned on '%s', this device is '%s'", path, dev.c_str(),
                    expect_device);
    // Parse every entry first; apply only if all are valid.
    std::vector<std::pair<int, int>> entries;
    std::vector<int> entry_lb;  // launch_bound of each entry (0 when the file has none)
    size_t p = s.find("\"entries\"");
    if (p == std::string::npos) return fail(WXPY_EINVAL, "%s: no entries", path);
    const size_t entries_end = s.find(']', p);
    if (entries_end == std::string::npos) return fail(WXPY_EINVAL, "%s: unterminated entries", path);
    while ((p = s.find('{', p + 1)) != std::string::npos && p < entries_end) {
        const size_t q = s.find('}', p);
        if (q == std::string::npos) return fail(WXPY_EINVAL, "%s: unterminated entry", path);
        long long key = -1, id = -1;
        if (!find_int(s, p, q, "key", &key) || !find_int(s, p, q, "variant", &id) || key < 0 ||
            key >= kTuneKeys || id < 0 || id >= kVariantCount)
            return fail(WXPY_EINVAL, "%s: malformed entry", path);
        entries.emplace_back((int)key, (int)id);
        long long lb = 0;
        if (find_int(s, p, q, "launch_bound", &lb) && (lb < 0 || lb > 1))
            return fail(WXPY_EINVAL, "%s: malformed entry", path);
        entry_lb.push_back((int)lb);
        p = q;
    }
    // Optional batch shapes (written by this library since the batched launch).
    BatchShape bs = current_batch_shape();
    bool have_batch = false;
    size_t bpos = s.find("\"batch\"");
    if (bpos != std::string::npos) {
        const size_t bend = s.find(']', bpos);
        if (bend == std::string::npos) return fail(WXPY_EINVAL, "%s: unterminated batch", path);
        size_t q = bpos;
        while ((q = s.find('{', q + 1)) != std::string::npos && q < bend) {
            const size_t r = s.find('}', q);
            long long b = -1, tile = -1, ul = -1;
            if (r == std::string::npos || !find_int(s, q, r, "bucket", &b) ||
                !find_int(s, q, r, "tile", &tile) || !find_int(s, q, r, "unroll_log2", &ul) ||
                b < 0 || b >= kBuckets || tile < 0 || tile > (1 << 30) || (tile % 32) || ul < 0 || ul > 2)
                return fail(WXPY_EINVAL, "%s: malformed batch entry", path);
            bs.tile_elems[b] = (int32_t)tile;
            bs.unroll_log2[b] = (int8_t)ul;
            q = r;
        }
        have_batch = true;
        const size_t lpos = s.find("\"batch_launch\"");
        if (lpos != std::string::npos) {
            const size_t lend = s.find('}', lpos);
            long long th = -1, bps = -1;
            if (lend == std::string::npos || !find_int(s, lpos, lend, "threads", &th) ||
                !find_int(s, lpos, lend, "blocks_per_sm", &bps) || th != 256 || bps < 1 || bps > 32)
                return fail(WXPY_EINVAL, "%s: malformed batch_launch", path);
            bs.threads = (int)th;
            bs.blocks_per_sm = (int)bps;
            long long of = -1;  // optional (files written before the knob existed)
            if (find_int(s, lpos, lend, "fp64_offload", &of)) {
                if (of != 0 && of != 1 && of != 3)
                    return fail(WXPY_EINVAL, "%s: malformed batch_launch", path);
                bs.offload = (int)of;
            }
        }
    }
    // Optional searched splits of the sibling kernels.
    std::vector<std::pair<int, VecPipes>> vec;
    size_t vpos = s.find("\"vecops\"");
    if (vpos != std::string::npos) {
        const size_t vend = s.find(']', vpos);
        if (vend == std::string::npos) return fail(WXPY_EINVAL, "%s: unterminated vecops", path);
        size_t q = vpos;
        while ((q = s.find('{', q + 1)) != std::string::npos && q < vend) {
            const size_t r = s.find('}', q);
            long long c = -1, a = -1, m = -1;
            if (r == std::string::npos || !find_int(s, q, r, "class", &c) ||
                !find_int(s, q, r, "add_offload", &a) || !find_int(s, q, r, "mul_sixteenths", &m) ||
                c < 0 || c >= WXPY_VEC_CLASSES || a < 0 || a > 2 || m < 0 || m > 16)
                return fail(WXPY_EINVAL, "%s: malformed vecops entry", path);
            vec.push_back({(int)c, VecPipes{(int)a, (int)m}});
            q = r;
        }
    }
    // Optional searched configurations of the fused reductions.
    std::vector<std::pair<int, ReduceConfig>> red;
    size_t rpos = s.find("\"reduce\"");
    if (rpos != std::string::npos) {
        const size_t rend = s.find(']', rpos);
        if (rend == std::string::npos) return fail(WXPY_EINVAL, "%s: unterminated reduce", path);
        size_t q = rpos;
        while ((q = s.find('{', q + 1)) != std::string::npos && q < rend) {
            const size_t r = s.find('}', q);
            long long k = -1, v = -1, m = -1, l = -1;
            if (r == std::string::npos || !find_int(s, q, r, "kind", &k) ||
                !find_int(s, q, r, "variant", &v) || !find_int(s, q, r, "mul_sixteenths", &m) ||
                !find_int(s, q, r, "sum_levels", &l) || k < 0 || k > 1 ||
                !reduce_config_valid((int)k, ReduceConfig{(int)v, (int)m, (int)l}))
                return fail(WXPY_EINVAL, "%s: malformed reduce entry", path);
            red.push_back({(int)k, ReduceConfig{(int)v, (int)m, (int)l}});
            q = r;
        }
    }
    for (size_t i = 0; i < entries.size(); ++i) {
        g_tuned[entries[i].first].store(entries[i].second);
        g_tuned_launch_bound[entries[i].first].store(entry_lb[i]);
    }
    if (have_batch) set_batch_shape(bs);
    for (auto &cv : vec) vecops_tuned_store(cv.first, &cv.second);
    for (auto &rc : red) reduce_tuned_store(rc.first, &rc.second);
    return WXPY_OK;
}

std::string current_device_key(int *status) {
    const DeviceProps *dp = current_device(status);
    return dp ? device_key(*dp) : std::string();
}

namespace {
std::once_flag g_autoload_once;
}

int tune_reps(int fallback) {
    const char *s = std::getenv("WXPY_TUNE_REPS");
    if (!s || !*s) return fallback;
    char *end = nullptr;
    const long v = std::strtol(s, &end, 10);
    return (*end == '\0' && v >= 1 && v <= 101) ? (int)v : fallback;
}

void autoload_tune_cache() {
    std::call_once(g_autoload_once, [] {
        const char *path = std::getenv("WXPY_TUNE_CACHE");
        if (!path || !*path) return;
        int st = WXPY_OK;
        const std::string key = current_device_key(&st);
        if (st == WXPY_OK) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            cache_load(path, key.c_str());
        }
        clear_error();
    });
}

}  // namespace wx

using namespace wx;

extern "C" {

int wxpy_tune(int64_t n, unsigned flags, wxpy_tune_result *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return tune_impl(n, flags, out);
}

int wxpy_tune_get(int tune_key, int *variant_id) {
    if (tune_key < 0 || tune_key >= kTuneKeys || !variant_id)
        return fail(WXPY_EINVAL, "bad tune key %d", tune_key);
    *variant_id = g_tuned[tune_key].load();
    return WXPY_OK;
}

int wxpy_tune_set(int tune_key, int variant_id) {
    if (tune_key < 0 || tune_key >= kTuneKeys) return fail(WXPY_EINVAL, "bad tune key %d", tune_key);
    if (variant_id < -1 || variant_id >= kVariantCount)
        return fail(WXPY_EINVAL, "bad variant id %d", variant_id);
    g_tuned[tune_key].store(variant_id);
    g_tuned_launch_bound[tune_key].store(0);
    return WXPY_OK;
}

int wxpy_tune_clear(void) {
    for (auto &t : g_tuned) t.store(-1);
    for (auto &t : g_tuned_launch_bound) t.store(0);
    for (int c = 0; c < WXPY_VEC_CLASSES; ++c) vecops_tuned_store(c, nullptr);
    for (int k = 0; k < 2; ++k) reduce_tuned_store(k, nullptr);
    return WXPY_OK;
}

int wxpy_tune_cache_save(const char *path) {
    if (!path) return fail(WXPY_EINVAL, "null path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return cache_save(path);
}

int wxpy_tune_cache_load(const char *path, int check_device) {
    if (!path) return fail(WXPY_EINVAL, "null path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!check_device) return cache_load(path, nullptr);
    int st = WXPY_OK;
    const std::string key = current_device_key(&st);
    if (st != WXPY_OK) return st;
    return cache_load(path, key.c_str());
}

}  // extern "C"
