// reduce_tune.cu -- the empirical search of paper Sec. 2 applied to the
// fused reductions (wxpy_norm2, wxpy_dot).
//
// Sec. 2: variants are run to obtain their performance and their outputs, the
// outputs are compared with the reference results of the unchanged code, and
// the best-performing variant is kept.  Here a variant is a configuration of
// the fused kernel: its form (register-loaded or one of the staged shapes),
// the share of tiles whose products run as exactly rounded integer-pipeline
// products, and, for the squared 2-norm, how many in-thread tree levels run
// as integer-pipeline sums.  The reference results are those of the
// register-loaded form with every operation in FP64 on the same inputs; a
// configuration whose w or result differs by a single bit is rejected.
// Candidates, per operation: the register-loaded form at product shares 0, 4,
// .., 16 sixteenths; for norm2, one to three integer tree levels at the best
// share and at half of it; the three staged shapes and the three warp-tiled
// shapes at the best share; for norm2, 2, 4 and 6 integer tree levels in the
// fastest warp-tiled shape.  Timing:
// median of five runs of three back-to-back calls, each run after an L2 flush
// and a short device delay (w never aliases an input here, so no restore is
// needed).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace wx {
namespace {

std::mutex g_rtune_mu;

constexpr int kReps = 5;
constexpr double kAlpha = -0.625;

struct RScratch {
    double *x = nullptr, *y = nullptr, *z = nullptr, *w = nullptr, *ref_w = nullptr;
    double *res = nullptr;  // [0] the candidate's result, [1] the reference result
    void *ws = nullptr, *flush = nullptr;
    int64_t ws_bytes = 0, flush_bytes = 0;
    unsigned long long *count = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~RScratch() {
        if (s) cudaStreamSynchronize(s);
        for (void *p : {(void *)x, (void *)y, (void *)z, (void *)w, (void *)ref_w, (void *)res, ws,
                        flush, (void *)count})
            if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

int ralloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(WXPY_ENOMEM, "reduction tuner scratch allocation of %zu bytes failed", bytes);
    }
    return WXPY_OK;
}

int run_once(int kind, int64_t n, ReduceConfig c, RScratch &sc, double *w, double *res) {
    return reduce_run(kind, n, kAlpha, sc.x, sc.y, w, kind == 1 ? sc.z : nullptr, res, sc.ws,
                      sc.ws_bytes, c, sc.s);
}

// Median device time (us per call) of kReps timed runs, each kBatch back-to-
// back calls (the event timestamps advance in 2.048 us steps on GB300; the
// operands exceed the L2, so every call reads them from memory).
constexpr int kBatch = 3;

int time_config(int kind, int64_t n, ReduceConfig c, RScratch &sc, double *median_us) {
    const int reps = tune_reps(kReps);
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) {
        int st;
        if ((st = launch_l2_flush(sc.flush, sc.flush_bytes, sc.count, sc.s)) != WXPY_OK) return st;
        launch_device_delay(20000 * kBatch, sc.s);
        cudaEventRecord(sc.e0, sc.s);
        for (int b = 0; b < kBatch; ++b)
            if ((st = run_once(kind, n, c, sc, sc.w, sc.res)) != WXPY_OK) return st;
        cudaEventRecord(sc.e1, sc.s);
        cudaError_t e = cudaEventSynchronize(sc.e1);
        if (e != cudaSuccess) return fail_cuda(e, "reduction tuner timing");
        cudaEventElapsedTime(&ms[r], sc.e0, sc.e1);
    }
    std::sort(ms.begin(), ms.end());
    *median_us = 1e3 * (double)ms[reps / 2] / kBatch;
    return WXPY_OK;
}

// Runs configuration c once; *bad = elements of w differing from the
// reference bitwise, plus one when the result's bits differ.
int run_checked(int kind, int64_t n, ReduceConfig c, RScratch &sc, unsigned long long *bad) {
    int st;
    cudaError_t e = cudaMemsetAsync(sc.w, 0xFF, (size_t)n * 8, sc.s);  // no stale w passes
    if (e != cudaSuccess) return fail_cuda(e, "reduction tuner verify");
    if ((st = run_once(kind, n, c, sc, sc.w, sc.res)) != WXPY_OK) return st;
    e = cudaMemsetAsync(sc.count, 0, sizeof(unsigned long long), sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "reduction tuner verify");
    if ((st = launch_count_mismatch(sc.w, sc.ref_w, n, sc.count, sc.s)) != WXPY_OK) return st;
    double r[2];
    e = cudaMemcpyAsync(bad, sc.count, sizeof *bad, cudaMemcpyDeviceToHost, sc.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, sc.res, sizeof r, cudaMemcpyDeviceToHost, sc.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "reduction tuner verify");
    uint64_t b0, b1;
    std::memcpy(&b0, &r[0], 8);
    std::memcpy(&b1, &r[1], 8);
    *bad += b0 != b1;
    return WXPY_OK;
}

int tune_kind(int kind, int64_t n, RScratch &sc, wxpy_reduce_tune_result *res) {
    int st;
    // reference: register-loaded, every operation in FP64
    if ((st = run_once(kind, n, ReduceConfig{0, 0, 0}, sc, sc.ref_w, sc.res + 1)) != WXPY_OK)
        return st;
    int candidates = 0, rejected = 0;
    ReduceConfig best{0, 0, 0};
    double best_us = 0.0;
    bool have = false;
    double last_us = 0.0;  // the last candidate's time, 0 when it was rejected
    auto consider = [&](ReduceConfig c) -> int {
        ++candidates;
        last_us = 0.0;
        unsigned long long mism = 0;
        int s2 = run_checked(kind, n, c, sc, &mism);
        if (s2 != WXPY_OK) return s2;
        if (mism) {
            ++rejected;
            return WXPY_OK;
        }
        double us = 0.0;
        if ((s2 = time_config(kind, n, c, sc, &us)) != WXPY_OK) return s2;
        last_us = us;
        if (!have || us < best_us) {
            best = c;
            best_us = us;
            have = true;
        }
        return WXPY_OK;
    };
    for (int mul = 0; mul <= 16; mul += 4)
        if ((st = consider(ReduceConfig{0, mul, 0})) != WXPY_OK) return st;
    if (!have) return fail(WXPY_EMISMATCH, "every configuration of reduction %d differed", kind);
    const int bmul = best.mul;
    if (kind == 0) {
        const int half = (bmul / 2) & ~1;
        for (int l = 1; l <= 3; ++l) {
            if ((st = consider(ReduceConfig{0, bmul, l})) != WXPY_OK) return st;
            if (half != bmul && (st = consider(ReduceConfig{0, half, l})) != WXPY_OK) return st;
        }
    }
    for (int v = 1; v <= 3; ++v)
        if ((st = consider(ReduceConfig{v, bmul, 0})) != WXPY_OK) return st;
    // the warp-tiled shapes at the best share; for norm2 then 2, 4 and 6
    // integer tree levels in the shape that did best among them
    double wbest_us = 0.0;
    int wbest = 4;
    for (int v = 4; v <= 6; ++v) {
        if ((st = consider(ReduceConfig{v, bmul, 0})) != WXPY_OK) return st;
        if (last_us > 0.0 && (wbest_us == 0.0 || last_us < wbest_us)) {
            wbest_us = last_us;
            wbest = v;
        }
    }
    if (kind == 0)
        for (int l = 2; l <= 6; l += 2)
            if ((st = consider(ReduceConfig{wbest, bmul, l})) != WXPY_OK) return st;
    double def_us = 0.0;
    if ((st = time_config(kind, n, reduce_default(kind), sc, &def_us)) != WXPY_OK) return st;
    reduce_tuned_store(kind, &best);
    if (res) {
        res->kind = kind;
        res->variant = best.variant;
        res->mul_sixteenths = best.mul;
        res->sum_levels = best.suml;
        res->candidates = candidates;
        res->rejected = rejected;
        res->best_us = best_us;
        res->default_us = def_us;
        res->gbs = (double)(kind == 1 ? 32 : 24) * (double)n / (best_us * 1e3);
    }
    return WXPY_OK;
}

int rtune_impl(int64_t n, wxpy_reduce_tune_result *results) {
    TraceRange trace("wxpy_reduce_tune");
    if (n <= 0) return fail(WXPY_EINVAL, "reduction tune needs n > 0");
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    RScratch sc;
    const size_t bytes = (size_t)n * 8;
    for (double **p : {&sc.x, &sc.y, &sc.z, &sc.w, &sc.ref_w})
        if ((st = ralloc((void **)p, bytes)) != WXPY_OK) return st;
    if ((st = ralloc((void **)&sc.res, 2 * sizeof(double))) != WXPY_OK) return st;
    sc.ws_bytes = wxpy_reduce_workspace_bytes(n);
    if ((st = ralloc(&sc.ws, (size_t)sc.ws_bytes)) != WXPY_OK) return st;
    sc.flush_bytes = std::max<int64_t>(2 * dp->l2_bytes, (int64_t)1 << 20);
    if ((st = ralloc(&sc.flush, (size_t)sc.flush_bytes)) != WXPY_OK) return st;
    if ((st = ralloc((void **)&sc.count, sizeof(unsigned long long))) != WXPY_OK) return st;
    cudaError_t e = cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.flush, 0, (size_t)sc.flush_bytes, sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "reduction tuner set-up");
    double *in[3] = {sc.x, sc.y, sc.z};
    for (int k = 0; k < 3; ++k)
        if ((st = launch_fill_uniform(in[k], n, 20130907ull + 70 + k, 1, 0, -1.0, 1.0, sc.s)) !=
            WXPY_OK)
            return st;
    for (int kind = 0; kind < 2; ++kind)
        if ((st = tune_kind(kind, n, sc, results ? &results[kind] : nullptr)) != WXPY_OK) return st;
    e = cudaStreamSynchronize(sc.s);
    return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "reduction tuner");
}

}  // namespace
}  // namespace wx

using namespace wx;

extern "C" {

int wxpy_reduce_tune(int64_t n, wxpy_reduce_tune_result *results) {
    std::lock_guard<std::mutex> lk(g_rtune_mu);
    return rtune_impl(n, results);
}

int wxpy_reduce_tuned_get(int kind, int *variant, int *mul_sixteenths, int *sum_levels) {
    if (kind < 0 || kind > 1 || !variant || !mul_sixteenths || !sum_levels)
        return fail(WXPY_EINVAL, "bad reduction kind %d", kind);
    ReduceConfig c{-1, -1, -1};
    reduce_tuned_load(kind, &c);
    *variant = c.variant;
    *mul_sixteenths = c.mul;
    *sum_levels = c.suml;
    return WXPY_OK;
}

int wxpy_reduce_tuned_set(int kind, int variant, int mul_sixteenths, int sum_levels) {
    if (kind < 0 || kind > 1) return fail(WXPY_EINVAL, "bad reduction kind %d", kind);
    if (variant == -1 && mul_sixteenths == -1 && sum_levels == -1) {
        reduce_tuned_store(kind, nullptr);
        return WXPY_OK;
    }
    const ReduceConfig c{variant, mul_sixteenths, sum_levels};
    if (!reduce_config_valid(kind, c))
        return fail(WXPY_EINVAL, "bad reduction configuration (%d, %d, %d)", variant,
                    mul_sixteenths, sum_levels);
    reduce_tuned_store(kind, &c);
    return WXPY_OK;
}

}  // extern "C"
