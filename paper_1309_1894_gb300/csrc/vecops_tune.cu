// vecops_tune.cu -- the empirical search of paper Sec. 2 applied to the pipe
// split of the sibling vector kernels (axpbypcz, maxpy groups, pointwise_mult).
//
// Sec. 2: variants are run to obtain their performance and their outputs, the
// outputs are compared with the reference results of the unchanged code, and
// the best-performing variant is kept.  Here a variant is a pipe split (how
// many products and sums run as the exactly rounded integer-pipeline
// operations instead of FP64 instructions); the reference results are those
// of the all-FP64 split on the same inputs; a split whose output differs by a
// single bit is rejected.  Candidates per class: the product share 0, 2, ..,
// 16 sixteenths with the sums in FP64, then the sums every other one or all
// in the integer pipeline at the best product share.  Timing: median of five
// runs of three back-to-back calls, each run after an L2 flush and a short
// device delay, with the in-place output restored from a pristine copy before
// every run.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.h"
#include "trace.h"

namespace wx {
namespace {

std::mutex g_vtune_mu;

constexpr int kMaxVecs = 9;  // inputs of the widest class (maxpy with 8 terms)
constexpr int kReps = 5;
constexpr double kCoef[8] = {0.75, -1.5, 1.25, -0.625, 1.875, -0.3125, 0.5625, -1.0625};

struct VScratch {
    double *v[kMaxVecs] = {};
    double *pristine = nullptr, *ref = nullptr, *w = nullptr;
    void *flush = nullptr;
    int64_t flush_bytes = 0;
    unsigned long long *count = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~VScratch() {
        if (s) cudaStreamSynchronize(s);
        for (double *p : v)
            if (p) cudaFree(p);
        for (void *p : {(void *)pristine, (void *)ref, (void *)w, flush, (void *)count})
            if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

int valloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(WXPY_ENOMEM, "vector tuner scratch allocation of %zu bytes failed", bytes);
    }
    return WXPY_OK;
}

// One class's operands: inputs, the output, and the vector restored before
// each run (the output when it is also an input).
struct ClassCall {
    int cls, nin;
    const double *in[kMaxVecs];
    double *out;
    double *restore;  // nullptr: out-of-place (pointwise_mult)
};

// The in-place output of a class (an input too): z of axpbypcz, y of axpby
// and of maxpy; pointwise_mult writes a separate vector.
double *inplace_out(int cls, VScratch &sc) {
    if (cls == WXPY_VEC_AXPBYPCZ) return sc.v[2];
    if (cls == WXPY_VEC_AXPBY) return sc.v[1];
    return sc.v[0];
}

ClassCall class_call(int cls, VScratch &sc) {
    ClassCall c{};
    c.cls = cls;
    c.nin = vecops_inputs(cls);
    for (int k = 0; k < c.nin; ++k) c.in[k] = sc.v[k];
    if (cls == WXPY_VEC_PMULT) {
        c.out = sc.w;
        c.restore = nullptr;
    } else {
        c.out = inplace_out(cls, sc);
        c.restore = c.out;
    }
    return c;
}

int restore(const ClassCall &c, int64_t n, VScratch &sc) {
    if (!c.restore) return WXPY_OK;
    cudaError_t e = cudaMemcpyAsync(c.restore, sc.pristine, (size_t)n * 8,
                                    cudaMemcpyDeviceToDevice, sc.s);
    return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "vector tuner restore");
}

// Median device time (us per call) of kReps timed runs, each kBatch back-to-
// back calls: the event timestamps advance in 2.048 us steps on GB300, about
// 3 % of one call at the search's size, and the operands of every class
// exceed the L2, so each call of a run reads them from memory.  The in-place
// output is restored before each run only (the coefficients keep a few
// repeated applications in range).
constexpr int kBatch = 3;

int time_split(const ClassCall &c, int64_t n, VecPipes p, VScratch &sc, double *median_us) {
    const int reps = tune_reps(kReps);
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) {
        int st;
        if ((st = restore(c, n, sc)) != WXPY_OK) return st;
        if ((st = launch_l2_flush(sc.flush, sc.flush_bytes, sc.count, sc.s)) != WXPY_OK) return st;
        launch_device_delay(20000 * kBatch, sc.s);
        cudaEventRecord(sc.e0, sc.s);
        for (int b = 0; b < kBatch; ++b)
            if ((st = vecops_run(c.cls, n, kCoef, c.in, c.out, p, sc.s)) != WXPY_OK) return st;
        cudaEventRecord(sc.e1, sc.s);
        cudaError_t e = cudaEventSynchronize(sc.e1);
        if (e != cudaSuccess) return fail_cuda(e, "vector tuner timing");
        cudaEventElapsedTime(&ms[r], sc.e0, sc.e1);
    }
    std::sort(ms.begin(), ms.end());
    *median_us = 1e3 * (double)ms[reps / 2] / kBatch;
    return WXPY_OK;
}

// Runs split p once from pristine inputs; *bad = bits differing from sc.ref
// (the reference run passes ref = nullptr and copies its output there).
int run_checked(const ClassCall &c, int64_t n, VecPipes p, VScratch &sc, bool reference,
                unsigned long long *bad) {
    int st;
    if ((st = restore(c, n, sc)) != WXPY_OK) return st;
    if ((st = vecops_run(c.cls, n, kCoef, c.in, c.out, p, sc.s)) != WXPY_OK) return st;
    cudaError_t e;
    if (reference) {
        e = cudaMemcpyAsync(sc.ref, c.out, (size_t)n * 8, cudaMemcpyDeviceToDevice, sc.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
        if (e != cudaSuccess) return fail_cuda(e, "vector tuner reference");
        *bad = 0;
        return WXPY_OK;
    }
    e = cudaMemsetAsync(sc.count, 0, sizeof(unsigned long long), sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "vector tuner verify");
    if ((st = launch_count_mismatch(c.out, sc.ref, n, sc.count, sc.s)) != WXPY_OK) return st;
    e = cudaMemcpyAsync(bad, sc.count, sizeof *bad, cudaMemcpyDeviceToHost, sc.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sc.s);
    return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "vector tuner verify");
}

int64_t class_bytes(int cls, int64_t n) {
    const int nin = vecops_inputs(cls);
    return (int64_t)(nin + 1) * 8 * n;  // every input read once, the output written
}

int tune_class(int cls, int64_t n, VScratch &sc, wxpy_vecops_tune_result *res) {
    const ClassCall c = class_call(cls, sc);
    int st;
    unsigned long long bad = 0;
    if ((st = run_checked(c, n, VecPipes{0, 0}, sc, true, &bad)) != WXPY_OK) return st;
    std::vector<VecPipes> cands;
    for (int mul = 0; mul <= 16; mul += 2) cands.push_back({0, mul});
    int candidates = 0, rejected = 0;
    VecPipes best{0, 0};
    double best_us = 0.0;
    bool have = false;
    auto consider = [&](VecPipes p) -> int {
        ++candidates;
        unsigned long long mism = 0;
        int s2 = run_checked(c, n, p, sc, false, &mism);
        if (s2 != WXPY_OK) return s2;
        if (mism) {
            ++rejected;
            return WXPY_OK;
        }
        double us = 0.0;
        if ((s2 = time_split(c, n, p, sc, &us)) != WXPY_OK) return s2;
        if (!have || us < best_us) {
            best = p;
            best_us = us;
            have = true;
        }
        return WXPY_OK;
    };
    for (const VecPipes &p : cands)
        if ((st = consider(p)) != WXPY_OK) return st;
    if (cls != WXPY_VEC_PMULT && have) {  // pointwise_mult has no sums
        const int mul = best.mul;
        for (int add = 1; add <= 2; ++add)
            if ((st = consider(VecPipes{add, mul})) != WXPY_OK) return st;
    }
    if (!have) return fail(WXPY_EMISMATCH, "every split of vector class %d differed", cls);
    double def_us = 0.0;
    if ((st = time_split(c, n, vecops_default(cls), sc, &def_us)) != WXPY_OK) return st;
    vecops_tuned_store(cls, &best);
    if (res) {
        res->op_class = cls;
        res->add_offload = best.add;
        res->mul_sixteenths = best.mul;
        res->candidates = candidates;
        res->rejected = rejected;
        res->reserved = 0;
        res->best_us = best_us;
        res->default_us = def_us;
        res->gbs = (double)class_bytes(cls, n) / (best_us * 1e3);
    }
    return WXPY_OK;
}

int vtune_impl(int64_t n, wxpy_vecops_tune_result *results) {
    TraceRange trace("wxpy_vecops_tune");
    if (n <= 0) return fail(WXPY_EINVAL, "vector tune needs n > 0");
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    VScratch sc;
    const size_t bytes = (size_t)n * 8;
    for (double *&p : sc.v)
        if ((st = valloc((void **)&p, bytes)) != WXPY_OK) return st;
    if ((st = valloc((void **)&sc.pristine, bytes)) != WXPY_OK) return st;
    if ((st = valloc((void **)&sc.ref, bytes)) != WXPY_OK) return st;
    if ((st = valloc((void **)&sc.w, bytes)) != WXPY_OK) return st;
    sc.flush_bytes = std::max<int64_t>(2 * dp->l2_bytes, (int64_t)1 << 20);
    if ((st = valloc(&sc.flush, (size_t)sc.flush_bytes)) != WXPY_OK) return st;
    if ((st = valloc((void **)&sc.count, sizeof(unsigned long long))) != WXPY_OK) return st;
    cudaError_t e = cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.flush, 0, (size_t)sc.flush_bytes, sc.s);
    if (e != cudaSuccess) return fail_cuda(e, "vector tuner set-up");
    for (int k = 0; k < kMaxVecs; ++k)
        if ((st = launch_fill_uniform(sc.v[k], n, 20130907ull + 50 + k, 1, 0, -1.0, 1.0, sc.s)) !=
            WXPY_OK)
            return st;
    for (int cls = 0; cls < WXPY_VEC_CLASSES; ++cls) {
        // pristine copy of the in-place output of this class
        double *out = inplace_out(cls, sc);
        e = cudaMemcpyAsync(sc.pristine, out, bytes, cudaMemcpyDeviceToDevice, sc.s);
        if (e != cudaSuccess) return fail_cuda(e, "vector tuner copy");
        if ((st = tune_class(cls, n, sc, results ? &results[cls] : nullptr)) != WXPY_OK) return st;
        // leave the inputs as generated for the next class
        if ((st = restore(class_call(cls, sc), n, sc)) != WXPY_OK) return st;
    }
    e = cudaStreamSynchronize(sc.s);
    return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "vector tuner");
}

}  // namespace
}  // namespace wx

using namespace wx;

extern "C" {

int wxpy_vecops_tune(int64_t n, wxpy_vecops_tune_result *results) {
    std::lock_guard<std::mutex> lk(g_vtune_mu);
    return vtune_impl(n, results);
}

int wxpy_vecops_tuned_get(int op_class, int *add_offload, int *mul_sixteenths) {
    if (op_class < 0 || op_class >= WXPY_VEC_CLASSES || !add_offload || !mul_sixteenths)
        return fail(WXPY_EINVAL, "bad vector class %d", op_class);
    VecPipes p{-1, -1};
    vecops_tuned_load(op_class, &p);
    *add_offload = p.add;
    *mul_sixteenths = p.mul;
    return WXPY_OK;
}

int wxpy_vecops_tuned_set(int op_class, int add_offload, int mul_sixteenths) {
    if (op_class < 0 || op_class >= WXPY_VEC_CLASSES)
        return fail(WXPY_EINVAL, "bad vector class %d", op_class);
    if (add_offload == -1 && mul_sixteenths == -1) {
        vecops_tuned_store(op_class, nullptr);
        return WXPY_OK;
    }
    if (add_offload < 0 || add_offload > 2 || mul_sixteenths < 0 || mul_sixteenths > 16 ||
        (op_class == WXPY_VEC_PMULT && add_offload != 0))
        return fail(WXPY_EINVAL, "bad split (%d, %d)", add_offload, mul_sixteenths);
    const VecPipes p{add_offload, mul_sixteenths};
    vecops_tuned_store(op_class, &p);
    return WXPY_OK;
}

}  // extern "C"
