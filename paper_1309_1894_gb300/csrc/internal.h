// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "wxpy.h"
#include "single_kernel.cuh"

namespace wx {

// ---- errors (thread-local detail, see wxpy_last_error_message) ----
int fail(int status, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail_cuda(cudaError_t e, const char *what);
void clear_error();

// ---- device properties, cached per ordinal ----
struct DeviceProps {
    int device = -1;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    int64_t l2_bytes = 0;
    int64_t global_bytes = 0;
    char name[128] = {0};
};
// Properties of the current device; nullptr (and the error recorded) on failure.
const DeviceProps *current_device(int *status);

// ---- the variant space ----
struct Variant {
    int vec_bytes, unroll, threads, blocks_per_sm, cache, carveout, streams;
    int offload = 0;  // integer pipeline: 0 nothing, 1 half the sums, 2 all sums, 3 all products
};
constexpr int kVecBytes[3] = {8, 16, 32};
constexpr int kUnroll[4] = {1, 2, 4, 8};
constexpr int kThreads[4] = {128, 256, 512, 1024};
constexpr int kBlocksPerSm[5] = {0, 1, 2, 4, 8};
constexpr int kCache[3] = {0, 1, 2};
constexpr int kCarveout[4] = {-1, 0, 50, 100};
constexpr int kStreams[4] = {1, 2, 4, 8};
constexpr int kOffload[4] = {0, 1, 2, 3};
constexpr int kVariantsPerOffload = 3 * 4 * 4 * 5 * 3 * 4 * 4;
constexpr int kVariantCount = kVariantsPerOffload * 4;

bool decode_variant(int id, Variant *v);
int encode_variant(const Variant &v);  // -1 if a field is out of the space
void to_info(const Variant &v, int id, wxpy_variant_info *out);

// ---- classification ----
struct CallClass {
    int alias;      // WXPY_ALIAS_* bits
    int align;      // 32, 16, 8
    int head;       // for `align`
    int bucket;     // floor(log2 n) or -1
    int tune_key;   // -1 when n == 0
};
int classify(int64_t n, const double *x, const double *y, const double *w, CallClass *c);
constexpr int kBuckets = 64;
constexpr int kTuneKeys = kBuckets * 3 * 4;
int tune_key_of(int bucket, int align, int alias);

// The variant after adjustment to a call class (width cap, cache under aliasing).
Variant adjust_variant(const Variant &v, const CallClass &c);
// Built-in default when nothing is tuned or forced.
Variant default_variant(const CallClass &c, int64_t n);

// Tuning table (flat variant ids, -1 = none) and the forced id.
extern std::atomic<int> g_forced_variant;
extern std::atomic<int> g_tuned[kTuneKeys];
// 1 where the search found the cell launch-bound (its choice fixed, not a pick among ties).
extern std::atomic<int> g_tuned_launch_bound[kTuneKeys];

// ---- launching ----
// Runs the (already adjusted) variant on stream s.  Handles the stream split.
int run_variant(const Variant &v, const CallClass &c, int64_t n, double alpha,
                const double *x, const double *y, double *w, cudaStream_t s);
// Launch gate for fault injection: returns cudaSuccess or the injected error.
cudaError_t injected_launch_error();

// ---- batched launch (batch.cu) ----
// One work item of the segmented launch.
struct TileRec {
    int64_t begin;    // first element of the tile within its segment
    int32_t seg;      // segment index in the descriptor table
    uint32_t len_ul;  // bits 0..29: elements in the tile; bits 30..31: log2 unroll
};
constexpr uint32_t kLenMask = (1u << 30) - 1;
constexpr int64_t kMaxTileElems = (1 << 30) - 32;
struct BatchShape {
    int threads;                   // block size of the persistent kernel
    int blocks_per_sm;             // grid = blocks_per_sm * sm_count (capped by tiles)
    int offload;                   // integer pipelines: 0 none, 1 half the sums, 3 every product
    int32_t tile_elems[kBuckets];  // per size bucket of a segment; 0 = whole segment
    int8_t unroll_log2[kBuckets];  // per size bucket: log2 of the unroll
};
BatchShape default_batch_shape();
BatchShape current_batch_shape();
void set_batch_shape(const BatchShape &s);
int validate_table(const wxpy_desc *t, int64_t count);
// Tile list of a validated table (largest first); returns the element total.
int64_t build_tiles(const wxpy_desc *t, int64_t count, const BatchShape &shape,
                    std::vector<TileRec> *out);
// One launch of the segmented kernel over `ntiles` device tile records.
cudaError_t launch_segmented(const wxpy_desc *dev_table, const TileRec *tiles, int64_t ntiles,
                             unsigned *status, const BatchShape &shape, int sm_count,
                             cudaStream_t s);

// api.cu: NVTX ranges on (WXPY_NVTX=1), read once; see trace.h.
bool trace_enabled();

// tune.cu: loads $WXPY_TUNE_CACHE once per process (errors ignored).
void autoload_tune_cache();

// gen.cu: seeded device inputs, bitwise comparison, L2 eviction.
uint64_t stream_key(uint64_t seed, uint32_t tag);
int launch_fill_uniform(double *dst, int64_t n, uint64_t seed, uint32_t tag, int64_t start,
                        double lo, double hi, cudaStream_t s);
int launch_count_mismatch(const double *a, const double *b, int64_t n,
                          unsigned long long *count_dev, cudaStream_t s);
int launch_l2_flush(const void *buf, int64_t bytes, void *sink, cudaStream_t s);
// Timed runs per candidate of a search: WXPY_TUNE_REPS (1..101) when set,
// else `fallback` (tune.cu).
int tune_reps(int fallback);
// A one-thread kernel that spins for `cycles` SM clocks: queued ahead of a
// timed region so that the host's launch latency is not timed.
void launch_device_delay(long long cycles, cudaStream_t s);

// vecops.cu: the sibling kernels by class (WXPY_VEC_*), under an explicit
// pipe split, and the table of searched splits.
struct VecPipes {
    int add, mul;  // add offload 0..2, product sixteenths 0..16
};
// Classes: axpbypcz in = {x, y, z}, out = z; maxpy with m = class + 1 terms
// in = {y, x0 .. x_{m-1}}, out = y; pointwise_mult in = {x, y}, out separate.
int vecops_inputs(int cls);
int vecops_run(int cls, int64_t n, const double *coef, const double *const *in, double *out,
               VecPipes p, cudaStream_t s);
VecPipes vecops_default(int cls);
bool vecops_tuned_load(int cls, VecPipes *p);
void vecops_tuned_store(int cls, const VecPipes *p);  // nullptr clears

// reduce.cu: the fused reductions (kind 0 norm2, 1 dot) under an explicit
// configuration, and the table of searched configurations.
struct ReduceConfig {
    int variant;  // 0 register-loaded, 1..3 staged shapes
    int mul;      // product sixteenths 0..16
    int suml;     // norm2: in-thread tree levels summed in the integer pipelines, 0..3
};
ReduceConfig reduce_default(int kind);
bool reduce_config_valid(int kind, ReduceConfig c);
int reduce_run(int kind, int64_t n, double alpha, const double *x, const double *y, double *w,
               const double *z, double *result, void *workspace, int64_t ws_bytes, ReduceConfig c,
               cudaStream_t s);
bool reduce_tuned_load(int kind, ReduceConfig *c);
void reduce_tuned_store(int kind, const ReduceConfig *c);  // nullptr clears

cudaError_t launch_reference(unsigned grid, unsigned tpb, const SingleArgs &a, cudaStream_t s);
SingleEntry single_entry(int vw, int offload, int u_idx, int gs, int cache, int xy);
// The mixed-alignment instance (mixed_kernel.cuh) for input load widths kx, ky.
SingleEntry mixed_entry(int kx, int ky, int u_idx, int cache, int xy, int offload);

}  // namespace wx
