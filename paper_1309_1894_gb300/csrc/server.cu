// server.cu -- a continuous-batching request server for VecWXPY.
//
// Clients submit requests: (n, alpha, seed), whose inputs the server generates
// on the device, or (n, alpha, x, y) with the caller's own data in device or
// host memory.  A scheduler thread
//   1. admits queued requests in arrival order while the device-memory budget
//      (one arena, first fit, 256-byte blocks holding x, y, w) and the slot
//      limit allow.  Strict order (admission = 0): a request that does not
//      fit waits, and nothing passes it.  Backfill (admission = A > 0 us):
//      while the head does not fit, later requests that do are admitted ahead
//      of it, for at most A us of the head's wait -- then the head holds the
//      line until memory frees, so it cannot starve;
//   2. coalesces every admitted, not yet launched request (up to max_batch)
//      into one batch and runs it on the next free stream in two steps:
//      (a) the inputs are put into the requests' resident buffers -- one
//      segmented fill launch generates x and y of every seeded request, and
//      the caller-data requests are copied in;
//      (b) one launch of the batched segmented kernel (wxpy_seg_kernel, the
//      same kernel and tile body as wxpy_batch) reads x and y from those
//      buffers and writes w -- 24 bytes per element, one launch per batch
//      whatever the number of requests in it;
//   3. polls the batches' completion events, stamps each request's completion
//      time, and frees the buffers of requests marked auto-release.
// Requests that arrive while batches run on other streams are admitted and
// launched as soon as memory and a stream free up, so their work overlaps on
// the device (continuous batching, not a queue drained batch by batch).  The
// serial mode is the baseline over the identical data path: per request the
// same inputs step (fill x and fill y, or the copies) and one wxpy() call,
// with no coalescing.  The fused mode is a separate option for seeded
// requests only: one kernel per batch generates x and y in registers and
// writes x, y and w without reading anything back.
//
// Each request's result is element-wise w = RN(RN(alpha*x) + y) on its own
// inputs (paper Sec. 3, Fig. 1 vecwxpy), so it is the same bits alone and in
// any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fp64_mul.cuh"
#include "gen.cuh"
#include "internal.h"
#include "trace.h"

namespace wx {
namespace {

using Clock = std::chrono::steady_clock;

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

constexpr int64_t kBlock = 256;  // arena granularity (bytes)

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, size) with coalescing of freed blocks.
class Arena {
  public:
    void init(int64_t size) {
        free_.clear();
        size_ = size / kBlock * kBlock;
        if (size_ > 0) free_[0] = size_;
        used_ = 0;
    }
    int64_t alloc(int64_t bytes) {
        bytes = round_up(bytes, kBlock);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const int64_t off = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[off + bytes] = rem;
            used_ += bytes;
            return off;
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = round_up(bytes, kBlock);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    int64_t used() const { return used_; }
    int64_t size() const { return size_; }

  private:
    std::map<int64_t, int64_t> free_;
    int64_t size_ = 0, used_ = 0;
};

enum ReqState { kQueued = 0, kAdmitted = 1, kRunning = 2, kDone = 3, kFailed = 4 };

// Request error for a batch whose tile bounds check fired (not a CUDA error code).
constexpr int kTileCheckFailed = -1;

struct Request {
    int64_t n = 0;
    double alpha = 0;
    uint64_t seed = 0;
    // Caller data: source pointers and kind (WXPY_SERVE_DATA_*), or -1 for a
    // seeded request whose inputs the server generates.
    int src_kind = -1;
    const double *src_x = nullptr, *src_y = nullptr;
    int state = kQueued;
    bool auto_release = false;
    int64_t off = -1, bytes = 0;
    double *x = nullptr, *y = nullptr, *w = nullptr;
    Clock::time_point t_submit, t_done;
    int error = 0;
};

// Per request of a batch: where its tiles start in the batch's tile numbering,
// its tile length and unroll.  The host writes only this (24 bytes per
// request); warps find their request by binary search over first_tile, so no
// per-tile list is built on the host however many tiles a batch has.
struct ServePlan {
    int64_t first_tile;  // exclusive prefix of tile counts over the batch
    int64_t tile_len;    // elements per tile
    int32_t ulog;        // log2 of the unroll
    int32_t pad;
};

// A batch in flight on one stream.  Its tables live in one staging region,
// pinned on the host and mirrored on the device, so that a batch's tables go
// up in ONE copy: [status word | descriptors | seeds | fill plan | tiles of
// the segmented kernel], each part 256-byte aligned.  The status word is
// uploaded as zero with the tables and comes back, after the kernels, into a
// separate pinned word.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::chrono::steady_clock::time_point t_launch;  // when the batch was queued
    double host_s = 0;                               // host time queueing it
    int64_t count = 0, elems = 0;                    // its requests and elements
    std::vector<uint64_t> tickets;
    int64_t cap_segs = 0, cap_tiles = 0;
    char *h_stage = nullptr, *d_stage = nullptr;
    size_t off_table = 0, off_seeds = 0, off_plan = 0, off_tiles = 0, stage_bytes = 0;
    unsigned *h_status = nullptr;  // the status word of the last batch, copied back
    template <class T>
    T *host(size_t off) const { return (T *)(h_stage + off); }
    template <class T>
    T *dev(size_t off) const { return (T *)(d_stage + off); }
};

// Elements per tile of the fill launch (one warp per tile), for batches large
// enough to fill the GPU with such tiles.
constexpr int64_t kFillTile = 8192;

// Largest s in [lo, count) with plan[s].first_tile <= t (tiles only grow
// along a warp's sequence, so the previous answer is a valid lower bound).
__device__ __forceinline__ int64_t find_request(const ServePlan *plan, int64_t count, int64_t t,
                                                int64_t lo) {
    int64_t hi = count - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (plan[mid].first_tile <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One pass per batch: for every element of every request, generate x and y
// from the request's seed, compute w = RN(RN(alpha*x) + y), and store all
// three (the request's result is x, y and w).  A warp takes a tile; a lane
// takes four consecutive elements and writes them as 32-byte vectors (tiles
// start at multiples of their length, a multiple of 4, in 256-byte-aligned
// buffers), the ragged end of a tile element by element.  Generating in
// registers saves writing x and y and reading them back (40 bytes per
// element in two passes become 24 in one).  PM: the products alpha*x run in
// the integer pipelines at no (0), odd (1) or every (2) position of a vector,
// fixed at compile time; the sums stay in FP64.
__device__ __forceinline__ uint64_t bits_of_d(double v) { return (uint64_t)__double_as_longlong(v); }

template <int PM>
__device__ __forceinline__ double serve_elem(double alpha, const MulCoef &ca, double x, double y,
                                             int q) {
    double p;
    if (PM == 2 || (PM == 1 && (q & 1))) {
        bool slow = false;
        uint64_t pb = mul_rn_core(ca, bits_of_d(x), slow);
        if (slow) pb = mul_rn_hw_bits(bits_of_d(alpha), bits_of_d(x));
        p = __longlong_as_double((long long)pb);
    } else {
        p = __dmul_rn(alpha, x);
    }
    return __dadd_rn(p, y);
}

__device__ __forceinline__ void st4_cs(double *p, double a, double b, double c, double d) {
    asm volatile("st.global.cs.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(a), "d"(b), "d"(c),
                 "d"(d)
                 : "memory");
}

template <int PM>
__global__ void __launch_bounds__(256) serve_fused_kernel(const wxpy_desc *table,
                                                          const uint64_t *seeds,
                                                          const ServePlan *plan, int64_t count,
                                                          int64_t ntiles) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t s = 0;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        s = find_request(plan, count, t, s);
        const wxpy_desc d = table[s];
        const ServePlan sp = plan[s];
        const int64_t begin = (t - sp.first_tile) * sp.tile_len;
        const int64_t end = min(d.n, begin + sp.tile_len);
        const uint64_t kx = stream_key_of(seeds[s], 1), ky = stream_key_of(seeds[s], 2);
        const MulCoef ca = mul_coef_of(bits_of_d(d.alpha));
        double *x = const_cast<double *>(d.x), *y = const_cast<double *>(d.y), *w = d.w;
        const int64_t nvec = (end - begin) >> 2;
        for (int64_t c = lane; c < nvec; c += 32) {
            const int64_t i0 = begin + 4 * c;
            double xv[4], yv[4], wv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xv[q] = uniform_pm1(kx, i0 + q);
                yv[q] = uniform_pm1(ky, i0 + q);
                wv[q] = serve_elem<PM>(d.alpha, ca, xv[q], yv[q], q);
            }
            st4_cs(x + i0, xv[0], xv[1], xv[2], xv[3]);
            st4_cs(y + i0, yv[0], yv[1], yv[2], yv[3]);
            st4_cs(w + i0, wv[0], wv[1], wv[2], wv[3]);
        }
        for (int64_t i = begin + 4 * nvec + lane; i < end; i += 32) {
            const double xi = uniform_pm1(kx, i), yi = uniform_pm1(ky, i);
            x[i] = xi;
            y[i] = yi;
            w[i] = serve_elem<0>(d.alpha, ca, xi, yi, 0);
        }
    }
}

// The inputs step of a batch: for every seeded request, x and y from the
// request's seed (streams (seed, 1) and (seed, 2), the values
// wxpy_fill_uniform writes) stored into its resident buffers.  A warp takes a
// tile of the plan's length (kFillTile, or shorter for a small batch: a
// multiple of 256); a lane writes four consecutive elements as 32-byte
// vectors (tiles start at multiples of that length in 256-byte-aligned
// buffers), the ragged end of a tile element by element.  Requests with
// caller data have no tiles in the plan.  Reads nothing; 16 bytes written per
// element.
__global__ void __launch_bounds__(256) serve_fill_kernel(const wxpy_desc *table,
                                                         const uint64_t *seeds,
                                                         const ServePlan *plan, int64_t count,
                                                         int64_t ntiles) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t s = 0;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        s = find_request(plan, count, t, s);
        const wxpy_desc d = table[s];
        const ServePlan sp = plan[s];
        const int64_t begin = (t - sp.first_tile) * sp.tile_len;
        const int64_t end = min(d.n, begin + sp.tile_len);
        const uint64_t kx = stream_key_of(seeds[s], 1), ky = stream_key_of(seeds[s], 2);
        double *x = const_cast<double *>(d.x), *y = const_cast<double *>(d.y);
        const int64_t nvec = (end - begin) >> 2;
        for (int64_t c = lane; c < nvec; c += 32) {
            const int64_t i0 = begin + 4 * c;
            double xv[4], yv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xv[q] = uniform_pm1(kx, i0 + q);
                yv[q] = uniform_pm1(ky, i0 + q);
            }
            st4_cs(x + i0, xv[0], xv[1], xv[2], xv[3]);
            st4_cs(y + i0, yv[0], yv[1], yv[2], yv[3]);
        }
        for (int64_t i = begin + 4 * nvec + lane; i < end; i += 32) {
            x[i] = uniform_pm1(kx, i);
            y[i] = uniform_pm1(ky, i);
        }
    }
}

// Tile length cap for a batch of `elems` elements: small batches are cut into
// shorter tiles (down to 256 elements), so that their warps still spread over
// every SM -- with the batched shape's 8192-element tiles, a lone request of
// 65k elements would run on one block.  Batches of kTargetTiles x 8192
// elements and more keep the shape's tiles.
constexpr int64_t kTargetTiles = 4864;  // 152 SMs x 4 blocks x 8 warps
int64_t tile_cap(int64_t elems) {
    int64_t t = 8192;
    while (t > 256 && elems / t < kTargetTiles) t >>= 1;
    return t;
}

// Tile list of a batch for the segmented kernel: each request cut into tiles
// of its size bucket's length (the batch shape, as in wxpy_batch; at most
// t_cap elements), ordered
// longest first by power-of-two class of the tile length -- a stable counting
// sort, linear in the tiles, so that the static round-robin over warps ends
// on short tiles.  Returns the tile count; writes the tiles only when they
// fit in `cap`.
int64_t serve_tiles(const wxpy_desc *t, int64_t count, const BatchShape &shape, int64_t t_cap,
                     TileRec *out, int64_t cap) {
    int64_t per_class[64] = {0};
    auto tile_len = [&](int64_t n) {
        const int b = 63 - __builtin_clzll((unsigned long long)n);
        const int64_t T = shape.tile_elems[b] > 0 ? shape.tile_elems[b] : n;
        return std::min<int64_t>(std::min<int64_t>(T, t_cap), kMaxTileElems);
    };
    auto cls = [](int64_t len) { return 63 - __builtin_clzll((unsigned long long)len); };
    int64_t total = 0;
    for (int64_t s = 0; s < count; ++s) {
        const int64_t n = t[s].n, T = tile_len(n);
        per_class[cls(T)] += n / T;
        if (n % T) per_class[cls(n % T)] += 1;
        total += (n + T - 1) / T;
    }
    if (total > cap) return total;
    int64_t start[64];
    int64_t pos = 0;
    for (int c = 63; c >= 0; --c) {
        start[c] = pos;
        pos += per_class[c];
    }
    for (int64_t s = 0; s < count; ++s) {
        const int64_t n = t[s].n, T = tile_len(n);
        const int b = 63 - __builtin_clzll((unsigned long long)n);
        const uint32_t ul =
            (uint32_t)std::min<int>(2, std::max<int>(0, shape.unroll_log2[b])) << 30;
        for (int64_t b0 = 0; b0 < n; b0 += T) {
            const int64_t len = std::min<int64_t>(T, n - b0);
            out[start[cls(len)]++] = TileRec{b0, (int32_t)s, (uint32_t)len | ul};
        }
    }
    return total;
}

// Saturated Poisson load on GB300 (n log-uniform in [2^8, 2^24]): 2.09e11
// elements/s with every product in FP64, 1.82e11 with half, 1.59e11 with all
// in the integer pipelines -- the generator keeps the ALU pipe busy and
// leaves FP64 free.
constexpr int kServePM = 0;

}  // namespace
}  // namespace wx

using namespace wx;

struct wxpy_server {
    wxpy_server_config cfg{};
    int device = 0;
    int sm_count = 0;
    char *arena_base = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    int next_slot = 0;

    std::mutex mu;
    std::condition_variable cv_submit;  // wakes the scheduler
    std::condition_variable cv_done;    // wakes waiters
    std::deque<uint64_t> queue;
    std::vector<uint64_t> admitted;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    int64_t resident = 0;

    // statistics since the last reset
    Clock::time_point t_reset;
    int64_t submitted = 0, rejected = 0, completed = 0, failed = 0, max_queue = 0;
    int64_t batches = 0, launches = 0, elements_done = 0, requests_launched = 0;
    int64_t max_inflight = 0;  // most batches on the device at once
    double max_launch_host = 0, max_batch = 0;  // seconds, see wxpy_server_stats
    int64_t backfilled = 0;
    double head_wait_frag = 0, head_wait_full = 0;  // seconds
    std::vector<double> latencies;

    // the queue head's wait: since when, and the last time it was accounted
    uint64_t waiting_head = 0;
    Clock::time_point head_since, head_accounted;

    std::thread sched;
    std::atomic<bool> stop{false};
    int sched_error = 0;
};

namespace wx {
namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

void free_stage(Slot &s) {
    if (s.d_stage) cudaFree(s.d_stage);
    if (s.h_stage) cudaFreeHost(s.h_stage);
    s.d_stage = s.h_stage = nullptr;
    s.stage_bytes = 0;
    s.cap_tiles = 0;
}

// (Re)allocates the slot's staging region for `segs` requests and `tiles`
// tile records; the slot must be idle.
cudaError_t alloc_stage(Slot &s, int64_t segs, int64_t tiles) {
    free_stage(s);
    s.off_table = 256;
    s.off_seeds = s.off_table + align256(sizeof(wxpy_desc) * segs);
    s.off_plan = s.off_seeds + align256(sizeof(uint64_t) * segs);
    s.off_tiles = s.off_plan + align256(sizeof(ServePlan) * segs);
    const size_t bytes = s.off_tiles + sizeof(TileRec) * (size_t)tiles;
    cudaError_t e = cudaMalloc(&s.d_stage, bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_stage, bytes);
    if (e != cudaSuccess) {
        free_stage(s);
        return e;
    }
    s.stage_bytes = bytes;
    s.cap_segs = segs;
    s.cap_tiles = tiles;
    return cudaSuccess;
}

void free_slot(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    free_stage(s);
    if (s.h_status) cudaFreeHost(s.h_status);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot{};
}

// `tiles`: initial capacity of the tile list (it grows when a batch needs more).
cudaError_t init_slot(Slot &s, int64_t segs, int64_t tiles) {
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_status, sizeof(unsigned));
    if (e == cudaSuccess) {
        *s.h_status = 0;
        e = alloc_stage(s, segs, std::max<int64_t>(tiles, 4096));
    }
    return e;
}

// Marks the requests of a finished (or failed) slot; caller holds the lock.
// WXPY_SERVE_SLOW_MS=<ms>: a diagnostic; every batch whose host queueing or
// queue-to-completion time exceeds that many milliseconds is reported on
// stderr with its size.  Read once.
double slow_batch_threshold_s() {
    static const double v = [] {
        const char *e = std::getenv("WXPY_SERVE_SLOW_MS");
        return e && *e ? std::atof(e) * 1e-3 : -1.0;
    }();
    return v;
}

void retire_slot(wxpy_server *sv, Slot &s, Clock::time_point now, int error) {
    const double batch_s = seconds(now - s.t_launch);
    sv->max_batch = std::max(sv->max_batch, batch_s);
    const double slow = slow_batch_threshold_s();
    if (slow > 0 && (batch_s > slow || s.host_s > slow))
        std::fprintf(stderr, "wxpy server: slow batch on stream %p: %lld requests, %lld elements, "
                     "host %.3f ms, queue to completion %.3f ms\n", (void *)s.stream,
                     (long long)s.count, (long long)s.elems, s.host_s * 1e3, batch_s * 1e3);
    // A set status word means the segmented kernel skipped a tile that did not
    // fit its descriptor: the batch's results are incomplete.
    if (!error && s.h_status && *s.h_status) error = kTileCheckFailed;
    if (s.h_status) *s.h_status = 0;
    for (uint64_t t : s.tickets) {
        auto it = sv->reqs.find(t);
        if (it == sv->reqs.end()) continue;
        Request &r = it->second;
        r.t_done = now;
        if (error) {
            r.state = kFailed;
            r.error = error;
            ++sv->failed;
        } else {
            r.state = kDone;
            ++sv->completed;
            sv->elements_done += r.n;
            sv->latencies.push_back(seconds(now - r.t_submit));
        }
        if (r.auto_release) {
            if (r.off >= 0) sv->arena.release(r.off, r.bytes);
            --sv->resident;
            sv->reqs.erase(it);
        }
    }
    s.tickets.clear();
    s.busy = false;
    sv->cv_done.notify_all();
}

// Copies a caller-data request's x and y into its resident buffers on `st`.
cudaError_t copy_in(const Request *r, cudaStream_t st) {
    const cudaMemcpyKind k =
        r->src_kind == WXPY_SERVE_DATA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t bytes = (size_t)r->n * 8;
    cudaError_t e = cudaMemcpyAsync(r->x, r->src_x, bytes, k, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->y, r->src_y, bytes, k, st);
    return e;
}

// Launches the requests in `batch` on slot s.  Caller does NOT hold the lock;
// the requests are already marked running.  Returns a cudaError_t.
cudaError_t launch_batch(wxpy_server *sv, Slot &s, const std::vector<Request *> &batch) {
    TraceRange trace("wxpy_server_batch");
    cudaError_t e = cudaSuccess;
    if (sv->cfg.mode == WXPY_SERVE_SERIAL) {
        // Baseline: the same requests over the same data path, call by call:
        // the inputs step (fill x, fill y -- or the copies) and one wxpy() per
        // request, nothing coalesced.
        for (Request *r : batch) {
            int st = WXPY_OK;
            if (r->src_kind < 0) {
                st = launch_fill_uniform(r->x, r->n, r->seed, 1, 0, -1.0, 1.0, s.stream);
                if (st == WXPY_OK)
                    st = launch_fill_uniform(r->y, r->n, r->seed, 2, 0, -1.0, 1.0, s.stream);
                if (st == WXPY_OK) sv->launches += 2;
            } else if ((e = copy_in(r, s.stream)) != cudaSuccess) {
                return e;
            }
            if (st == WXPY_OK) st = wxpy(r->n, r->alpha, r->x, r->y, r->w, s.stream);
            if (st != WXPY_OK) return (cudaError_t)(wxpy_last_cuda_error() ? wxpy_last_cuda_error() : 1);
            sv->launches += 1;
        }
        return cudaEventRecord(s.done, s.stream);
    }
    const bool fused = sv->cfg.mode == WXPY_SERVE_FUSED;
    const int64_t count = (int64_t)batch.size();
    const BatchShape shape = current_batch_shape();
    // Descriptors, and the plan of the generated inputs: the fill's tiles in
    // the batched mode, the fused kernel's (per-bucket tile length) in the
    // fused mode; caller-data requests get none.
    wxpy_desc *h_table = s.host<wxpy_desc>(s.off_table);
    uint64_t *h_seeds = s.host<uint64_t>(s.off_seeds);
    ServePlan *h_plan = s.host<ServePlan>(s.off_plan);
    int64_t nplan = 0, elems = 0, seeded = 0;
    for (const Request *r : batch) {
        elems += r->n;
        if (r->src_kind < 0) seeded += r->n;
    }
    const int64_t fill_tile = std::min<int64_t>(kFillTile, tile_cap(seeded));
    for (int64_t i = 0; i < count; ++i) {
        const Request *r = batch[i];
        h_table[i] = wxpy_desc{r->n, r->alpha, r->x, r->y, r->w};
        h_seeds[i] = r->seed;
        int64_t T = fill_tile;
        int ulog = 0;
        if (fused) {
            const int b = 63 - __builtin_clzll((unsigned long long)r->n);
            T = std::min<int64_t>(shape.tile_elems[b] > 0 ? shape.tile_elems[b] : r->n,
                                  kMaxTileElems);
            ulog = std::min<int>(2, std::max<int>(0, shape.unroll_log2[b]));
        }
        h_plan[i] = ServePlan{nplan, T, ulog, 0};
        if (r->src_kind < 0) nplan += (r->n + T - 1) / T;
    }
    int64_t ntiles = 0;
    if (!fused) {
        // The tile list of step (b), before anything of this batch is queued:
        // the slot is idle (its last batch completed), so a region too short
        // for this batch can be reallocated here (the tables are rewritten).
        ntiles = serve_tiles(h_table, count, shape, tile_cap(elems), s.host<TileRec>(s.off_tiles),
                             s.cap_tiles);
        if (ntiles > s.cap_tiles) {
            std::vector<wxpy_desc> t(h_table, h_table + count);
            std::vector<uint64_t> sd(h_seeds, h_seeds + count);
            std::vector<ServePlan> pl(h_plan, h_plan + count);
            if ((e = alloc_stage(s, s.cap_segs, ntiles + ntiles / 4)) != cudaSuccess) return e;
            h_table = s.host<wxpy_desc>(s.off_table);
            h_seeds = s.host<uint64_t>(s.off_seeds);
            h_plan = s.host<ServePlan>(s.off_plan);
            std::copy(t.begin(), t.end(), h_table);
            std::copy(sd.begin(), sd.end(), h_seeds);
            std::copy(pl.begin(), pl.end(), h_plan);
            ntiles = serve_tiles(h_table, count, shape, tile_cap(elems),
                                 s.host<TileRec>(s.off_tiles), s.cap_tiles);
        }
    }
    // One upload: status word (zero), descriptors, seeds, plan, and the tiles.
    *s.host<unsigned>(0) = 0u;
    const size_t up = fused ? s.off_tiles : s.off_tiles + sizeof(TileRec) * (size_t)ntiles;
    e = cudaMemcpyAsync(s.d_stage, s.h_stage, up, cudaMemcpyHostToDevice, s.stream);
    if (e != cudaSuccess) return e;
    const wxpy_desc *d_table = s.dev<wxpy_desc>(s.off_table);
    const uint64_t *d_seeds = s.dev<uint64_t>(s.off_seeds);
    const ServePlan *d_plan = s.dev<ServePlan>(s.off_plan);
    const int64_t wpb = 256 / 32;
    if (fused) {
        const unsigned grid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((int64_t)8 * sv->sm_count, (nplan + wpb - 1) / wpb));
        e = injected_launch_error();
        if (e != cudaSuccess) return e;
        serve_fused_kernel<kServePM><<<grid, 256, 0, s.stream>>>(d_table, d_seeds, d_plan, count,
                                                                 nplan);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sv->launches += 1;
        return cudaEventRecord(s.done, s.stream);
    }
    // (a) inputs into the resident buffers
    for (const Request *r : batch)
        if (r->src_kind >= 0 && (e = copy_in(r, s.stream)) != cudaSuccess) return e;
    if (nplan > 0) {
        const unsigned grid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((int64_t)8 * sv->sm_count, (nplan + wpb - 1) / wpb));
        e = injected_launch_error();
        if (e != cudaSuccess) return e;
        serve_fill_kernel<<<grid, 256, 0, s.stream>>>(d_table, d_seeds, d_plan, count, nplan);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sv->launches += 1;
    }
    // (b) one segmented launch over the batch: reads x, y, writes w; its
    // status word (uploaded as zero) comes back with the batch
    unsigned *d_status = s.dev<unsigned>(0);
    e = launch_segmented(d_table, s.dev<TileRec>(s.off_tiles), ntiles, d_status, shape,
                         sv->sm_count, s.stream);
    if (e != cudaSuccess) return e;
    sv->launches += 1;
    e = cudaMemcpyAsync(s.h_status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s.stream);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(s.done, s.stream);
}

void scheduler(wxpy_server *sv) {
    cudaSetDevice(sv->device);
    std::vector<Request *> batch;
    while (true) {
        bool progress = false;
        // 1. completions
        for (Slot &s : sv->slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            const Clock::time_point now = Clock::now();
            std::lock_guard<std::mutex> lk(sv->mu);
            retire_slot(sv, s, now, q == cudaSuccess ? 0 : (int)q);
            progress = true;
        }
        // 2. admission, in arrival order (with backfill ahead of a blocked head)
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            auto admit = [&](uint64_t ticket, int64_t off) {
                Request &r = sv->reqs[ticket];
                const int64_t vb = round_up(r.n * 8, kBlock);
                r.off = off;
                r.bytes = 3 * vb;
                r.x = (double *)(sv->arena_base + off);
                r.y = (double *)(sv->arena_base + off + vb);
                r.w = (double *)(sv->arena_base + off + 2 * vb);
                r.state = kAdmitted;
                sv->admitted.push_back(ticket);
                ++sv->resident;
                progress = true;
            };
            while (!sv->queue.empty() && sv->resident < sv->cfg.max_slots) {
                const uint64_t head = sv->queue.front();
                const int64_t need = 3 * round_up(sv->reqs[head].n * 8, kBlock);
                const int64_t off = sv->arena.alloc(need);
                const Clock::time_point now = Clock::now();
                if (off >= 0) {
                    // (its wait is accounted up to the previous scheduler pass)
                    if (sv->waiting_head == head) sv->waiting_head = 0;
                    sv->queue.pop_front();
                    admit(head, off);
                    continue;
                }
                // the head waits: account the time since the last check by cause
                if (sv->waiting_head != head) {
                    sv->waiting_head = head;
                    sv->head_since = sv->head_accounted = now;
                } else {
                    const double dt = seconds(now - sv->head_accounted);
                    if (sv->arena.size() - sv->arena.used() >= need) sv->head_wait_frag += dt;
                    else sv->head_wait_full += dt;
                    sv->head_accounted = now;
                }
                const int32_t aging = sv->cfg.admission;
                if (aging > 0 && seconds(now - sv->head_since) * 1e6 < (double)aging) {
                    // backfill: later requests that fit, up to 64 places back
                    for (size_t k = 1; k < sv->queue.size() && k <= 64 &&
                                       sv->resident < sv->cfg.max_slots;) {
                        const uint64_t t = sv->queue[k];
                        const int64_t off2 = sv->arena.alloc(3 * round_up(sv->reqs[t].n * 8, kBlock));
                        if (off2 < 0) {
                            ++k;
                            continue;
                        }
                        sv->queue.erase(sv->queue.begin() + (std::ptrdiff_t)k);
                        admit(t, off2);
                        ++sv->backfilled;
                    }
                }
                break;
            }
        }
        // 3. launch the admitted requests on a free stream
        Slot *free_slot_ptr = nullptr;
        for (size_t k = 0; k < sv->slots.size(); ++k) {
            Slot &s = sv->slots[(sv->next_slot + k) % sv->slots.size()];
            if (!s.busy) {
                free_slot_ptr = &s;
                sv->next_slot = (int)((sv->next_slot + k + 1) % sv->slots.size());
                break;
            }
        }
        if (free_slot_ptr) {
            Slot &s = *free_slot_ptr;
            batch.clear();
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                const int64_t maxb = sv->cfg.max_batch;
                // A batch holds at most its stream's share of the budget, so
                // that the next batch can be admitted and launched on another
                // stream while this one runs.
                const int64_t share = sv->arena.size() / (int64_t)sv->slots.size();
                int64_t bytes = 0;
                size_t taken = 0;
                for (; taken < sv->admitted.size() && (int64_t)taken < maxb &&
                       (int64_t)taken < s.cap_segs;
                     ++taken) {
                    Request &r = sv->reqs[sv->admitted[taken]];
                    if (taken > 0 && bytes + r.bytes > share) break;
                    bytes += r.bytes;
                    r.state = kRunning;
                    batch.push_back(&r);
                    s.tickets.push_back(sv->admitted[taken]);
                }
                sv->admitted.erase(sv->admitted.begin(), sv->admitted.begin() + taken);
                if (!batch.empty()) {
                    s.busy = true;
                    int64_t inflight = 0;
                    for (const Slot &o : sv->slots) inflight += o.busy ? 1 : 0;
                    sv->max_inflight = std::max(sv->max_inflight, inflight);
                    ++sv->batches;
                    sv->requests_launched += (int64_t)batch.size();
                }
            }
            if (!batch.empty()) {
                const Clock::time_point t0 = Clock::now();
                s.t_launch = t0;
                const cudaError_t e = launch_batch(sv, s, batch);
                {
                    const double dt = seconds(Clock::now() - t0);
                    std::lock_guard<std::mutex> lk(sv->mu);
                    sv->max_launch_host = std::max(sv->max_launch_host, dt);
                    s.host_s = dt;
                    s.count = (int64_t)batch.size();
                    s.elems = 0;
                    for (const Request *r : batch) s.elems += r->n;
                }
                progress = true;
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    // the stream may still hold part of the batch: let it drain
                    cudaStreamSynchronize(s.stream);
                    std::lock_guard<std::mutex> lk(sv->mu);
                    retire_slot(sv, s, Clock::now(), (int)e);
                }
            }
        }
        if (sv->stop.load()) {
            bool idle = true;
            for (Slot &s : sv->slots) idle = idle && !s.busy;
            if (idle) break;
        }
        if (!progress) {
            bool inflight = false;
            for (Slot &s : sv->slots) inflight = inflight || s.busy;
            std::unique_lock<std::mutex> lk(sv->mu);
            if (!inflight && !sv->stop.load() && sv->queue.empty() && sv->admitted.empty()) {
                sv->cv_submit.wait_for(lk, std::chrono::milliseconds(2));
            } else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(inflight ? 2 : 20));
            }
        }
    }
}

int submit_locked(wxpy_server *sv, int64_t n, double alpha, uint64_t seed, bool auto_release,
                  uint64_t *ticket, int src_kind = -1, const double *src_x = nullptr,
                  const double *src_y = nullptr) {
    if (n <= 0) return fail(WXPY_EINVAL, "request needs n > 0");
    const int64_t bytes = 3 * round_up(n * 8, kBlock);
    if (n > (int64_t)1 << 40 || bytes > sv->arena.size())
        return fail(WXPY_EBUDGET, "request of %lld elements needs %lld bytes, budget %lld",
                    (long long)n, (long long)bytes, (long long)sv->arena.size());
    if ((int64_t)sv->queue.size() >= sv->cfg.max_queue) {
        ++sv->rejected;
        return fail(WXPY_EBUSY, "admission queue full (%lld)", (long long)sv->cfg.max_queue);
    }
    const uint64_t t = sv->next_ticket++;
    Request &r = sv->reqs[t];
    r.n = n;
    r.alpha = alpha;
    r.seed = seed;
    r.src_kind = src_kind;
    r.src_x = src_x;
    r.src_y = src_y;
    r.auto_release = auto_release;
    r.t_submit = Clock::now();
    sv->queue.push_back(t);
    sv->max_queue = std::max<int64_t>(sv->max_queue, (int64_t)sv->queue.size());
    ++sv->submitted;
    *ticket = t;
    return WXPY_OK;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)k, v.end());
    return v[k];
}

}  // namespace
}  // namespace wx

extern "C" {

int wxpy_server_create(const wxpy_server_config *cfg, wxpy_server **out) {
    if (!cfg || !out) return fail(WXPY_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->budget_bytes < 3 * kBlock || cfg->max_slots < 1 || cfg->n_streams < 1 ||
        cfg->n_streams > 16 || cfg->max_batch < 1 || cfg->max_queue < 1 ||
        (cfg->mode != WXPY_SERVE_BATCHED && cfg->mode != WXPY_SERVE_SERIAL &&
         cfg->mode != WXPY_SERVE_FUSED) ||
        cfg->admission < 0)
        return fail(WXPY_EINVAL, "bad server configuration");
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    auto *sv = new wxpy_server;
    sv->cfg = *cfg;
    sv->device = dp->device;
    sv->sm_count = dp->sm_count;
    cudaError_t e = cudaMalloc(&sv->arena_base, (size_t)cfg->budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete sv;
        return fail(WXPY_ENOMEM, "server arena of %lld bytes", (long long)cfg->budget_bytes);
    }
    sv->arena.init(cfg->budget_bytes);
    const int64_t segs = std::min<int64_t>(cfg->max_batch, cfg->max_slots);
    // Tile list: room for a batch of its stream's share of the budget at the
    // default tile length, plus one ragged tile per request; a batch that
    // needs more (shorter tuned tiles) grows it.
    const int64_t tiles = cfg->budget_bytes / cfg->n_streams / (24 * 8192) + segs;
    sv->slots.resize((size_t)cfg->n_streams);
    for (Slot &s : sv->slots) {
        e = init_slot(s, segs, tiles);
        if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
        for (Slot &s : sv->slots) free_slot(s);
        cudaFree(sv->arena_base);
        delete sv;
        return fail_cuda(e, "server stream/staging setup");
    }
    sv->t_reset = Clock::now();
    sv->sched = std::thread(scheduler, sv);
    *out = sv;
    return WXPY_OK;
}

int wxpy_server_submit(wxpy_server *sv, int64_t n, double alpha, uint64_t seed, uint64_t *ticket) {
    if (!sv || !ticket) return fail(WXPY_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    const int st = submit_locked(sv, n, alpha, seed, false, ticket);
    if (st == WXPY_OK) sv->cv_submit.notify_one();
    return st;
}

int wxpy_server_submit_data(wxpy_server *sv, int64_t n, double alpha, const double *x,
                            const double *y, int kind, uint64_t *ticket) {
    if (!sv || !ticket) return fail(WXPY_EINVAL, "null argument");
    if (kind != WXPY_SERVE_DATA_DEVICE && kind != WXPY_SERVE_DATA_HOST)
        return fail(WXPY_EINVAL, "data kind %d is neither device (0) nor host (1)", kind);
    if (n > 0 && (!x || !y)) return fail(WXPY_EINVAL, "null input pointer");
    if ((((uintptr_t)x) | ((uintptr_t)y)) & 7u)
        return fail(WXPY_EINVAL, "input pointers must be 8-byte aligned");
    if (sv->cfg.mode == WXPY_SERVE_FUSED)
        return fail(WXPY_EINVAL, "the fused mode generates its inputs: caller data needs the "
                                 "batched or serial mode");
    std::lock_guard<std::mutex> lk(sv->mu);
    const int st = submit_locked(sv, n, alpha, 0, false, ticket, kind, x, y);
    if (st == WXPY_OK) sv->cv_submit.notify_one();
    return st;
}

int wxpy_server_poll(wxpy_server *sv, uint64_t ticket, int *state, double *latency_s) {
    if (!sv || !state) return fail(WXPY_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(WXPY_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    *state = it->second.state;
    if (latency_s)
        *latency_s = it->second.state >= kDone ? seconds(it->second.t_done - it->second.t_submit) : -1.0;
    return WXPY_OK;
}

int wxpy_server_wait(wxpy_server *sv, uint64_t ticket, double timeout_s, double *latency_s) {
    if (!sv) return fail(WXPY_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s));
    while (true) {
        auto it = sv->reqs.find(ticket);
        if (it == sv->reqs.end()) return fail(WXPY_ENOTFOUND, "unknown ticket");
        if (it->second.state >= kDone) {
            if (latency_s) *latency_s = seconds(it->second.t_done - it->second.t_submit);
            if (it->second.state == kFailed) {
                if (it->second.error == kTileCheckFailed)
                    return fail(WXPY_ECUDA, "request failed: the batch's tile bounds check fired");
                return fail(WXPY_ECUDA, "request failed with CUDA error %d", it->second.error);
            }
            return WXPY_OK;
        }
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            Clock::now() >= deadline)
            return fail(WXPY_ETIMEOUT, "ticket %llu not done after %.3f s",
                        (unsigned long long)ticket, timeout_s);
    }
}

int wxpy_server_result(wxpy_server *sv, uint64_t ticket, const double **x, const double **y,
                       const double **w, int64_t *n) {
    if (!sv) return fail(WXPY_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(WXPY_ENOTFOUND, "unknown ticket");
    const Request &r = it->second;
    if (r.state != kDone) return fail(WXPY_EBUSY, "ticket not done (state %d)", r.state);
    if (x) *x = r.x;
    if (y) *y = r.y;
    if (w) *w = r.w;
    if (n) *n = r.n;
    return WXPY_OK;
}

int wxpy_server_release(wxpy_server *sv, uint64_t ticket) {
    if (!sv) return fail(WXPY_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(WXPY_ENOTFOUND, "unknown ticket");
    if (it->second.state < kDone) return fail(WXPY_EBUSY, "ticket still in flight");
    if (it->second.off >= 0) sv->arena.release(it->second.off, it->second.bytes);
    --sv->resident;
    sv->reqs.erase(it);
    sv->cv_submit.notify_one();  // memory and a slot freed
    return WXPY_OK;
}

int wxpy_server_get_stats(wxpy_server *sv, int reset, wxpy_server_stats *out) {
    if (!sv || !out) return fail(WXPY_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = sv->submitted;
    out->rejected = sv->rejected;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued_now = (int64_t)sv->queue.size();
    out->resident_now = sv->resident;
    out->max_queue = sv->max_queue;
    out->batches = sv->batches;
    out->launches = sv->launches;
    out->mean_batch = sv->batches ? (double)sv->requests_launched / (double)sv->batches : 0.0;
    out->elements_done = sv->elements_done;
    out->arena_used = sv->arena.used();
    out->max_inflight = sv->max_inflight;
    out->max_launch_host_s = sv->max_launch_host;
    out->max_batch_s = sv->max_batch;
    out->window_s = seconds(Clock::now() - sv->t_reset);
    out->p50_s = percentile(sv->latencies, 0.50);
    out->p99_s = percentile(sv->latencies, 0.99);
    double sum = 0, mx = 0;
    for (double v : sv->latencies) {
        sum += v;
        mx = std::max(mx, v);
    }
    out->mean_s = sv->latencies.empty() ? 0.0 : sum / (double)sv->latencies.size();
    out->max_s = mx;
    out->head_wait_frag_s = sv->head_wait_frag;
    out->head_wait_full_s = sv->head_wait_full;
    out->backfilled = sv->backfilled;
    out->reserved = 0;
    if (reset) {
        sv->head_wait_frag = sv->head_wait_full = 0;
        sv->backfilled = 0;
        sv->submitted = sv->rejected = sv->completed = sv->failed = 0;
        sv->batches = sv->launches = sv->elements_done = sv->requests_launched = 0;
        sv->max_inflight = 0;
        sv->max_launch_host = sv->max_batch = 0;
        sv->max_queue = (int64_t)sv->queue.size();
        sv->latencies.clear();
        sv->t_reset = Clock::now();
    }
    return WXPY_OK;
}

int wxpy_server_destroy(wxpy_server *sv) {
    if (!sv) return WXPY_OK;
    sv->stop.store(true);
    sv->cv_submit.notify_all();
    if (sv->sched.joinable()) sv->sched.join();
    for (Slot &s : sv->slots) free_slot(s);
    if (sv->arena_base) cudaFree(sv->arena_base);
    delete sv;
    return WXPY_OK;
}

int wxpy_server_loadgen(wxpy_server *sv, const wxpy_loadgen_config *cfg, wxpy_loadgen_result *out) {
    if (!sv || !cfg || !out) return fail(WXPY_EINVAL, "null argument");
    if (!(cfg->rate > 0) || !(cfg->duration_s > 0) || cfg->n_min < 1 || cfg->n_max < cfg->n_min)
        return fail(WXPY_EINVAL, "bad load configuration");
    std::memset(out, 0, sizeof *out);
    wxpy_server_stats dummy;
    wxpy_server_get_stats(sv, 1, &dummy);  // start a fresh statistics window
    // Arrival times, lengths and alphas from the counter-based generator.
    auto u01 = [](uint64_t key, uint64_t i) {
        return (double)(mix64(key + (i + 1) * kGolden) >> 11) * 0x1.0p-53;
    };
    const uint64_t k_gap = stream_key_of(cfg->seed, 5), k_len = stream_key_of(cfg->seed, 4),
                   k_alpha = stream_key_of(cfg->seed, 3);
    const double la = std::log2((double)cfg->n_min), lb = std::log2((double)cfg->n_max + 1.0);
    const Clock::time_point t0 = Clock::now();
    double t_next = 0.0;
    int64_t offered = 0, accepted = 0, refused = 0;
    std::vector<uint64_t> tickets;
    for (uint64_t i = 0;; ++i) {
        t_next += -std::log1p(-u01(k_gap, i)) / cfg->rate;
        if (t_next > cfg->duration_s) break;
        while (seconds(Clock::now() - t0) < t_next) {
            const double ahead = t_next - seconds(Clock::now() - t0);
            if (ahead > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        int64_t n = (int64_t)std::floor(std::exp2(la + u01(k_len, i) * (lb - la)));
        n = std::min<int64_t>(std::max<int64_t>(n, cfg->n_min), cfg->n_max);
        const double alpha = 4.0 * u01(k_alpha, i) - 2.0;
        ++offered;
        uint64_t t = 0;
        int st;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            st = submit_locked(sv, n, alpha, cfg->seed + 1000003ull * (i + 1), true, &t);
        }
        if (st == WXPY_OK) {
            ++accepted;
            sv->cv_submit.notify_one();
        } else {
            ++refused;
        }
    }
    const double arrivals_end = seconds(Clock::now() - t0);
    int64_t backlog_end = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        backlog_end = (int64_t)sv->queue.size() + (int64_t)sv->admitted.size();
    }
    // Drain: wait (bounded) for every accepted request to finish.
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(cfg->drain_timeout_s));
    bool drained = false;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        while (true) {
            if (sv->completed + sv->failed >= accepted) {
                drained = true;
                break;
            }
            if (Clock::now() >= deadline) break;
            sv->cv_done.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    const double wall = seconds(Clock::now() - t0);
    wxpy_server_stats s;
    wxpy_server_get_stats(sv, 0, &s);
    out->offered = offered;
    out->submitted = accepted;
    out->rejected = refused;
    out->completed = s.completed;
    out->failed = s.failed;
    out->p50_s = s.p50_s;
    out->p99_s = s.p99_s;
    out->mean_s = s.mean_s;
    out->max_s = s.max_s;
    out->wall_s = wall;
    out->arrivals_s = arrivals_end;
    out->elem_per_s = (double)s.elements_done / wall;
    out->gbs = 24.0 * (double)s.elements_done / wall / 1e9;
    out->max_queue = s.max_queue;
    out->backlog_at_end = backlog_end;
    out->mean_batch = s.mean_batch;
    out->launches = s.launches;
    out->drained = drained ? 1 : 0;
    return drained ? WXPY_OK : fail(WXPY_ETIMEOUT, "load did not drain within %.1f s",
                                    cfg->drain_timeout_s);
}

}  // extern "C"
