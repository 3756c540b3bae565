// batch.cu -- many independent VecWXPY problems in one persistent, segmented launch.
//
// Segment s computes w_s = RN(RN(alpha_s*x_s) + y_s) over n_s elements (the
// vecwxpy of paper Sec. 3, Fig. 1, once per segment).  Instead of one launch
// per segment, a plan cuts every segment into tiles (per-size-bucket tile
// length), and one launch of a persistent kernel walks the tile list: warp k
// of the grid takes tiles k, k + W, k + 2W, ... (W = warps in the grid).  A
// tile record names its segment and its element range; the warp reads the
// segment's descriptor (pointers, alpha, n) from the caller's device table,
// peels the tile's head to the widest vector width the three pointers share,
// streams the body with per-bucket unroll, and finishes the ragged tail.
//
// The plan owns the device tile list and a status word.  The kernel checks
// every tile against the n of the descriptor it reads and skips (and flags)
// any tile that would reach past it, so a device table whose lengths differ
// from the host table the plan was built from cannot write out of bounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "trace.h"
#include "seg_tile.cuh"

namespace wx {

static_assert(sizeof(TileRec) == 16, "tile records are 16 bytes");
static_assert(sizeof(wxpy_desc) == 40, "descriptor layout");

struct SegParams {
    const wxpy_desc *table;
    const TileRec *tiles;
    int64_t ntiles;
    unsigned *status;  // bit 0: a tile exceeded its descriptor's n
};

// EMU: the integer-pipeline share (0 none, 1 half the sums, 3 every product),
// chosen per launch.
template <int EMU>
__global__ void __launch_bounds__(256, 2) wxpy_seg_kernel(const SegParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < p.ntiles; t += nwarps) {
        const TileRec r = p.tiles[t];
        const wxpy_desc d = p.table[r.seg];
        const int64_t len = (int64_t)(r.len_ul & kLenMask);
        if (r.begin < 0 || len <= 0 || r.begin + len > d.n) {
            if (lane == 0) atomicOr(p.status, 1u);
            continue;
        }
        tile_wxpy<EMU>(d.x + r.begin, d.y + r.begin, d.w + r.begin, d.alpha, len, lane,
                       1 << (r.len_ul >> 30));
    }
}

static const void *seg_kernel_fn(int offload) {
    return offload == 3   ? (const void *)&wxpy_seg_kernel<3>
           : offload != 0 ? (const void *)&wxpy_seg_kernel<1>
                          : (const void *)&wxpy_seg_kernel<0>;
}

static cudaError_t seg_launch(int offload, unsigned grid, int threads, const SegParams &sp,
                              cudaStream_t s) {
    if (offload == 3) wxpy_seg_kernel<3><<<grid, threads, 0, s>>>(sp);
    else if (offload) wxpy_seg_kernel<1><<<grid, threads, 0, s>>>(sp);
    else wxpy_seg_kernel<0><<<grid, threads, 0, s>>>(sp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- shapes
// Per-bucket tile length (elements; 0 = whole segment) and unroll, plus the
// launch geometry; set by the batch search or left at the defaults.
std::mutex g_shape_mu;
BatchShape g_shape = default_batch_shape();

BatchShape default_batch_shape() {
    BatchShape s;
    s.threads = 256;
    s.blocks_per_sm = 4;
    s.offload = 3;  // every product in the integer pipelines: 6910 GB/s against 6767
                    // with half the sums there, on the 4096-segment batch (GB300)
    for (int b = 0; b < kBuckets; ++b) {
        s.tile_elems[b] = b < 13 ? 0 : 8192;
        s.unroll_log2[b] = 2;
    }
    return s;
}

BatchShape current_batch_shape() {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    return g_shape;
}

void set_batch_shape(const BatchShape &s) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shape = s;
}

// ---------------------------------------------------------------- validation
namespace {
struct Interval {
    uintptr_t lo, hi;
    int64_t seg;
};
}  // namespace

int validate_table(const wxpy_desc *t, int64_t count) {
    if (count < 0) return fail(WXPY_EINVAL, "negative segment count");
    if (count > 0 && !t) return fail(WXPY_EINVAL, "null descriptor table");
    if (count > (int64_t)0x7fffffff) return fail(WXPY_EINVAL, "more than 2^31-1 segments");
    std::vector<Interval> writes;
    writes.reserve((size_t)count);
    for (int64_t s = 0; s < count; ++s) {
        CallClass c;
        int st = classify(t[s].n, t[s].x, t[s].y, t[s].w, &c);
        if (st != WXPY_OK)
            return fail(st, "segment %lld: %s", (long long)s, wxpy_last_error_message());
        if (t[s].n > 0)
            writes.push_back({(uintptr_t)t[s].w, (uintptr_t)t[s].w + (uintptr_t)t[s].n * 8u, s});
    }
    // No two segments may write overlapping ranges, and no segment may read a
    // range another segment writes: segments run concurrently.
    std::sort(writes.begin(), writes.end(),
              [](const Interval &a, const Interval &b) { return a.lo < b.lo; });
    for (size_t i = 1; i < writes.size(); ++i)
        if (writes[i].lo < writes[i - 1].hi)
            return fail(WXPY_EOVERLAP, "segments %lld and %lld write overlapping ranges",
                        (long long)writes[i - 1].seg, (long long)writes[i].seg);
    for (int64_t s = 0; s < count; ++s) {
        if (t[s].n == 0) continue;
        for (const double *r : {t[s].x, t[s].y}) {
            const uintptr_t lo = (uintptr_t)r, hi = lo + (uintptr_t)t[s].n * 8u;
            // first write interval with hi > lo
            auto it = std::upper_bound(writes.begin(), writes.end(), lo,
                                       [](uintptr_t v, const Interval &w) { return v < w.hi; });
            for (; it != writes.end() && it->lo < hi; ++it)
                if (it->seg != s)
                    return fail(WXPY_EOVERLAP, "segment %lld reads what segment %lld writes",
                                (long long)s, (long long)it->seg);
        }
    }
    return WXPY_OK;
}

// Tile list of a validated table, largest tiles first (static round-robin
// assignment then spreads the work evenly over the warps).
int64_t build_tiles(const wxpy_desc *t, int64_t count, const BatchShape &shape,
                    std::vector<TileRec> *out) {
    out->clear();
    int64_t total = 0;
    for (int64_t s = 0; s < count; ++s) {
        const int64_t n = t[s].n;
        if (n == 0) continue;
        total += n;
        const int b = 63 - __builtin_clzll((unsigned long long)n);
        int64_t T = shape.tile_elems[b] > 0 ? shape.tile_elems[b] : n;
        T = std::min<int64_t>(T, kMaxTileElems);
        const uint32_t ul = (uint32_t)std::min<int>(2, std::max<int>(0, shape.unroll_log2[b])) << 30;
        for (int64_t b0 = 0; b0 < n; b0 += T)
            out->push_back(TileRec{b0, (int32_t)s, (uint32_t)std::min<int64_t>(T, n - b0) | ul});
    }
    std::stable_sort(out->begin(), out->end(), [](const TileRec &a, const TileRec &b) {
        return (a.len_ul & kLenMask) > (b.len_ul & kLenMask);
    });
    return total;
}

cudaError_t launch_segmented(const wxpy_desc *dev_table, const TileRec *tiles, int64_t ntiles,
                             unsigned *status, const BatchShape &shape, int sm_count,
                             cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    const int64_t wpb = shape.threads / 32;
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)shape.blocks_per_sm * sm_count, (ntiles + wpb - 1) / wpb));
    cudaError_t e = injected_launch_error();
    if (e != cudaSuccess) return e;
    SegParams sp;
    sp.table = dev_table;
    sp.tiles = tiles;
    sp.ntiles = ntiles;
    sp.status = status;
    return seg_launch(shape.offload, grid, shape.threads, sp, s);
}

}  // namespace wx

using namespace wx;

struct wxpy_batch_plan {
    int device = -1;
    int64_t count = 0;
    int64_t ntiles = 0;
    int64_t total_elems = 0;
    BatchShape shape;
    TileRec *d_tiles = nullptr;
    unsigned *d_status = nullptr;
    unsigned grid = 0;
    // graph of the launch, with the table it was built for
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    const wxpy_desc *graph_table = nullptr;
};

namespace {

SegParams params_of(const wxpy_batch_plan *p, const wxpy_desc *dev_table) {
    SegParams sp;
    sp.table = dev_table;
    sp.tiles = p->d_tiles;
    sp.ntiles = p->ntiles;
    sp.status = p->d_status;
    return sp;
}

void destroy_plan(wxpy_batch_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_tiles) cudaFree(p->d_tiles);
    if (p->d_status) cudaFree(p->d_status);
    delete p;
}

}  // namespace

extern "C" {

int wxpy_batch_plan_create(const wxpy_desc *host_table, int64_t count, wxpy_batch_plan **out) {
    if (!out) return fail(WXPY_EINVAL, "null output");
    *out = nullptr;
    int st = validate_table(host_table, count);
    if (st != WXPY_OK) return st;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    auto *p = new wxpy_batch_plan;
    p->device = dp->device;
    p->count = count;
    p->shape = current_batch_shape();
    std::vector<TileRec> tiles;
    p->total_elems = build_tiles(host_table, count, p->shape, &tiles);
    p->ntiles = (int64_t)tiles.size();
    const int64_t warps_per_block = p->shape.threads / 32;
    const int64_t max_grid = (int64_t)p->shape.blocks_per_sm * dp->sm_count;
    p->grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(max_grid, (p->ntiles + warps_per_block - 1) / warps_per_block));
    cudaError_t e = cudaMalloc(&p->d_status, 256);
    if (e == cudaSuccess && p->ntiles > 0)
        e = cudaMalloc(&p->d_tiles, sizeof(TileRec) * (size_t)p->ntiles);
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_plan(p);
        return fail(WXPY_ENOMEM, "batch plan allocation failed");
    }
    e = cudaMemset(p->d_status, 0, 256);
    if (e == cudaSuccess && p->ntiles > 0)
        e = cudaMemcpy(p->d_tiles, tiles.data(), sizeof(TileRec) * tiles.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        destroy_plan(p);
        return fail_cuda(e, "batch plan upload");
    }
    *out = p;
    return WXPY_OK;
}

int wxpy_batch_launch(wxpy_batch_plan *plan, const wxpy_desc *dev_table, void *stream) {
    TraceRange trace("wxpy_batch_launch");
    if (!plan) return fail(WXPY_EINVAL, "null plan");
    if (plan->ntiles == 0) return WXPY_OK;
    if (!dev_table) return fail(WXPY_EINVAL, "null device table");
    cudaError_t e = injected_launch_error();
    if (e == cudaSuccess)
        e = seg_launch(plan->shape.offload, plan->grid, plan->shape.threads,
                       params_of(plan, dev_table), (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "batch kernel launch");
    return WXPY_OK;
}

int wxpy_batch_graph_launch(wxpy_batch_plan *plan, const wxpy_desc *dev_table, void *stream) {
    TraceRange trace("wxpy_batch_graph_launch");
    if (!plan) return fail(WXPY_EINVAL, "null plan");
    if (plan->ntiles == 0) return WXPY_OK;
    if (!dev_table) return fail(WXPY_EINVAL, "null device table");
    cudaError_t e = cudaSuccess;
    SegParams sp = params_of(plan, dev_table);
    void *args[] = {&sp};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void *>(seg_kernel_fn(plan->shape.offload));
    kp.gridDim = dim3(plan->grid);
    kp.blockDim = dim3(plan->shape.threads);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    if (!plan->exec) {
        e = cudaGraphCreate(&plan->graph, 0);
        if (e == cudaSuccess) e = cudaGraphAddKernelNode(&plan->node, plan->graph, nullptr, 0, &kp);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        if (e != cudaSuccess) return fail_cuda(e, "batch graph build");
        plan->graph_table = dev_table;
    } else if (plan->graph_table != dev_table) {
        e = cudaGraphExecKernelNodeSetParams(plan->exec, plan->node, &kp);
        if (e != cudaSuccess) return fail_cuda(e, "batch graph update");
        plan->graph_table = dev_table;
    }
    e = injected_launch_error();
    if (e == cudaSuccess) e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_cuda(e, "batch graph launch");
    return WXPY_OK;
}

int wxpy_batch_plan_info(const wxpy_batch_plan *plan, wxpy_batch_info *out) {
    if (!plan || !out) return fail(WXPY_EINVAL, "null argument");
    std::memset(out, 0, sizeof *out);
    out->segments = plan->count;
    out->tiles = plan->ntiles;
    out->elements = plan->total_elems;
    out->bytes = plan->total_elems * 24;
    out->grid = (int32_t)plan->grid;
    out->threads = plan->shape.threads;
    return WXPY_OK;
}

int wxpy_batch_status(wxpy_batch_plan *plan, unsigned *status, int clear) {
    if (!plan || !status) return fail(WXPY_EINVAL, "null argument");
    cudaError_t e = cudaMemcpy(status, plan->d_status, sizeof *status, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && clear) e = cudaMemset(plan->d_status, 0, sizeof *status);
    if (e != cudaSuccess) return fail_cuda(e, "batch status read");
    return WXPY_OK;
}

int wxpy_batch_plan_destroy(wxpy_batch_plan *plan) {
    destroy_plan(plan);
    return WXPY_OK;
}

int wxpy_batch(const wxpy_desc *host_table, const wxpy_desc *dev_table, int64_t count,
               void *stream) {
    int st = validate_table(host_table, count);
    if (st != WXPY_OK) return st;
    if (count == 0) return WXPY_OK;
    if (!dev_table) return fail(WXPY_EINVAL, "null device table");
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const BatchShape shape = current_batch_shape();
    std::vector<TileRec> tiles;
    build_tiles(host_table, count, shape, &tiles);
    if (tiles.empty()) return WXPY_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // Stream-ordered scratch: tile list + status word, freed after the kernel.
    const size_t bytes = sizeof(TileRec) * tiles.size() + 256;
    void *buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WXPY_ENOMEM, "batch scratch allocation failed");
    }
    auto *d_tiles = (TileRec *)((char *)buf + 256);
    e = cudaMemsetAsync(buf, 0, 256, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TileRec) * tiles.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        SegParams sp;
        sp.table = dev_table;
        sp.tiles = d_tiles;
        sp.ntiles = (int64_t)tiles.size();
        sp.status = (unsigned *)buf;
        const int64_t wpb = shape.threads / 32;
        const unsigned grid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((int64_t)shape.blocks_per_sm * dp->sm_count,
                                 ((int64_t)tiles.size() + wpb - 1) / wpb));
        e = injected_launch_error();
        if (e == cudaSuccess) e = seg_launch(shape.offload, grid, shape.threads, sp, s);
    }
    cudaError_t e2 = cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return fail_cuda(e, "batch launch");
    if (e2 != cudaSuccess) return fail_cuda(e2, "batch scratch free");
    return WXPY_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batch search
// The search of Sec. 2 for the batched launch: for each size bucket b, a
// synthetic batch whose segments all fall in b (lengths spread over
// [2^b, 2^(b+1)), starts 256-byte aligned, as separate allocations would be)
// is run with every (tile length, unroll) candidate; each candidate's output
// must equal, bit for bit, the reference results obtained by running the
// plain reference variant on every segment; the fastest (median of `reps`
// back-to-back launches) is stored for bucket b.  Then the grid size
// (blocks per SM) is chosen the same way on a mixed batch of buckets bmin..bmax.
namespace wx {
namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    int alloc(size_t bytes) {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(WXPY_ENOMEM, "batch search allocation of %zu bytes failed", bytes);
        }
        return WXPY_OK;
    }
};

struct SynthBatch {
    std::vector<wxpy_desc> host;
    DevBuf x, y, w, wref, table, tiles, status, count;
    int64_t elems = 0, slots = 0;
};

// Lengths for a batch: bucket b only (b >= 0), or log-uniform over buckets
// [bmin, bmax] (b < 0).
int make_batch(int b, int bmin, int bmax, SynthBatch *sb, cudaStream_t s) {
    std::vector<int64_t> ns;
    if (b >= 0) {
        const int64_t lo = (int64_t)1 << b;
        const int64_t target = std::max<int64_t>((int64_t)1 << 25, 8 * lo);
        const int64_t count = std::min<int64_t>(32768, std::max<int64_t>(8, target / lo));
        for (int64_t i = 0; i < count; ++i) ns.push_back(lo + (lo * i) / count);
    } else {
        const int count = 2048;
        uint64_t z = 0x1234567ull;
        for (int i = 0; i < count; ++i) {
            z += 0x9E3779B97F4A7C15ull;
            uint64_t h = z;
            h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ull;
            h = (h ^ (h >> 27)) * 0x94D049BB133111EBull;
            h ^= h >> 31;
            const int bb = bmin + (int)(h % (uint64_t)(bmax - bmin + 1));
            const int64_t lo = (int64_t)1 << bb;
            ns.push_back(lo + (int64_t)((h >> 20) % (uint64_t)lo));
        }
    }
    // 32-element (256-byte) aligned starts
    int64_t slots = 0;
    for (int64_t n : ns) slots += (n + 31) / 32 * 32;
    sb->slots = slots;
    int st;
    const size_t bytes = (size_t)slots * 8;
    if ((st = sb->x.alloc(bytes)) || (st = sb->y.alloc(bytes)) || (st = sb->w.alloc(bytes)) ||
        (st = sb->wref.alloc(bytes)) ||
        (st = sb->table.alloc(sizeof(wxpy_desc) * ns.size())) || (st = sb->status.alloc(256)) ||
        (st = sb->count.alloc(64)))
        return st;
    if ((st = launch_fill_uniform((double *)sb->x.p, slots, 77, 1, 0, -1.0, 1.0, s)) ||
        (st = launch_fill_uniform((double *)sb->y.p, slots, 77, 2, 0, -1.0, 1.0, s)))
        return st;
    int64_t off = 0;
    sb->host.clear();
    for (size_t i = 0; i < ns.size(); ++i) {
        const double alpha = 0.5 + 0.001 * (double)(i % 1000);
        sb->host.push_back(wxpy_desc{ns[i], alpha, (double *)sb->x.p + off, (double *)sb->y.p + off,
                                     (double *)sb->w.p + off});
        off += (ns[i] + 31) / 32 * 32;
    }
    sb->elems = 0;
    for (int64_t n : ns) sb->elems += n;
    cudaError_t e = cudaMemcpyAsync(sb->table.p, sb->host.data(), sizeof(wxpy_desc) * ns.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb->status.p, 0, 256, s);
    // reference results of Sec. 2: the plain reference variant, segment by segment
    if (e == cudaSuccess) e = cudaMemsetAsync(sb->wref.p, 0xff, bytes, s);
    for (size_t i = 0; i < ns.size() && e == cudaSuccess; ++i) {
        const wxpy_desc &d = sb->host[i];
        SingleArgs a{d.x, d.y, (double *)sb->wref.p + (d.w - (double *)sb->w.p), d.alpha, d.n, 0, 0, MulCoef{}};
        e = launch_reference((unsigned)((d.n + 255) / 256), 256u, a, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "batch search setup");
    return WXPY_OK;
}

// Uploads the tiles of `shape` and returns the grid.  Tiles buffer grows as needed.
int upload_tiles(SynthBatch &sb, const BatchShape &shape, const DeviceProps &dp, int64_t *ntiles,
                 unsigned *grid, cudaStream_t s) {
    std::vector<TileRec> tiles;
    build_tiles(sb.host.data(), (int64_t)sb.host.size(), shape, &tiles);
    *ntiles = (int64_t)tiles.size();
    static thread_local size_t cap = 0;
    if (!sb.tiles.p || cap < tiles.size()) {
        if (sb.tiles.p) {
            cudaFree(sb.tiles.p);
            sb.tiles.p = nullptr;
        }
        int st = sb.tiles.alloc(sizeof(TileRec) * tiles.size());
        if (st) return st;
        cap = tiles.size();
    }
    cudaError_t e = cudaMemcpyAsync(sb.tiles.p, tiles.data(), sizeof(TileRec) * tiles.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "batch search tile upload");
    const int64_t wpb = shape.threads / 32;
    *grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)shape.blocks_per_sm * dp.sm_count, (*ntiles + wpb - 1) / wpb));
    return WXPY_OK;
}

int run_shape(SynthBatch &sb, const BatchShape &shape, const DeviceProps &dp, int reps,
              cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double *median_us,
              unsigned long long *mismatches) {
    int64_t ntiles = 0;
    unsigned grid = 0;
    int st = upload_tiles(sb, shape, dp, &ntiles, &grid, s);
    if (st) return st;
    SegParams sp;
    sp.table = (const wxpy_desc *)sb.table.p;
    sp.tiles = (const TileRec *)sb.tiles.p;
    sp.ntiles = ntiles;
    sp.status = (unsigned *)sb.status.p;
    // verification run on a poisoned output
    cudaError_t e = cudaMemsetAsync(sb.w.p, 0xff, (size_t)sb.slots * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sb.count.p, 0, 8, s);
    if (e == cudaSuccess) e = seg_launch(shape.offload, grid, shape.threads, sp, s);
    if (e != cudaSuccess) return fail_cuda(e, "batch search launch");
    if ((st = launch_count_mismatch((const double *)sb.w.p, (const double *)sb.wref.p, sb.slots,
                                    (unsigned long long *)sb.count.p, s)))
        return st;
    e = cudaMemcpyAsync(mismatches, sb.count.p, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "batch search verify");
    std::vector<float> ms(reps);
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        seg_launch(shape.offload, grid, shape.threads, sp, s);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return fail_cuda(e, "batch search timing");
        cudaEventElapsedTime(&ms[r], e0, e1);
    }
    std::sort(ms.begin(), ms.end());
    *median_us = 1e3 * (double)ms[reps / 2];
    return WXPY_OK;
}

}  // namespace

int batch_tune_impl(int bmin, int bmax, unsigned flags, wxpy_batch_tune_result *out) {
    TraceRange trace("wxpy_batch_tune");
    if (bmin < 0 || bmax > 30 || bmin > bmax) return fail(WXPY_EINVAL, "bucket range must be within 0..30");
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const bool quick = flags & WXPY_TUNE_QUICK;
    const int reps = quick ? 3 : 7;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return fail_cuda(e, "batch search stream");
    struct Cleanup {
        cudaStream_t s;
        cudaEvent_t a, b;
        ~Cleanup() {
            if (s) cudaStreamSynchronize(s);
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
            if (s) cudaStreamDestroy(s);
        }
    } cleanup{s, e0, e1};
    BatchShape shape = current_batch_shape();
    if (out) std::memset(out, 0, sizeof *out);
    int rejected = 0, candidates = 0;
    static const int32_t kTiles[] = {0, 1024, 2048, 4096, 8192, 16384, 32768, 65536};
    for (int b = bmin; b <= bmax; ++b) {
        SynthBatch sb;
        if ((st = make_batch(b, 0, 0, &sb, s))) return st;
        double best_us = 1e30;
        int32_t best_tile = shape.tile_elems[b];
        int8_t best_u = shape.unroll_log2[b];
        for (int32_t T : kTiles) {
            if (T != 0 && T >= ((int64_t)2 << b)) continue;  // no cut: same as whole segment
            for (int8_t ul = 0; ul < 3; ++ul) {
                if (quick && (ul == 0 || (T != 0 && T != 8192))) continue;
                BatchShape cand = shape;
                cand.tile_elems[b] = T;
                cand.unroll_log2[b] = ul;
                double us = 0;
                unsigned long long bad = 0;
                if ((st = run_shape(sb, cand, *dp, reps, s, e0, e1, &us, &bad))) return st;
                ++candidates;
                if (bad) {
                    ++rejected;
                    continue;
                }
                if (us < best_us) {
                    best_us = us;
                    best_tile = T;
                    best_u = ul;
                }
            }
        }
        if (best_us >= 1e30) return fail(WXPY_EMISMATCH, "every batch candidate of bucket %d differed", b);
        shape.tile_elems[b] = best_tile;
        shape.unroll_log2[b] = best_u;
        if (out) {
            out->tile_elems[b] = best_tile;
            out->unroll[b] = 1 << best_u;
            out->us[b] = best_us;
            out->gbs[b] = 24.0 * (double)sb.elems / (best_us * 1e-6) / 1e9;
        }
    }
    // grid size on a mixed batch
    {
        SynthBatch sb;
        if ((st = make_batch(-1, bmin, bmax, &sb, s))) return st;
        double best_us = 1e30;
        int best_bps = shape.blocks_per_sm, best_of = shape.offload;
        for (int of : {0, 1, 3})
            for (int bps : {1, 2, 4, 8}) {
                BatchShape cand = shape;
                cand.blocks_per_sm = bps;
                cand.offload = of;
                double us = 0;
                unsigned long long bad = 0;
                if ((st = run_shape(sb, cand, *dp, reps, s, e0, e1, &us, &bad))) return st;
                ++candidates;
                if (bad) {
                    ++rejected;
                    continue;
                }
                if (us < best_us) {
                    best_us = us;
                    best_bps = bps;
                    best_of = of;
                }
            }
        shape.blocks_per_sm = best_bps;
        shape.offload = best_of;
        if (out) {
            out->blocks_per_sm = best_bps;
            out->fp64_offload = best_of;
            out->mixed_us = best_us;
            out->mixed_gbs = 24.0 * (double)sb.elems / (best_us * 1e-6) / 1e9;
        }
    }
    set_batch_shape(shape);
    if (out) {
        out->candidates = candidates;
        out->rejected = rejected;
        out->threads = shape.threads;
    }
    return WXPY_OK;
}

}  // namespace wx

extern "C" int wxpy_batch_tune(int bucket_min, int bucket_max, unsigned flags,
                               wxpy_batch_tune_result *out) {
    return wx::batch_tune_impl(bucket_min, bucket_max, flags, out);
}

extern "C" int wxpy_batch_shape_get(int bucket, int *tile_elems, int *unroll) {
    if (bucket < 0 || bucket >= wx::kBuckets || !tile_elems || !unroll)
        return wx::fail(WXPY_EINVAL, "bad bucket %d", bucket);
    const wx::BatchShape s = wx::current_batch_shape();
    *tile_elems = s.tile_elems[bucket];
    *unroll = 1 << s.unroll_log2[bucket];
    return WXPY_OK;
}

extern "C" int wxpy_batch_shape_set(int bucket, int tile_elems, int unroll) {
    if (bucket < 0 || bucket >= wx::kBuckets) return wx::fail(WXPY_EINVAL, "bad bucket %d", bucket);
    if (tile_elems < 0 || (tile_elems % 32) != 0 || tile_elems > (1 << 30))
        return wx::fail(WXPY_EINVAL, "tile length must be 0 or a multiple of 32 up to 2^30");
    int ul = unroll == 1 ? 0 : unroll == 2 ? 1 : unroll == 4 ? 2 : -1;
    if (ul < 0) return wx::fail(WXPY_EINVAL, "unroll must be 1, 2 or 4");
    wx::BatchShape s = wx::current_batch_shape();
    s.tile_elems[bucket] = tile_elems;
    s.unroll_log2[bucket] = (int8_t)ul;
    wx::set_batch_shape(s);
    return WXPY_OK;
}

extern "C" int wxpy_batch_shape_reset(void) {
    wx::set_batch_shape(wx::default_batch_shape());
    return WXPY_OK;
}
