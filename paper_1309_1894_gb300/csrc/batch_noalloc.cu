// batch_noalloc.cu -- the batched launch for callers that cannot allocate.
//
// wxpy_batch_plan_create() allocates device memory for its tile list, and the
// one-shot wxpy_batch() takes stream-ordered scratch with cudaMallocAsync.
// Some callers can do neither: code whose device memory is entirely owned by
// another allocator (a framework's caching pool or a server's fixed arena)
// that must not see a cudaMalloc it did not make, one that could fail or
// synchronise the device in the middle of its work; and hot loops that cannot
// afford an allocation call at all.  wxpy_batch_noalloc() serves them: it
// computes the same results as wxpy_batch() from the caller's device table,
// and its only scratch is the fixed file-scope device array below, which
// every GPU that loads the library holds until the process exits.
//
// The plan is made on the device, in the caller's stream, in three launches:
//   1. one block scans the table's lengths into a tile prefix (each segment
//      gets at most kMaxTiles / count tiles, so the list always fits);
//   2. a grid maps every tile to its segment and index (binary search);
//   3. a persistent grid of warps runs the tiles, as the batched kernel does.
// Descriptors with n <= 0, or with a null or misaligned pointer, get no
// tiles: they are skipped, never dereferenced.  Nothing else is checked: the
// caller guarantees that within each descriptor w is x, is y, or overlaps
// neither, and that no descriptor writes what another one reads or writes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace wx {
namespace {

constexpr int64_t kNaMaxSegments = 65536;  // largest table this entry accepts
constexpr int64_t kNaMaxTiles = 262144;    // tile slots in the scratch
constexpr int64_t kNaBaseTile = 8192;      // elements per tile before clamping

struct NaScratch {
    int64_t prefix[kNaMaxSegments + 1];  // tiles of segments [0, s)
    int64_t tile_len[kNaMaxSegments];    // elements per tile of segment s
    int32_t tile_seg[kNaMaxTiles];       // segment of tile t
    int32_t tile_idx[kNaMaxTiles];       // index of tile t within its segment
    int64_t ntiles;
};

// The scratch: about 3 MiB, fixed, shared by every call of the process on a
// device.  Host code must not use this name as an address (it is a host-side
// stand-in); the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

__device__ __forceinline__ bool usable(const wxpy_desc &d) {
    const uintptr_t bits = (uintptr_t)d.x | (uintptr_t)d.y | (uintptr_t)d.w;
    return d.n > 0 && d.x && d.y && d.w && (bits & 7u) == 0;
}

// 1. Per-segment tile count and length, exclusive prefix over segments.
__global__ void __launch_bounds__(1024) na_plan_kernel(const wxpy_desc *table, int64_t count,
                                                       NaScratch *sc) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t running;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per_seg = kNaMaxTiles / count;  // >= 4 since count <= kNaMaxSegments
    if (tid == 0) running = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += 1024) {
        const int64_t s = base + tid;
        int64_t tiles = 0;
        if (s < count) {
            const wxpy_desc d = table[s];
            int64_t len = 0;
            if (usable(d)) {
                int64_t t = (d.n + kNaBaseTile - 1) / kNaBaseTile;
                if (t > per_seg) t = per_seg;
                len = ((d.n + t - 1) / t + 31) / 32 * 32;
                tiles = (d.n + len - 1) / len;
            }
            sc->tile_len[s] = len;
        }
        // inclusive scan of `tiles` across the block
        int64_t v = tiles;
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        if (lane == 31) warp_sums[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int64_t ws = warp_sums[lane];
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, ws, off);
                if (lane >= off) ws += u;
            }
            warp_sums[lane] = ws;  // inclusive over warps
        }
        __syncthreads();
        const int64_t before_warp = wid ? warp_sums[wid - 1] : 0;
        const int64_t inclusive = running + before_warp + v;
        if (s < count) sc->prefix[s] = inclusive - tiles;
        __syncthreads();
        if (tid == 1023) running = inclusive;
        __syncthreads();
    }
    if (tid == 0) {
        sc->prefix[count] = running;
        sc->ntiles = running;
    }
}

// 2. Segment and index of every tile.
__global__ void na_map_kernel(int64_t count, NaScratch *sc) {
    const int64_t ntiles = sc->ntiles;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += stride) {
        int64_t lo = 0, hi = count - 1;  // largest s with prefix[s] <= t
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (sc->prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        sc->tile_seg[t] = (int32_t)lo;
        sc->tile_idx[t] = (int32_t)(t - sc->prefix[lo]);
    }
}

// 32-byte vectors, four per lane per pass, all loads before any store.
__device__ __forceinline__ void na_body4(const double *x, const double *y, double *w,
                                         double alpha, int64_t nch, int lane) {
    constexpr int U = 4;
    for (int64_t c0 = lane; c0 < nch; c0 += 32 * U) {
        double xv[U][4], yv[U][4], wv[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = c0 + 32 * u;
            if (c < nch) {
                ld_vec<4, 2>(x + c * 4, xv[u]);
                ld_vec<4, 2>(y + c * 4, yv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = c0 + 32 * u;
            if (c < nch) {
                wxpy_vec<4>(alpha, xv[u], yv[u], wv[u]);
                st_vec<4, 2>(w + c * 4, wv[u]);
            }
        }
    }
}

__device__ __forceinline__ void na_scalar(const double *x, const double *y, double *w, double alpha,
                                          int64_t e) {
    double xv[1], yv[1], wv[1];
    ld_vec<1, 2>(x + e, xv);
    ld_vec<1, 2>(y + e, yv);
    wxpy_vec<1>(alpha, xv, yv, wv);
    st_vec<1, 2>(w + e, wv);
}

// 3. Persistent warps over the tiles.
__global__ void __launch_bounds__(256, 2) na_run_kernel(const wxpy_desc *table, const NaScratch *sc) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntiles = sc->ntiles;
    for (int64_t t = warp; t < ntiles; t += nwarps) {
        const int32_t s = sc->tile_seg[t];
        const wxpy_desc d = table[s];
        const int64_t T = sc->tile_len[s];
        const int64_t begin = (int64_t)sc->tile_idx[t] * T;
        const int64_t len = min(T, d.n - begin);
        if (len <= 0) continue;
        const double *x = d.x + begin;
        const double *y = d.y + begin;
        double *w = d.w + begin;
        const uintptr_t ax = (uintptr_t)x, ay = (uintptr_t)y, aw = (uintptr_t)w;
        if ((((ax ^ aw) | (ay ^ aw)) & 31u) == 0) {
            const int64_t head = min(len, (int64_t)((4 - (int)((aw >> 3) & 3)) & 3));
            const int64_t nch = (len - head) / 4;
            const int64_t body_end = head + nch * 4;
            if (lane < head) na_scalar(x, y, w, d.alpha, lane);
            if (lane >= 4 && body_end + (lane - 4) < len)
                na_scalar(x, y, w, d.alpha, body_end + (lane - 4));
            na_body4(x + head, y + head, w + head, d.alpha, nch, lane);
        } else {
            for (int64_t e = lane; e < len; e += 32) na_scalar(x, y, w, d.alpha, e);
        }
    }
}

constexpr int kMaxDev = 64;
// Device address of the scratch array per device: null until a lookup has
// succeeded.  Only a successful lookup is kept, so a lookup that failed (a
// first call made during a stream capture, or with an error pending) is
// simply tried again by the next call.
std::atomic<void *> g_na_ptr[kMaxDev];
std::mutex g_na_mu;

// The scratch's device address on device `dev` (current); nullptr and the
// error recorded when the lookup fails.
NaScratch *scratch_address(int dev, int *status) {
    void *p = g_na_ptr[dev].load(std::memory_order_acquire);
    if (p) return (NaScratch *)p;
    std::lock_guard<std::mutex> lk(g_na_mu);
    p = g_na_ptr[dev].load(std::memory_order_relaxed);
    if (!p) {
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();  // clear a non-sticky error; the next call retries
            *status = fail_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                "cudaGetSymbolAddress(scratch)");
            return nullptr;
        }
        g_na_ptr[dev].store(p, std::memory_order_release);
    }
    return (NaScratch *)p;
}

}  // namespace
}  // namespace wx

using namespace wx;

extern "C" int wxpy_batch_noalloc(const wxpy_desc *dev_table, int64_t count, void *stream) {
    if (count < 0) return fail(WXPY_EINVAL, "negative segment count");
    if (count == 0) return WXPY_OK;
    if (count > kNaMaxSegments)
        return fail(WXPY_EINVAL,
                    "%lld segments exceed the %lld that the fixed scratch of "
                    "wxpy_batch_noalloc holds; use wxpy_batch or split the table",
                    (long long)count, (long long)kNaMaxSegments);
    if (!dev_table || ((uintptr_t)dev_table & 7u))
        return fail(WXPY_EINVAL, "null or misaligned device table");
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const int dev = dp->device;
    if (dev >= kMaxDev) return fail(WXPY_EINVAL, "device ordinal %d out of range", dev);
    // With the device current: the device address of the scratch array,
    // looked up on the first successful call for this device.
    NaScratch *sc = scratch_address(dev, &st);
    if (!sc) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = injected_launch_error();
    if (e == cudaSuccess) {
        na_plan_kernel<<<1, 1024, 0, s>>>(dev_table, count, sc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        na_map_kernel<<<(unsigned)dp->sm_count * 2, 256, 0, s>>>(count, sc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        na_run_kernel<<<(unsigned)dp->sm_count * 4, 256, 0, s>>>(dev_table, sc);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail_cuda(e, "wxpy_batch_noalloc launch");
    return WXPY_OK;
}
