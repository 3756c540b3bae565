// reduce.cu -- the update of the paper (Sec. 3, Fig. 1: w = RN(RN(alpha*x) + y))
// fused with a reduction of its result: a squared 2-norm (terms RN(w*w)) or a
// dot product with a fourth vector (terms RN(w*z)), as a residual update is
// followed by its norm.  One pass over the vectors; the reduction is a fixed
// tree, so the result is the same bits whatever the grid.
//
// The tree (the operation's definition; the paper has no reduction): tiles of
// T = 8192 consecutive indices; the sum of a tile is the halving tree
// (e[i] = RN(e[i] + e[i + s]) for s = T/2, ..., 1, +0 past n); the tile sums,
// padded with +0 to a power of two, are summed by the same tree.
//
// Mapping.  A block of 256 threads takes a tile; thread t owns the 32-byte
// vectors at element 1024k + 4t (k = 0..7), so element i = 1024k + 4t + q has
// bits 12..10 = k, 9..7 = warp, 6..2 = lane, 1..0 = q.  The halving tree
// reduces bits from the top down, and each level is done where its two
// operands live: bits 12..10 inside the thread (k and k + 4 as they arrive,
// then k + 2, k + 1), bits 9..7 across warps through shared memory, bits 6..2
// by warp shuffles, bits 1..0 inside lane 0.  Every load and store is a
// coalesced 32-byte vector.  The tile sums go to a workspace; the last block to
// finish (an atomic ticket, no waiting) sums them with the same tree.
//
// Pipes: per element two products (alpha*x and the term) and, on average, two
// sums (the update's and one tree level).  A share of the tiles (mul_sixteenths,
// by a rotation over blocks and tile iterations) computes both products in the
// integer pipelines (fp64_mul.cuh); the sums stay in FP64.  The choice is made
// once per tile between two instantiated bodies: a choice per element slot was
// if-converted by the compiler, which then issued the FP64 body, predicated
// off, for the integer-pipeline slots too.  The bits are the same either way.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "fp64_emu.cuh"
#include "fp64_mul.cuh"
#include "internal.h"

namespace wx {
namespace {

constexpr int kTile = 8192;
constexpr int kThreads = 256;
constexpr int64_t kHeaderBytes = 256;  // ticket counter, then the tile sums

struct ReduceArgs {
    const double *x, *y, *z;  // z: dot only
    double *w;
    double *result;
    unsigned int *ticket;
    double *partial;  // padded_tiles slots
    int64_t n, ntiles, padded_tiles;
    double alpha;
    MulCoef ca;
    int mul_sixteenths;
};

__device__ __forceinline__ uint64_t bits_of(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ double double_of(uint64_t b) { return __longlong_as_double((long long)b); }

// w and the term of one element.  EMU: both products in the integer pipelines.
template <int KIND, bool EMU>
__device__ __forceinline__ void element(const ReduceArgs &a, double x, double y, double z,
                                        double &w, double &t) {
    if constexpr (EMU) {
        bool slow = false;
        uint64_t pb = mul_rn_core(a.ca, bits_of(x), slow);
        if (slow) pb = mul_rn_hw_bits(bits_of(a.alpha), bits_of(x));  // out of line
        w = __dadd_rn(double_of(pb), y);
        const uint64_t wb = opaque_bits(w);
        const uint64_t tb = mul_rn_bits(wb, KIND == 0 ? wb : bits_of(z));
        t = double_of(tb);
    } else {
        w = __dadd_rn(__dmul_rn(a.alpha, x), y);
        t = __dmul_rn(w, KIND == 0 ? w : z);
    }
}

// Coherent evict-first loads: w may be one of the inputs.
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    asm volatile("ld.global.cs.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p));
}

__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
    asm volatile("st.global.cs.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
                 "d"(v[2]), "d"(v[3])
                 : "memory");
}

// Terms of the four elements of vector k of this thread (base = its first
// index in the vector); w stored.  VEC: whole, 32-byte co-aligned vector;
// else element by element with bounds (ragged tile, or unaligned pointers),
// +0 terms past n.
template <int KIND, bool EMU, bool VEC>
__device__ __forceinline__ void vector_terms(const ReduceArgs &a, int64_t base, double (&t)[4]) {
    double x[4], y[4], z[4], w[4];
    if constexpr (VEC) {
        ld4(a.x + base, x);
        ld4(a.y + base, y);
        if constexpr (KIND == 1) ld4(a.z + base, z);
#pragma unroll
        for (int q = 0; q < 4; ++q) element<KIND, EMU>(a, x[q], y[q], KIND == 1 ? z[q] : 0.0, w[q], t[q]);
        st4(a.w + base, w);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = base + q;
            if (i < a.n) {
                const double zi = KIND == 1 ? a.z[i] : 0.0;
                double wi;
                element<KIND, EMU>(a, a.x[i], a.y[i], zi, wi, t[q]);
                a.w[i] = wi;
            } else {
                t[q] = 0.0;
            }
        }
    }
}

// The sum of tile `tile`; valid in thread 0.  red: 256 x 4 doubles of shared memory.
template <int KIND, bool VEC, bool EMU>
__device__ double tile_sum(const ReduceArgs &a, int64_t tile, double (*red)[4]) {
    const int t = threadIdx.x, lane = t & 31;
    const int64_t t0 = tile * kTile + 4 * t;
    // bits 12..10: r[j] = tree over k = j, j+4 (bit 12), then j, j+2 (bit 11), then bit 10
    double r[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double lo[4], hi[4];
        vector_terms<KIND, EMU, VEC>(a, t0 + 1024 * j, lo);
        vector_terms<KIND, EMU, VEC>(a, t0 + 1024 * (j + 4), hi);
#pragma unroll
        for (int q = 0; q < 4; ++q) r[j][q] = __dadd_rn(lo[q], hi[q]);
    }
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        r[0][q] = __dadd_rn(r[0][q], r[2][q]);
        r[1][q] = __dadd_rn(r[1][q], r[3][q]);
        v[q] = __dadd_rn(r[0][q], r[1][q]);
    }
    // bits 9..7: threads t and t + 128, t + 64, t + 32 through shared memory
#pragma unroll
    for (int q = 0; q < 4; ++q) red[t][q] = v[q];
    __syncthreads();
    if (t < 128) {
#pragma unroll
        for (int q = 0; q < 4; ++q) red[t][q] = __dadd_rn(red[t][q], red[t + 128][q]);
    }
    __syncthreads();
    if (t < 64) {
#pragma unroll
        for (int q = 0; q < 4; ++q) red[t][q] = __dadd_rn(red[t][q], red[t + 64][q]);
    }
    __syncthreads();
    double s = 0.0;
    if (t < 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(red[t][q], red[t + 32][q]);
        // bits 6..2: lanes L and L + 16, 8, 4, 2, 1
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(v[q], __shfl_down_sync(0xffffffffu, v[q], sh));
        }
        // bits 1..0 in lane 0: q and q + 2, then q and q + 1
        if (lane == 0) s = __dadd_rn(__dadd_rn(v[0], v[2]), __dadd_rn(v[1], v[3]));
    }
    __syncthreads();  // red is reused by the next tile
    return s;
}

// The halving tree over partial[0 .. padded-1] (entries from ntiles on are +0),
// by one block, in place.
__device__ void final_tree(const ReduceArgs &a) {
    const int t = threadIdx.x;
    for (int64_t i = a.ntiles + t; i < a.padded_tiles; i += blockDim.x) a.partial[i] = 0.0;
    __syncthreads();
    for (int64_t s = a.padded_tiles / 2; s >= 1; s >>= 1) {
        for (int64_t i = t; i < s; i += blockDim.x)
            a.partial[i] = __dadd_rn(__ldcg(a.partial + i), __ldcg(a.partial + i + s));
        __syncthreads();
    }
    if (t == 0) *a.result = __ldcg(a.partial);
}

// Four resident blocks (64 registers): measured 4-5 % faster than three.
template <int KIND, bool VEC>
__global__ void __launch_bounds__(kThreads, 4) wxpy_reduce_kernel(const ReduceArgs a) {
    __shared__ double red[kThreads][4];
    __shared__ bool last;
    const int64_t full = VEC ? a.n / kTile : 0;  // tiles with every element present
    unsigned slot = (blockIdx.x * 7u) & 15u;    // block-uniform rotation of the pipe choice
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double s;
        if (tile >= full) s = tile_sum<KIND, false, false>(a, tile, red);
        else if ((int)slot < a.mul_sixteenths) s = tile_sum<KIND, VEC, true>(a, tile, red);
        else s = tile_sum<KIND, VEC, false>(a, tile, red);
        if (threadIdx.x == 0) a.partial[tile] = s;
        slot = (slot + 1u) & 15u;
    }
    // the last block to finish sums the tile sums
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        final_tree(a);
    }
}

template <int KIND, bool VEC>
int blocks_per_sm(int device) {
    static std::atomic<int> cached[64];
    if (device < 0 || device >= 64) return 1;
    int v = cached[device].load(std::memory_order_relaxed);
    if (v > 0) return v;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wxpy_reduce_kernel<KIND, VEC>, kThreads,
                                                      0) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    cached[device].store(nb, std::memory_order_relaxed);
    return nb;
}

std::atomic<int> g_reduce_mul{-1};
constexpr int kDefaultMulSixteenths = 16;  // measured fastest on GB300 (both operations)

int64_t padded_tiles(int64_t n) {
    const int64_t tiles = (n + kTile - 1) / kTile;
    int64_t p = 1;
    while (p < tiles) p *= 2;
    return p;
}

bool overlaps(const void *a, int64_t abytes, const void *b, int64_t bbytes) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + (uintptr_t)bbytes && pb < pa + (uintptr_t)abytes;
}

template <int KIND>
int launch_reduce(int64_t n, double alpha, const double *x, const double *y, double *w,
                  const double *z, double *result, void *workspace, int64_t ws_bytes,
                  cudaStream_t s) {
    if (n < 0) return fail(WXPY_EINVAL, "n = %lld is negative", (long long)n);
    if (n > ((int64_t)1 << 40)) return fail(WXPY_EINVAL, "n too large");
    if (!result || ((uintptr_t)result & 7)) return fail(WXPY_EINVAL, "null or misaligned result");
    if (n > 0) {
        const double *in[3] = {x, y, z};
        for (int k = 0; k < (KIND == 1 ? 3 : 2); ++k)
            if (!in[k] || ((uintptr_t)in[k] & 7))
                return fail(WXPY_EINVAL, "null or misaligned input %d", k);
        if (!w || ((uintptr_t)w & 7)) return fail(WXPY_EINVAL, "null or misaligned w");
        const int64_t bytes = n * 8;
        for (int k = 0; k < (KIND == 1 ? 3 : 2); ++k)
            if (in[k] != w && overlaps(in[k], bytes, w, bytes))
                return fail(WXPY_EOVERLAP, "w partially overlaps input %d", k);
        if (overlaps(result, 8, w, bytes)) return fail(WXPY_EOVERLAP, "result inside w");
        const int64_t need = wxpy_reduce_workspace_bytes(n);
        if (!workspace || ((uintptr_t)workspace & 15) || ws_bytes < need)
            return fail(WXPY_EINVAL, "workspace: need %lld bytes, 16-byte aligned", (long long)need);
        for (int k = 0; k < (KIND == 1 ? 3 : 2); ++k)
            if (overlaps(workspace, need, in[k], bytes))
                return fail(WXPY_EOVERLAP, "workspace overlaps input %d", k);
        if (overlaps(workspace, need, w, bytes) || overlaps(workspace, need, result, 8))
            return fail(WXPY_EOVERLAP, "workspace overlaps w or result");
    }
    cudaError_t e = injected_launch_error();
    if (e != cudaSuccess) return fail_cuda(e, "reduce launch");
    if (n == 0) {
        e = cudaMemsetAsync(result, 0, 8, s);  // the empty sum is +0
        return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "reduce empty");
    }
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    ReduceArgs a;
    a.x = x;
    a.y = y;
    a.z = KIND == 1 ? z : nullptr;
    a.w = w;
    a.result = result;
    a.ticket = (unsigned int *)workspace;
    a.partial = (double *)((char *)workspace + kHeaderBytes);
    a.n = n;
    a.ntiles = (n + kTile - 1) / kTile;
    a.padded_tiles = padded_tiles(n);
    a.alpha = alpha;
    uint64_t ab;
    std::memcpy(&ab, &alpha, 8);
    a.ca = mul_coef_of(ab);
    const int m = g_reduce_mul.load();
    a.mul_sixteenths = m < 0 ? kDefaultMulSixteenths : m;
    uintptr_t any = (uintptr_t)x | (uintptr_t)y | (uintptr_t)w | (KIND == 1 ? (uintptr_t)z : 0);
    const bool vec = (any & 31u) == 0;
    e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return fail_cuda(e, "reduce ticket");
    const int nb = vec ? blocks_per_sm<KIND, true>(dp->device) : blocks_per_sm<KIND, false>(dp->device);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)dp->sm_count * nb, a.ntiles));
    if (vec) wxpy_reduce_kernel<KIND, true><<<(unsigned)grid, kThreads, 0, s>>>(a);
    else wxpy_reduce_kernel<KIND, false><<<(unsigned)grid, kThreads, 0, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "reduce launch");
}

}  // namespace
}  // namespace wx

using namespace wx;

extern "C" {

int64_t wxpy_reduce_workspace_bytes(int64_t n) {
    if (n < 0) return -1;
    return kHeaderBytes + 8 * padded_tiles(n);
}

int wxpy_norm2(int64_t n, double alpha, const double *x, const double *y, double *w,
               double *result, void *workspace, int64_t workspace_bytes, void *stream) {
    return launch_reduce<0>(n, alpha, x, y, w, nullptr, result, workspace, workspace_bytes,
                            (cudaStream_t)stream);
}

int wxpy_dot(int64_t n, double alpha, const double *x, const double *y, double *w,
             const double *z, double *result, void *workspace, int64_t workspace_bytes,
             void *stream) {
    return launch_reduce<1>(n, alpha, x, y, w, z, result, workspace, workspace_bytes,
                            (cudaStream_t)stream);
}

int wxpy_reduce_pipes(int mul_sixteenths) {
    if (mul_sixteenths < -1 || mul_sixteenths > 16)
        return fail(WXPY_EINVAL, "mul_sixteenths must be -1..16");
    g_reduce_mul.store(mul_sixteenths);
    return WXPY_OK;
}

}  // extern "C"
