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
// Register-loaded kernel (the default).  A persistent grid of 256-thread
// blocks, four per SM; a block takes a tile, thread t the 32-byte vectors at
// 1024k + 4t (k = 0..7), so element i = 1024k + 4t + q has bits 12..10 = k,
// 9..7 = warp, 6..2 = lane, 1..0 = q.  The halving tree reduces bits from the
// top down, each level where its operands live: bits 12..10 inside the
// thread, 9..7 across warps through shared memory, 6..2 by warp shuffles,
// 1..0 inside lane 0.  With pointers that are not 32-byte co-aligned (and for
// the last, ragged tile) the same threads read and write every element on its
// own.  For norm2, the first 0..3 in-thread levels may run as the integer-
// pipeline sum of non-negative values (fp64_addpos.cuh).
//
// Staged kernels (variants 1..3, co-aligned pointers).  One producer warp
// copies a tile as eight 1024-element chunks of every input into a shared-
// memory ring (bulk asynchronous copies completed on "full" mbarriers; a stage
// is reused once all eight consumer warps have released it on its "empty"
// barrier).  Chunk c of a tile holds indices 1024c .. 1024c + 1023, and
// consumer thread (warp v, lane l) takes the 16-byte pairs 128v + 64h + 2l
// (h = 0, 1) of every chunk, so element i = 1024c + 128v + 64h + 2l + q has
// bits 12..10 = c, 9..7 = v, 6 = h, 5..1 = l, 0 = q; every shared-memory and
// global access of a warp is 512 contiguous bytes.  The halving tree:
//   - bits 12..10 in the thread: the producer copies the chunks in bit-
//     reversed order (0, 4, 2, 6, 1, 5, 3, 7), so consecutive chunk pairs
//     are the tree's first level and their four sums, kept in order, its
//     next two;
//   - bits 9..7 across warps: every warp writes its four node values to one
//     of two exchange slots (an mbarrier pair per slot, so no warp waits for
//     the others except through a bounded wait), and one warp, rotating with
//     the tile, finishes the tile: bits 9..7, then bit 6 in the thread,
//     bits 5..1 by warp shuffles, bit 0 in lane 0.
// The last tile, when n is not a multiple of 8192, is read from global memory
// by the same threads in the same order, +0 past n.  Every mbarrier wait is
// bounded (bulk.cuh); one that runs out ends the kernel and is reported by
// wxpy_reduce_status().
//
// Either way the tile sums go to a workspace, and the last block to finish
// (an atomic ticket, no waiting) sums them with the same tree.
//
// Pipes: per element two products (alpha*x and the term) and, on average, two
// sums (the update's and one tree level).  A share of the tiles (mul_sixteenths,
// by a rotation over blocks and tile iterations) computes both products in the
// integer pipelines (fp64_mul.cuh).  The choice is made once per tile between
// two instantiated bodies: a choice per element slot was if-converted by the
// compiler, which then issued the FP64 body, predicated off, for the
// integer-pipeline slots too.  The bits are the same for every configuration;
// wxpy_reduce_tune searches them (reduce_tune.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "bulk.cuh"
#include "internal.h"
#include "reduce_common.cuh"

namespace wx {
namespace {

constexpr int kThreads = 256;

// The sum of tile `tile`; valid in thread 0.  red: 256 x 4 doubles of shared memory.
// SUML (norm2 only): the first SUML of the three in-thread tree levels run as
// integer-pipeline sums of non-negative values.
template <int KIND, bool VEC, bool EMU, int SUML = 0>
__device__ double tile_sum(const ReduceArgs &a, int64_t tile, double (*red)[4]) {
    static_assert(SUML == 0 || KIND == 0, "integer tree sums need non-negative terms");
    const int t = threadIdx.x, lane = t & 31;
    const int64_t t0 = tile * kTile + 4 * t;
    // bits 12..10: r[j] = tree over k = j, j+4 (bit 12), then j, j+2 (bit 11), then bit 10
    // j in the order 0, 2, 1, 3: each pair (0, 2), (1, 3) is summed (bit 11)
    // as soon as both are formed, so at most two level-1 vectors are live
    double p[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double r[2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int j = h + 2 * m;
            double lo[4], hi[4];
            vector_terms<KIND, EMU, VEC>(a, t0 + 1024 * j, lo);
            vector_terms<KIND, EMU, VEC>(a, t0 + 1024 * (j + 4), hi);
#pragma unroll
            for (int q = 0; q < 4; ++q) r[m][q] = tree_add<(SUML >= 1)>(lo[q], hi[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) p[h][q] = tree_add<(SUML >= 2)>(r[0][q], r[1][q]);
    }
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = tree_add<(SUML >= 3)>(p[0][q], p[1][q]);
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

// Register-loaded path: four resident blocks (64 registers), measured 4-5 %
// faster than three.  VEC: full tiles by 32-byte vectors (32-byte aligned
// pointers), else element by element; the last, ragged tile always element by
// element with FP64 products.  The product split applies to every full tile.
template <int KIND, bool VEC, int SUML = 0>
__global__ void __launch_bounds__(kThreads, 4) wxpy_reduce_kernel(const ReduceArgs a) {
    __shared__ double red[kThreads][4];
    __shared__ bool last;
    const int64_t full = a.n / kTile;        // tiles with every element present
    unsigned slot = (blockIdx.x * 7u) & 15u;  // block-uniform rotation of the pipe choice
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        double s;
        if (tile >= full) s = tile_sum<KIND, false, false>(a, tile, red);
        else if ((int)slot < a.mul_sixteenths) s = tile_sum<KIND, VEC, true, SUML>(a, tile, red);
        else s = tile_sum<KIND, VEC, false, SUML>(a, tile, red);
        if (threadIdx.x == 0) a.partial[tile] = s;
        slot = (slot + 1u) & 15u;
    }
    finish_grid(a, last);
}

// ---- staged path ---------------------------------------------------------------

constexpr int kChunk = 1024;  // elements of one input per stage
constexpr int kConsumerWarps = 8;
constexpr int kStagedThreads = 32 * (kConsumerWarps + 1);

// Bitmask of the waits that ran out (1: producer, 2: consumer, 4: exchange);
// read and cleared by wxpy_reduce_status().
__device__ unsigned int g_reduce_fault;

template <int KIND, int S>
struct ReduceStage {
    static constexpr int kIn = KIND == 1 ? 3 : 2;
    static constexpr int kStages = S;
    static constexpr int kStageElems = kIn * kChunk;
    static constexpr int kRingBytes = kStages * kStageElems * 8;
    static constexpr int kExchBytes = 2 * kConsumerWarps * 32 * 4 * 8;  // two slots
    static constexpr int kSmem = kRingBytes + kExchBytes;
};

// j-th chunk of a tile in copy order: j with its three bits reversed.
__device__ __forceinline__ int chunk_of(int j) { return ((j & 1) << 2) | (j & 2) | ((j >> 2) & 1); }

__device__ __forceinline__ void ld_shared_v2(const double *p, double &a, double &b) {
    asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(a), "=d"(b) : "r"(smem_addr(p)));
}

__device__ __forceinline__ void st_shared_v2(double *p, double a, double b) {
    asm volatile("st.shared.v2.f64 [%0], {%1,%2};" ::"r"(smem_addr(p)), "d"(a), "d"(b) : "memory");
}

__device__ __forceinline__ void st_global_v2_cs(double *p, double a, double b) {
    asm volatile("st.global.cs.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(a), "d"(b) : "memory");
}

// Folds the terms of the j-th chunk (in copy order) into the three partial
// vectors: after j = 7, acc0 holds the tree over bits 12..10.
__device__ __forceinline__ void fold(int j, double (&acc0)[4], double (&acc1)[4], double (&acc2)[4],
                                     const double (&e)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        switch (j) {
            case 0: acc0[q] = e[q]; break;
            case 1: acc0[q] = __dadd_rn(acc0[q], e[q]); break;
            case 2: acc1[q] = e[q]; break;
            case 3: acc0[q] = __dadd_rn(acc0[q], __dadd_rn(acc1[q], e[q])); break;
            case 4: acc1[q] = e[q]; break;
            case 5: acc1[q] = __dadd_rn(acc1[q], e[q]); break;
            case 6: acc2[q] = e[q]; break;
            default:
                acc0[q] = __dadd_rn(acc0[q], __dadd_rn(acc1[q], __dadd_rn(acc2[q], e[q])));
        }
    }
}

// Terms of one staged chunk (copy position i of this block), w stored; false
// when the wait ran out.
template <int KIND, int S, bool EMU>
__device__ __forceinline__ bool staged_chunk(const ReduceArgs &a, const double *ring,
                                             uint64_t *full, uint64_t *empty, int i, double *wp,
                                             int off, int lane, double (&e)[4]) {
    using RS = ReduceStage<KIND, S>;
    const int s = i % S;
    if (!mbar_wait(smem_addr(&full[s]), (i / S) & 1)) return false;
    const double *sb = ring + (size_t)s * RS::kStageElems + off;
    double x[4], y[4], z[4], w[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        ld_shared_v2(sb + 64 * h, x[2 * h], x[2 * h + 1]);
        ld_shared_v2(sb + kChunk + 64 * h, y[2 * h], y[2 * h + 1]);
        if constexpr (KIND == 1) ld_shared_v2(sb + 2 * kChunk + 64 * h, z[2 * h], z[2 * h + 1]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_addr(&empty[s]));  // the stage is in registers
#pragma unroll
    for (int q = 0; q < 4; ++q) element<KIND, EMU>(a, x[q], y[q], KIND == 1 ? z[q] : 0.0, w[q], e[q]);
    st_global_v2_cs(wp, w[0], w[1]);
    st_global_v2_cs(wp + 64, w[2], w[3]);
    return true;
}

// The four node values (bits 12..10 reduced; index 2h + q) of this thread for
// a full tile, from the ring; `i` counts the chunks this block has consumed.
// A rolled loop over the four chunk pairs of the copy order, (0, 4), (2, 6),
// (1, 5), (3, 7): each pair's sum is the tree's first level, and a shift of
// the four pair sums through registers leaves them in order for the last two
// levels, so no sum is ever predicated off.  False when a wait ran out.
template <int KIND, int S, bool EMU>
__device__ __forceinline__ bool staged_tile(const ReduceArgs &a, const double *ring,
                                            uint64_t *full, uint64_t *empty, int &i, int64_t tile,
                                            int warp, int lane, double (&v)[4]) {
    const int off = 128 * warp + 2 * lane;
    double r0[4], r1[4], r2[4], r3[4];
#pragma unroll 1
    for (int m = 0; m < 4; ++m) {
        double e0[4], e1[4];
        double *wp = a.w + tile * kTile + off;
        if (!staged_chunk<KIND, S, EMU>(a, ring, full, empty, i, wp + chunk_of(2 * m) * kChunk, off,
                                        lane, e0))
            return false;
        if (!staged_chunk<KIND, S, EMU>(a, ring, full, empty, i + 1,
                                        wp + chunk_of(2 * m + 1) * kChunk, off, lane, e1))
            return false;
        i += 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            r0[q] = r1[q];
            r1[q] = r2[q];
            r2[q] = r3[q];
            r3[q] = __dadd_rn(e0[q], e1[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(__dadd_rn(r0[q], r1[q]), __dadd_rn(r2[q], r3[q]));
    return true;
}

// The same for the last, ragged tile, from global memory; +0 terms past n.
template <int KIND>
__device__ __forceinline__ void ragged_tile(const ReduceArgs &a, int64_t tile, int warp, int lane,
                                            double (&v)[4]) {
    const int off = 128 * warp + 2 * lane;
    double acc1[4], acc2[4];
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
        double e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = tile * kTile + chunk_of(j) * kChunk + off + 64 * (q >> 1) + (q & 1);
            if (i < a.n) {
                double wi;
                element<KIND, false>(a, a.x[i], a.y[i], KIND == 1 ? a.z[i] : 0.0, wi, e[q]);
                a.w[i] = wi;
            } else {
                e[q] = 0.0;
            }
        }
        fold(j, v, acc1, acc2, e);
    }
}

// Exchange slot layout: [warp][h][lane][q], so that every access of a warp is
// 512 contiguous bytes.
__device__ __forceinline__ int exch_index(int warp, int h, int lane) {
    return ((warp * 2 + h) * 32 + lane) * 2;
}

// Bits 9..7, 6, 5..1 and 0 of tile `tile` from an exchange slot, by one warp;
// lane 0 writes the tile sum.
__device__ __forceinline__ void finish_tile(const ReduceArgs &a, const double *xs, int64_t tile,
                                            int lane) {
    double r[kConsumerWarps][4];
#pragma unroll
    for (int v = 0; v < kConsumerWarps; ++v) {
        ld_shared_v2(xs + exch_index(v, 0, lane), r[v][0], r[v][1]);
        ld_shared_v2(xs + exch_index(v, 1, lane), r[v][2], r[v][3]);
    }
    double u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // bits 9..7: v and v + 4, v + 2, v + 1
        const double b0 = __dadd_rn(r[0][q], r[4][q]), b1 = __dadd_rn(r[1][q], r[5][q]);
        const double b2 = __dadd_rn(r[2][q], r[6][q]), b3 = __dadd_rn(r[3][q], r[7][q]);
        u[q] = __dadd_rn(__dadd_rn(b0, b2), __dadd_rn(b1, b3));
    }
    double p[2] = {__dadd_rn(u[0], u[2]), __dadd_rn(u[1], u[3])};  // bit 6: h = 0 and 1
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) {  // bits 5..1: lanes l and l + 16, .., l + 1
#pragma unroll
        for (int q = 0; q < 2; ++q) p[q] = __dadd_rn(p[q], __shfl_down_sync(0xffffffffu, p[q], sh));
    }
    if (lane == 0) {
        a.partial[tile] = __dadd_rn(p[0], p[1]);  // bit 0
        __threadfence();
    }
}

template <int KIND, int S, int MINB>
__global__ void __launch_bounds__(kStagedThreads, MINB) wxpy_reduce_staged_kernel(const ReduceArgs a) {
    using RS = ReduceStage<KIND, S>;
    constexpr int NIN = RS::kIn;
    extern __shared__ __align__(128) double ring[];  // [S][NIN][kChunk], then the exchange
    double *exch = ring + (size_t)S * RS::kStageElems;  // two slots of 8 x 128 doubles
    __shared__ __align__(8) uint64_t full[S], empty[S], xfull[2], xempty[2];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t full_tiles = a.n / kTile;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), kConsumerWarps);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_addr(&xfull[s]), kConsumerWarps);
            mbar_init(smem_addr(&xempty[s]), 1);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0) {
            const double *in[3] = {a.x, a.y, a.z};
            const uint64_t policy = evict_first_policy();
            bool ok = true;
            int i = 0;
            for (int64_t t = blockIdx.x; t < full_tiles && ok; t += gridDim.x) {
                for (int j = 0; j < 8; ++j, ++i) {
                    const int64_t chunk = t * 8 + chunk_of(j);
                    if (chunk == a.drop_chunk) {
                        t = full_tiles;  // stop issuing; the consumers' waits run out
                        break;
                    }
                    const int s = i % S;
                    if (i >= S && !mbar_wait(smem_addr(&empty[s]), ((i / S) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bar = smem_addr(&full[s]);
                    mbar_arrive_expect_tx(bar, NIN * kChunk * 8u);
#pragma unroll
                    for (int k = 0; k < NIN; ++k)
                        bulk_load(smem_addr(ring + (size_t)s * RS::kStageElems + k * kChunk),
                                  in[k] + chunk * kChunk, kChunk * 8u, bar, policy);
                }
            }
            // every issued copy lands before the block exits
            for (int j = i > S ? i - S : 0; j < i; ++j)
                if (!mbar_wait(smem_addr(&full[j % S]), (j / S) & 1)) ok = false;
            if (!ok) atomicOr(&g_reduce_fault, 1u);
        }
    } else {
        unsigned slot = (blockIdx.x * 7u) & 15u;  // block-uniform rotation of the pipe choice
        int i = 0, k = 0;
        for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
            double v[4];
            if (t < full_tiles) {
                const bool ok = (int)slot < a.mul_sixteenths
                                    ? staged_tile<KIND, S, true>(a, ring, full, empty, i, t, warp, lane, v)
                                    : staged_tile<KIND, S, false>(a, ring, full, empty, i, t, warp, lane, v);
                if (!ok) {
                    if (lane == 0) atomicOr(&g_reduce_fault, 2u);
                    break;
                }
            } else {
                ragged_tile<KIND>(a, t, warp, lane, v);
            }
            // exchange slot k & 1: free once the tile two back was finished
            const int xs = k & 1;
            if (k >= 2 && !mbar_wait(smem_addr(&xempty[xs]), ((k >> 1) - 1) & 1)) {
                if (lane == 0) atomicOr(&g_reduce_fault, 4u);
                break;
            }
            double *slotp = exch + (size_t)xs * kConsumerWarps * 128;
            st_shared_v2(slotp + exch_index(warp, 0, lane), v[0], v[1]);
            st_shared_v2(slotp + exch_index(warp, 1, lane), v[2], v[3]);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&xfull[xs]));
            if (warp == (k & 7)) {
                if (!mbar_wait(smem_addr(&xfull[xs]), (k >> 1) & 1)) {
                    if (lane == 0) atomicOr(&g_reduce_fault, 4u);
                    break;
                }
                finish_tile(a, slotp, t, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&xempty[xs]));
            }
            slot = (slot + 1u) & 15u;
        }
    }
    finish_grid(a, last);
}

// Per staged shape and device: the dynamic shared-memory opt-in done and the
// resident blocks per SM (0 on failure).
template <int KIND, int S, int MINB>
int staged_blocks_per_sm(int device) {
    static std::atomic<int> cached[64];
    if (device < 0 || device >= 64) return 0;
    int v = cached[device].load(std::memory_order_relaxed);
    if (v > 0) return v;
    constexpr int smem = ReduceStage<KIND, S>::kSmem;
    if (cudaFuncSetAttribute(wxpy_reduce_staged_kernel<KIND, S, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wxpy_reduce_staged_kernel<KIND, S, MINB>,
                                                      kStagedThreads, smem) != cudaSuccess ||
        nb < 1)
        return 0;
    cached[device].store(nb, std::memory_order_relaxed);
    return nb;
}

template <int KIND, int S, int MINB>
cudaError_t launch_staged(const ReduceArgs &a, const DeviceProps *dp, cudaStream_t s) {
    const int nb = staged_blocks_per_sm<KIND, S, MINB>(dp->device);
    if (nb == 0) {
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? cudaErrorInvalidConfiguration : e;
    }
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)dp->sm_count * nb, a.ntiles));
    wxpy_reduce_staged_kernel<KIND, S, MINB>
        <<<(unsigned)grid, kStagedThreads, ReduceStage<KIND, S>::kSmem, s>>>(a);
    return cudaGetLastError();
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
std::atomic<long long> g_reduce_drop{-1};
std::atomic<int> g_reduce_variant{-1};
std::atomic<int> g_reduce_sum_levels{-1};
std::atomic<int> g_reduce_tuned[2] = {-1, -1};  // (variant << 10) | (suml << 5) | mul
constexpr int kDefaultSumLevels = 0;
constexpr int kReduceVariants = 7;  // 0 register-loaded, 1..3 staged, 4..6 warp-tiled
// Measured on GB300 at n = 2^26 with every product in the integer pipelines
// (GB/s of algorithmic bytes, norm2 / dot): register-loaded 4482 / 5485;
// staged (4, 2) 3771 / 4575, (3, 3) 3822 / 4252, (2, 3) 3904 / 4851.
constexpr int kDefaultVariant[2] = {0, 0};  // norm2, dot
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

// The configuration of a call: each knob set explicitly (>= 0) wins, then the
// searched configuration of the operation, then the built-in default.
ReduceConfig config_for(int kind) {
    ReduceConfig c = reduce_default(kind);
    reduce_tuned_load(kind, &c);
    const int v = g_reduce_variant.load(), m = g_reduce_mul.load(), l = g_reduce_sum_levels.load();
    if (v >= 0) c.variant = v;
    if (m >= 0) c.mul = m;
    if (l >= 0) c.suml = l;
    return c;
}

template <int KIND>
int launch_reduce(int64_t n, double alpha, const double *x, const double *y, double *w,
                  const double *z, double *result, void *workspace, int64_t ws_bytes,
                  ReduceConfig cfg, cudaStream_t s) {
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
    a.mul_sixteenths = cfg.mul;
    a.drop_chunk = g_reduce_drop.load();
    uintptr_t any = (uintptr_t)x | (uintptr_t)y | (uintptr_t)w | (KIND == 1 ? (uintptr_t)z : 0);
    const bool vec = (any & 31u) == 0;
    e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return fail_cuda(e, "reduce ticket");
    const int variant = vec ? cfg.variant : 0;
    if (variant == 0) {
        const int nb = vec ? blocks_per_sm<KIND, true>(dp->device) : blocks_per_sm<KIND, false>(dp->device);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)dp->sm_count * nb, a.ntiles));
        if (!vec) wxpy_reduce_kernel<KIND, false><<<(unsigned)grid, kThreads, 0, s>>>(a);
        else if constexpr (KIND == 0) {
            switch (std::min(cfg.suml, 3)) {  // the form's three in-thread levels
                case 0: wxpy_reduce_kernel<0, true, 0><<<(unsigned)grid, kThreads, 0, s>>>(a); break;
                case 1: wxpy_reduce_kernel<0, true, 1><<<(unsigned)grid, kThreads, 0, s>>>(a); break;
                case 2: wxpy_reduce_kernel<0, true, 2><<<(unsigned)grid, kThreads, 0, s>>>(a); break;
                default: wxpy_reduce_kernel<0, true, 3><<<(unsigned)grid, kThreads, 0, s>>>(a);
            }
        } else {
            wxpy_reduce_kernel<KIND, true><<<(unsigned)grid, kThreads, 0, s>>>(a);
        }
    } else if (variant >= 4) {
        const cudaError_t le = launch_reduce_warp(KIND, KIND == 0 ? cfg.suml : 0, variant - 4, a, dp, s);
        if (le != cudaSuccess) return fail_cuda(le, "warp-tiled reduce launch");
    } else {
        // staged shapes (ring stages, resident blocks): 1 (4, 2), 2 (3, 3), 3 (2, 3)
        cudaError_t le = variant == 1   ? launch_staged<KIND, 4, 2>(a, dp, s)
                         : variant == 2 ? launch_staged<KIND, 3, 3>(a, dp, s)
                                        : launch_staged<KIND, 2, 3>(a, dp, s);
        if (le != cudaSuccess) return fail_cuda(le, "staged reduce launch");
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? WXPY_OK : fail_cuda(e, "reduce launch");
}

}  // namespace

ReduceConfig reduce_default(int kind) {
    return ReduceConfig{kDefaultVariant[kind == 1 ? 1 : 0], kDefaultMulSixteenths,
                        kind == 0 ? kDefaultSumLevels : 0};
}

bool reduce_config_valid(int kind, ReduceConfig c) {
    return c.variant >= 0 && c.variant < kReduceVariants && c.mul >= 0 && c.mul <= 16 &&
           c.suml >= 0 && c.suml <= 6 && (kind == 0 || c.suml == 0);
}

bool reduce_tuned_load(int kind, ReduceConfig *c) {
    if (kind < 0 || kind > 1) return false;
    const int v = g_reduce_tuned[kind].load();
    if (v < 0) return false;
    c->variant = v >> 10;
    c->suml = (v >> 5) & 31;
    c->mul = v & 31;
    return true;
}

void reduce_tuned_store(int kind, const ReduceConfig *c) {
    if (kind < 0 || kind > 1) return;
    g_reduce_tuned[kind].store(c ? (c->variant << 10) | (c->suml << 5) | c->mul : -1);
}

int reduce_run(int kind, int64_t n, double alpha, const double *x, const double *y, double *w,
               const double *z, double *result, void *workspace, int64_t ws_bytes, ReduceConfig c,
               cudaStream_t s) {
    if (!reduce_config_valid(kind, c)) return fail(WXPY_EINVAL, "bad reduce configuration");
    return kind == 1 ? launch_reduce<1>(n, alpha, x, y, w, z, result, workspace, ws_bytes, c, s)
                     : launch_reduce<0>(n, alpha, x, y, w, nullptr, result, workspace, ws_bytes, c, s);
}

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
                            config_for(0), (cudaStream_t)stream);
}

int wxpy_dot(int64_t n, double alpha, const double *x, const double *y, double *w,
             const double *z, double *result, void *workspace, int64_t workspace_bytes,
             void *stream) {
    return launch_reduce<1>(n, alpha, x, y, w, z, result, workspace, workspace_bytes,
                            config_for(1), (cudaStream_t)stream);
}

int wxpy_reduce_status(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned int fault = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&fault, g_reduce_fault, sizeof(fault));
    const unsigned int zero = 0;
    if (e == cudaSuccess && fault) e = cudaMemcpyToSymbol(g_reduce_fault, &zero, sizeof(zero));
    if (e != cudaSuccess) return fail_cuda(e, "reduce status");
    if (fault)
        return fail(WXPY_ETIMEOUT, "a staged reduction's bounded wait ran out (mask %u: 1 producer, "
                    "2 consumer, 4 exchange)", fault);
    return WXPY_OK;
}

int wxpy_debug_reduce_drop_chunk(int64_t chunk) {
    if (chunk < -1) return fail(WXPY_EINVAL, "chunk must be >= -1");
    g_reduce_drop.store(chunk);
    return WXPY_OK;
}

int wxpy_reduce_sum_levels(int levels) {
    if (levels < -1 || levels > 6) return fail(WXPY_EINVAL, "levels must be -1..6");
    g_reduce_sum_levels.store(levels);
    return WXPY_OK;
}

int wxpy_reduce_variant(int variant) {
    if (variant < -1 || variant >= kReduceVariants)
        return fail(WXPY_EINVAL, "variant must be -1..%d", kReduceVariants - 1);
    g_reduce_variant.store(variant);
    return WXPY_OK;
}

int wxpy_reduce_pipes(int mul_sixteenths) {
    if (mul_sixteenths < -1 || mul_sixteenths > 16)
        return fail(WXPY_EINVAL, "mul_sixteenths must be -1..16");
    g_reduce_mul.store(mul_sixteenths);
    return WXPY_OK;
}

}  // extern "C"
