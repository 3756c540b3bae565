// vecops.cu -- the sibling vector kernels of VecWXPY in the same library:
// VecAXPBYPCZ, VecMAXPY and VecPointwiseMult as streaming kernels, and VecAXPY
// / VecAYPX as the in-place special cases of wxpy().
//
// Definitions (PETSc's, every product and sum rounded to nearest-even in
// binary64, left to right, no fused multiply-add):
//   axpy:      y = RN(RN(alpha*x) + y)                       = wxpy(alpha, x, y) into y
//   aypx:      y = RN(x + RN(alpha*y)) = RN(RN(alpha*y) + x) = wxpy(alpha, y, x) into y
//   axpby:     y = RN(RN(alpha*x) + RN(beta*y))
//   axpbypcz:  z = RN(RN(RN(alpha*x) + RN(beta*y)) + RN(gamma*z))
//   maxpy:     y = RN(... RN(RN(y + RN(a0*x0)) + RN(a1*x1)) ... + RN(a_{m-1}*x_{m-1}))
//   pmult:     w = RN(x*y)
//
// One element-wise kernel template serves the three streaming operations: a
// grid-stride loop over 32-byte vectors when every pointer shares its offset
// modulo 32 bytes (the head peeled to that boundary and the tail finished
// with scalars), else over single elements.  A pass loads every input before
// it stores, so the output may be exactly one of the inputs.
//
// Pipe balance.  On GB300 the FP64 pipeline issues about two operations per
// clock per SM, and these kernels need more of it than wxpy does: axpbypcz
// has 3 products and 2 sums per element (32 bytes of traffic), maxpy with m
// terms 2m operations per 8(m + 2) bytes.  Both are FP64-bound far below the
// HBM roofline unless part of the arithmetic moves to the integer pipelines
// (fp64_emu.cuh, fp64_mul.cuh).  A product costs about thirty ALU operations
// there and a sum about seventy-five, so products are the cheaper ones to
// move: a runtime fraction (in sixteenths) of each warp's loop iterations
// computes all of its products in the integer pipeline, the rest in FP64;
// the choice is uniform across the warp (no divergence) and rotates with the
// iteration, so every SM sub-partition sees the same mix.  Sums can move too
// (add offload 1: every other one, 2: all).  Every split gives the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "bulk.cuh"
#include "fp64_mul.cuh"
#include "internal.h"

namespace wx {
namespace {

// Coefficients of one launch: as doubles for the FP64 instructions and split
// once on the host for the integer-pipeline products.
struct Coefs {
    double d[8];
    MulCoef m[8];
};

template <int NIN>
struct EwArgs {
    const double *in[NIN];
    double *out;
    int64_t n, head, nch;  // nch: 4-element chunks (32-byte path) or elements after `head`
    int pm;                // sixteenths of warp iterations whose products run in the integer pipeline
    int64_t drop_tile;     // debug: the producer stops before this tile (-1: never)
    Coefs cf;
};

template <int OFF>
__device__ __forceinline__ double add_sel(double a, double b, int position) {
    if constexpr (OFF == 2) return add_rn_int(a, b);
    else if constexpr (OFF == 1) return (position & 1) ? add_rn_int(a, b) : __dadd_rn(a, b);
    else return __dadd_rn(a, b);
}

__device__ __forceinline__ uint64_t bits_of(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ double double_of(uint64_t b) { return __longlong_as_double((long long)b); }

// p[j] = RN(c_j * e[F + j]), j < K, F = NIN - K (the data operands follow any
// others).  PM = 1: integer-pipeline products, one out-of-line fallback to the
// hardware instruction for the whole element when any of them leaves the
// fast path.
template <int PM, int K, int NIN>
__device__ __forceinline__ void products(const Coefs &c, const double (&e)[NIN], double (&p)[K]) {
    constexpr int F = NIN - K;
    if constexpr (PM == 0) {
#pragma unroll
        for (int j = 0; j < K; ++j) p[j] = __dmul_rn(c.d[j], e[F + j]);
    } else {
        bool slow = false;
        uint64_t b[K];
#pragma unroll
        for (int j = 0; j < K; ++j) b[j] = mul_rn_core(c.m[j], bits_of(e[F + j]), slow);
        if (slow) {
#pragma unroll
            for (int j = 0; j < K; ++j) b[j] = mul_rn_hw_bits(bits_of(c.d[j]), bits_of(e[F + j]));
        }
#pragma unroll
        for (int j = 0; j < K; ++j) p[j] = double_of(b[j]);
    }
}

// The fast path of the integer-pipeline products alone: p[j] as in
// products<1>, with `slow` set when any of them left the fast path (its
// bits are then meaningless and the caller recomputes the element).
template <int K, int NIN>
__device__ __forceinline__ void products_fast(const Coefs &c, const double (&e)[NIN], double (&p)[K],
                                              bool &slow) {
    constexpr int F = NIN - K;
#pragma unroll
    for (int j = 0; j < K; ++j) p[j] = double_of(mul_rn_core(c.m[j], bits_of(e[F + j]), slow));
}

template <int OFF>
struct AxpbyOp {
    static constexpr int kIn = 2;  // x, y
    static constexpr bool kStaged = true;
    template <int PM>
    __device__ __forceinline__ static double apply(const Coefs &c, const double (&e)[kIn]) {
        double p[2];
        products<PM>(c, e, p);
        return add_sel<OFF>(p[0], p[1], 1);
    }
    __device__ __forceinline__ static double apply_fast(const Coefs &c, const double (&e)[kIn],
                                                        bool &slow) {
        double p[2];
        products_fast(c, e, p, slow);
        return add_sel<OFF>(p[0], p[1], 1);
    }
};

template <int OFF>
struct AxpbypczOp {
    static constexpr int kIn = 3;  // x, y, z
    static constexpr bool kStaged = true;
    template <int PM>
    __device__ __forceinline__ static double apply(const Coefs &c, const double (&e)[kIn]) {
        double p[3];
        products<PM>(c, e, p);
        const double s1 = add_sel<OFF>(p[0], p[1], 1);
        return add_sel<OFF>(s1, p[2], OFF == 1 ? 0 : 1);
    }
    __device__ __forceinline__ static double apply_fast(const Coefs &c, const double (&e)[kIn],
                                                        bool &slow) {
        double p[3];
        products_fast(c, e, p, slow);
        const double s1 = add_sel<OFF>(p[0], p[1], 1);
        return add_sel<OFF>(s1, p[2], OFF == 1 ? 0 : 1);
    }
};

template <int M, int OFF>
struct MaxpyOp {
    static constexpr int kIn = M + 1;  // y, x0 .. x_{M-1}
    static constexpr bool kStaged = true;
    template <int PM>
    __device__ __forceinline__ static double apply(const Coefs &c, const double (&e)[kIn]) {
        double p[M];
        products<PM>(c, e, p);
        double acc = e[0];
#pragma unroll
        for (int j = 0; j < M; ++j) acc = add_sel<OFF>(acc, p[j], j + 1);
        return acc;
    }
    __device__ __forceinline__ static double apply_fast(const Coefs &c, const double (&e)[kIn],
                                                        bool &slow) {
        double p[M];
        products_fast(c, e, p, slow);
        double acc = e[0];
#pragma unroll
        for (int j = 0; j < M; ++j) acc = add_sel<OFF>(acc, p[j], j + 1);
        return acc;
    }
};

struct PmultOp {
    static constexpr int kIn = 2;
    static constexpr bool kStaged = false;
    template <int PM>
    __device__ __forceinline__ static double apply(const Coefs &, const double (&e)[kIn]) {
        if constexpr (PM == 1) return double_of(mul_rn_bits(bits_of(e[0]), bits_of(e[1])));
        else return __dmul_rn(e[0], e[1]);
    }
};

template <class Op>
__device__ __forceinline__ void ew_scalar(const EwArgs<Op::kIn> &a, int64_t i) {
    double e[Op::kIn];
#pragma unroll
    for (int k = 0; k < Op::kIn; ++k) {
        double v[1];
        ld_vec<1, 2>(a.in[k] + i, v);
        e[k] = v[0];
    }
    const double r[1] = {Op::template apply<0>(a.cf, e)};
    st_vec<1, 2>(a.out + i, r);
}

// ---- element path: pointers not sharing their offset modulo 32 bytes --------

template <class Op, int PM>
__device__ __forceinline__ void elem_iter(const EwArgs<Op::kIn> &a, int64_t i0, int64_t tpb) {
    constexpr int NIN = Op::kIn, U = NIN <= 3 ? 4 : (NIN <= 5 ? 2 : 1);
    double v[U][NIN];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + u * tpb;
        if (i < a.n) {
#pragma unroll
            for (int k = 0; k < NIN; ++k) {
                double t[1];
                ld_vec<1, 2>(a.in[k] + i, t);
                v[u][k] = t[0];
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + u * tpb;
        if (i < a.n) {
            const double r[1] = {Op::template apply<PM>(a.cf, v[u])};
            st_vec<1, 2>(a.out + i, r);
        }
    }
}

template <class Op>
__global__ void __launch_bounds__(256) ew_elem_kernel(const EwArgs<Op::kIn> a) {
    constexpr int U = Op::kIn <= 3 ? 4 : (Op::kIn <= 5 ? 2 : 1);  // as elem_iter
    const int64_t tpb = blockDim.x;
    const int64_t stride = (int64_t)gridDim.x * tpb * U;
    // Warp-uniform rotation through 16 slots; slots below a.pm take the
    // integer-pipeline products.
    unsigned slot = ((threadIdx.x >> 5) * 5u + blockIdx.x * 3u) & 15u;
    for (int64_t i0 = (int64_t)blockIdx.x * tpb * U + threadIdx.x; i0 < a.n; i0 += stride) {
        if ((int)slot < a.pm) elem_iter<Op, 1>(a, i0, tpb);
        else elem_iter<Op, 0>(a, i0, tpb);
        slot = (slot + 1u) & 15u;
    }
}

// ---- direct path: 32-byte register loads, for operations light on arithmetic
// (pointwise_mult: one product per 24 bytes), where a shared-memory ring only
// adds hand-off latency.

template <class Op, int PM>
__device__ __forceinline__ void direct_iter(const EwArgs<Op::kIn> &a, int64_t c0, int64_t tpb) {
    constexpr int NIN = Op::kIn, U = 2;
    double v[U][NIN][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + u * tpb;
        if (c < a.nch) {
#pragma unroll
            for (int k = 0; k < NIN; ++k) ld_vec<4, 2>(a.in[k] + a.head + c * 4, v[u][k]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + u * tpb;
        if (c < a.nch) {
            double r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double e[NIN];
#pragma unroll
                for (int k = 0; k < NIN; ++k) e[k] = v[u][k][q];
                r[q] = Op::template apply<PM>(a.cf, e);
            }
            st_vec<4, 2>(a.out + a.head + c * 4, r);
        }
    }
}

template <class Op>
__global__ void __launch_bounds__(256) ew_direct_kernel(const EwArgs<Op::kIn> a) {
    const int64_t tpb = blockDim.x;
    const int64_t stride = (int64_t)gridDim.x * tpb * 2;
    unsigned slot = ((threadIdx.x >> 5) * 5u + blockIdx.x * 3u) & 15u;
    for (int64_t c0 = (int64_t)blockIdx.x * tpb * 2 + threadIdx.x; c0 < a.nch; c0 += stride) {
        if ((int)slot < a.pm) direct_iter<Op, 1>(a, c0, tpb);
        else direct_iter<Op, 0>(a, c0, tpb);
        slot = (slot + 1u) & 15u;
    }
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        const int t = threadIdx.x;
        const int64_t body_end = a.head + a.nch * 4;
        if (t < 4 && t < a.head) ew_scalar<Op>(a, t);
        if (t >= 4 && body_end + (t - 4) < a.n) ew_scalar<Op>(a, body_end + (t - 4));
    }
}

// ---- staged path: bulk copies into a shared-memory ring ----------------------
//
// Eight consumer warps and one producer warp per block; the grid is persistent
// (tiles blockIdx.x, blockIdx.x + gridDim.x, ...).  A tile is TE = 256 * EPT
// elements of every input; the ring holds S tiles.  The producer's lane 0
// waits until all eight consumer warps have released a stage ("empty"
// barrier, one arrival per warp), then issues one bulk copy per input into it
// ("full" barrier, completed by the copies' bytes).  A consumer thread takes
// element pairs 2c, 2c + 512, ... of the tile from shared memory, computes
// them in registers and writes them straight to global memory (16-byte
// stores, coalesced per warp).  Loads never wait on compute: up to S - 1
// tiles are in flight while one is computed, and no register holds a loaded
// vector before its turn.  Each warp picks its product pipe per tile by the
// rotation of ew_elem_kernel; a warp that is ahead runs into the next stage
// without waiting for the others.  Output aliasing: a tile's inputs are in
// shared memory before any of its outputs is written, and no other tile
// touches its addresses, so the output may be one of the inputs.

constexpr int kConsumerWarps = 8;
constexpr int kStagedThreads = 32 * (kConsumerWarps + 1);

// Bitmask of the waits that ran out in this device's kernels (1: producer,
// 2: consumer); read and cleared by wxpy_vecops_status().
__device__ unsigned int g_vec_fault;

template <int NIN>
struct StageShape {
    static constexpr int kEpt = NIN <= 3 ? 4 : 2;  // elements per consumer thread per tile
    static constexpr int kTile = 256 * kEpt;
    static constexpr int kTileBytes = NIN * kTile * 8;
    static constexpr int kStages = std::max(2, std::min(4, (72 * 1024) / kTileBytes));
    static constexpr int kSmem = kStages * kTileBytes;
    // three resident blocks for the widest maxpy groups (a register cap of 75
    // measured 6 % faster there; narrower operations gain nothing from it)
    static constexpr int kMinBlocks = NIN >= 7 ? 3 : 2;
};

__device__ __forceinline__ void ld_shared_v2(const double *p, double &a, double &b) {
    asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(a), "=d"(b) : "r"(smem_addr(p)));
}

__device__ __forceinline__ void st_global_v2_cs(double *p, double a, double b) {
    asm volatile("st.global.cs.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(a), "d"(b) : "memory");
}

// This thread's elements of a tile, every product in FP64 (PM 0), from the
// stage, which is still held; d: the launch's coefficients.  Out of line: it
// runs only when an integer-pipeline product left its fast path, and inlined
// it would be issued, predicated off, on the FP64 pipeline for every tile.
template <class Op, int TE>
__device__ __noinline__ void staged_tile_fp64(double d0, double d1, double d2, double d3,
                                              double d4, double d5, double d6, double d7,
                                              const double *sb, double *out, int len, int c) {
    constexpr int NIN = Op::kIn;
    Coefs cf;  // the FP64 products read only the doubles
    cf.d[0] = d0, cf.d[1] = d1, cf.d[2] = d2, cf.d[3] = d3;
    cf.d[4] = d4, cf.d[5] = d5, cf.d[6] = d6, cf.d[7] = d7;
    for (int j = 0; j < TE / 512; ++j) {
        const int p = 2 * c + 512 * j;
        if (p < len) {
            double v[NIN][2];
#pragma unroll
            for (int k = 0; k < NIN; ++k) ld_shared_v2(sb + k * TE + p, v[k][0], v[k][1]);
            double r[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                double e[NIN];
#pragma unroll
                for (int k = 0; k < NIN; ++k) e[k] = v[k][q];
                r[q] = Op::template apply<0>(cf, e);
            }
            st_global_v2_cs(out + p, r[0], r[1]);
        }
    }
}

// PM = 1: the integer-pipeline products take their fast path with no test
// between them and the sums, so the tile's arithmetic is one straight run
// that the compiler can interleave (one element's FP64 sums with another's
// integer products); if any product left the fast path, the thread's
// elements are recomputed in FP64 and written again (nothing reads them
// before the kernel ends, and the stage still holds the inputs).
template <class Op, int PM, int TE>
__device__ __forceinline__ void staged_tile(const Coefs &cf, const double *sb, double *out, int len,
                                            int c) {
    constexpr int NIN = Op::kIn;
    bool slow = false;
#pragma unroll
    for (int j = 0; j < TE / 512; ++j) {
        const int p = 2 * c + 512 * j;
        if (p < len) {
            double v[NIN][2];
#pragma unroll
            for (int k = 0; k < NIN; ++k) ld_shared_v2(sb + k * TE + p, v[k][0], v[k][1]);
            double r[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                double e[NIN];
#pragma unroll
                for (int k = 0; k < NIN; ++k) e[k] = v[k][q];
                if constexpr (PM == 1) r[q] = Op::apply_fast(cf, e, slow);
                else r[q] = Op::template apply<0>(cf, e);
            }
            st_global_v2_cs(out + p, r[0], r[1]);
        }
    }
    if constexpr (PM == 1) {
        if (slow)
            staged_tile_fp64<Op, TE>(cf.d[0], cf.d[1], cf.d[2], cf.d[3], cf.d[4], cf.d[5], cf.d[6],
                                     cf.d[7], sb, out, len, c);
    }
}

template <class Op>
__global__ void __launch_bounds__(kStagedThreads, StageShape<Op::kIn>::kMinBlocks)
    ew_staged_kernel(const EwArgs<Op::kIn> a) {
    constexpr int NIN = Op::kIn;
    using SS = StageShape<NIN>;
    constexpr int TE = SS::kTile, S = SS::kStages;
    extern __shared__ __align__(128) double ring[];  // [S][NIN][TE]
    __shared__ __align__(8) uint64_t full[S], empty[S];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t body = a.nch * 4;  // elements from a.head, a multiple of 4
    const int64_t ntiles = (body + TE - 1) / TE;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), kConsumerWarps);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (warp == kConsumerWarps) {
        if (lane == 0) {
            const uint64_t policy = evict_first_policy();
            bool ok = true;
            int i = 0;
            for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
                if (t == a.drop_tile) break;
                const int s = i % S;
                if (i >= S && !mbar_wait(smem_addr(&empty[s]), ((i / S) - 1) & 1)) {
                    ok = false;
                    break;
                }
                const int64_t e0 = t * TE;
                const uint32_t len = (uint32_t)(body - e0 < TE ? body - e0 : TE);
                const uint32_t bar = smem_addr(&full[s]);
                mbar_arrive_expect_tx(bar, len * 8u * NIN);
#pragma unroll
                for (int k = 0; k < NIN; ++k)
                    bulk_load(smem_addr(ring + ((size_t)s * NIN + k) * TE), a.in[k] + a.head + e0,
                              len * 8u, bar, policy);
            }
            // Every issued copy lands before the block exits (the earlier
            // ones were consumed before their stage was reused).
            for (int j = i > S ? i - S : 0; j < i; ++j)
                if (!mbar_wait(smem_addr(&full[j % S]), (j / S) & 1)) ok = false;
            if (!ok) atomicOr(&g_vec_fault, 1u);
        }
    } else {
        unsigned slot = (warp * 5u + blockIdx.x * 3u) & 15u;
        int i = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int s = i % S;
            if (!mbar_wait(smem_addr(&full[s]), (i / S) & 1)) {
                if (lane == 0) atomicOr(&g_vec_fault, 2u);
                break;
            }
            const int64_t e0 = t * TE;
            const int len = (int)(body - e0 < TE ? body - e0 : TE);
            const double *sb = ring + (size_t)s * NIN * TE;
            double *out = a.out + a.head + e0;
            if ((int)slot < a.pm) staged_tile<Op, 1, TE>(a.cf, sb, out, len, threadIdx.x);
            else staged_tile<Op, 0, TE>(a.cf, sb, out, len, threadIdx.x);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
            slot = (slot + 1u) & 15u;
        }
        // head (< 4) and tail (< 4) elements by threads 0..7 of block 0
        if (blockIdx.x == 0 && threadIdx.x < 8) {
            const int t = threadIdx.x;
            const int64_t body_end = a.head + body;
            if (t < 4 && t < a.head) ew_scalar<Op>(a, t);
            if (t >= 4 && body_end + (t - 4) < a.n) ew_scalar<Op>(a, body_end + (t - 4));
        }
    }
}

// Per device: the dynamic shared-memory opt-in done and the resident blocks
// per SM of one staged kernel.
template <class Op>
int staged_blocks_per_sm(int device) {
    static std::atomic<int> cached[64];
    if (device < 0 || device >= 64) return 0;
    int v = cached[device].load(std::memory_order_relaxed);
    if (v > 0) return v;
    constexpr int smem = StageShape<Op::kIn>::kSmem;
    if (cudaFuncSetAttribute(ew_staged_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ew_staged_kernel<Op>, kStagedThreads,
                                                      smem) != cudaSuccess || nb < 1)
        return 0;
    cached[device].store(nb, std::memory_order_relaxed);
    return nb;
}

std::atomic<long long> g_drop_tile{-1};

// Validation shared by the three streaming operations: n >= 0, 8-byte aligned
// non-null pointers, and the output either disjoint from or exactly equal to
// each input.
int validate(int64_t n, const double *const *in, int nin, const double *out) {
    if (n < 0) return fail(WXPY_EINVAL, "n = %lld is negative", (long long)n);
    if (n == 0) return WXPY_OK;
    if (n > ((int64_t)1 << 56)) return fail(WXPY_EINVAL, "n too large");
    const uint64_t bytes = (uint64_t)n * 8;
    const uintptr_t po = (uintptr_t)out;
    if (!out || (po & 7)) return fail(WXPY_EINVAL, "null or misaligned output");
    for (int k = 0; k < nin; ++k) {
        const uintptr_t p = (uintptr_t)in[k];
        if (!in[k] || (p & 7)) return fail(WXPY_EINVAL, "null or misaligned input %d", k);
        if (p != po && p < po + bytes && po < p + bytes)
            return fail(WXPY_EOVERLAP, "output partially overlaps input %d", k);
    }
    return WXPY_OK;
}

template <class Op>
int launch_ew(const double *const *in, double *out, int64_t n, const double *coef, int ncoef,
              int pm, cudaStream_t s) {
    constexpr int NIN = Op::kIn;
    int st = validate(n, in, NIN, out);
    if (st != WXPY_OK || n == 0) return st;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    EwArgs<NIN> a;
    uintptr_t diff = 0;
    for (int k = 0; k < NIN; ++k) {
        a.in[k] = in[k];
        diff |= (uintptr_t)in[k] ^ (uintptr_t)out;
    }
    a.out = out;
    a.n = n;
    a.pm = pm;
    a.drop_tile = g_drop_tile.load();
    for (int k = 0; k < 8; ++k) {
        a.cf.d[k] = k < ncoef ? coef[k] : 0.0;
        uint64_t b;
        std::memcpy(&b, &a.cf.d[k], 8);
        a.cf.m[k] = mul_coef_of(b);
    }
    cudaError_t e = injected_launch_error();
    if (e == cudaSuccess && (diff & 31u) == 0) {
        // 32-byte co-aligned: peel the head to the boundary, stage the body
        a.head = std::min<int64_t>((4 - (int64_t)(((uintptr_t)out >> 3) & 3)) & 3, n);
        a.nch = (n - a.head) / 4;
        if constexpr (Op::kStaged) {
            const int nb = staged_blocks_per_sm<Op>(dp->device);
            if (nb == 0) return fail_cuda(cudaGetLastError(), "staged kernel set-up");
            constexpr int TE = StageShape<NIN>::kTile;
            const int64_t tiles = (a.nch * 4 + TE - 1) / TE;
            const int64_t grid =
                std::max<int64_t>(1, std::min<int64_t>((int64_t)dp->sm_count * nb, tiles));
            ew_staged_kernel<Op><<<(unsigned)grid, kStagedThreads, StageShape<NIN>::kSmem, s>>>(a);
        } else {
            const int64_t per_block = 256 * 2;
            const int64_t grid = std::max<int64_t>(
                1, std::min<int64_t>((int64_t)dp->sm_count * 8, (a.nch + per_block - 1) / per_block));
            ew_direct_kernel<Op><<<(unsigned)grid, 256, 0, s>>>(a);
        }
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        a.head = 0;
        a.nch = n;
        const int64_t per_block = 256 * 4;
        const int64_t grid = std::max<int64_t>(
            1, std::min<int64_t>((int64_t)dp->sm_count * 8, (n + per_block - 1) / per_block));
        ew_elem_kernel<Op><<<(unsigned)grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail_cuda(e, "vector kernel launch");
    return WXPY_OK;
}

// Pipe split: add offload (0, 1, 2) and product sixteenths (0..16); -1 in
// either leaves the operation's searched split, else its default (below).
std::atomic<int> g_vec_add{-1};
std::atomic<int> g_vec_mul{-1};
std::atomic<int> g_vec_tuned[WXPY_VEC_CLASSES] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1};

using Pipes = VecPipes;

Pipes pipes_for(int cls) {
    Pipes p = vecops_default(cls);
    vecops_tuned_load(cls, &p);
    const int add = g_vec_add.load(), mul = g_vec_mul.load();
    if (add >= 0) p.add = add;
    if (mul >= 0) p.mul = mul;
    return p;
}

template <int M>
int maxpy_group(int64_t n, const double *alpha, const double *const *in, Pipes p, cudaStream_t s) {
    switch (p.add) {
        case 0: return launch_ew<MaxpyOp<M, 0>>(in, (double *)in[0], n, alpha, M, p.mul, s);
        case 1: return launch_ew<MaxpyOp<M, 1>>(in, (double *)in[0], n, alpha, M, p.mul, s);
        default: return launch_ew<MaxpyOp<M, 2>>(in, (double *)in[0], n, alpha, M, p.mul, s);
    }
}

}  // namespace

// Defaults, measured on GB300 at n = 2^26 (sums in FP64, the cheaper pipe for
// them; the product share that balanced the FP64 and ALU pipelines best).
VecPipes vecops_default(int cls) {
    if (cls == WXPY_VEC_AXPBYPCZ) return {0, 14};
    if (cls == WXPY_VEC_AXPBY) return {0, 10};
    if (cls == WXPY_VEC_PMULT) return {0, 4};
    return {0, cls + 1 == 2 ? 14 : 16};  // maxpy with cls + 1 terms
}

int vecops_inputs(int cls) {
    if (cls == WXPY_VEC_AXPBYPCZ) return 3;
    if (cls == WXPY_VEC_PMULT || cls == WXPY_VEC_AXPBY) return 2;
    return cls + 2;  // y and cls + 1 x vectors
}

bool vecops_tuned_load(int cls, VecPipes *p) {
    if (cls < 0 || cls >= WXPY_VEC_CLASSES) return false;
    const int v = g_vec_tuned[cls].load();
    if (v < 0) return false;
    p->add = v >> 5;
    p->mul = v & 31;
    return true;
}

void vecops_tuned_store(int cls, const VecPipes *p) {
    if (cls < 0 || cls >= WXPY_VEC_CLASSES) return;
    g_vec_tuned[cls].store(p ? (p->add << 5) | p->mul : -1);
}

int vecops_run(int cls, int64_t n, const double *coef, const double *const *in, double *out,
               VecPipes p, cudaStream_t s) {
    switch (cls) {
        case WXPY_VEC_AXPBYPCZ:
            switch (p.add) {
                case 0: return launch_ew<AxpbypczOp<0>>(in, out, n, coef, 3, p.mul, s);
                case 1: return launch_ew<AxpbypczOp<1>>(in, out, n, coef, 3, p.mul, s);
                default: return launch_ew<AxpbypczOp<2>>(in, out, n, coef, 3, p.mul, s);
            }
        case WXPY_VEC_PMULT: return launch_ew<PmultOp>(in, out, n, nullptr, 0, p.mul, s);
        case WXPY_VEC_AXPBY:
            switch (p.add) {
                case 0: return launch_ew<AxpbyOp<0>>(in, out, n, coef, 2, p.mul, s);
                default: return launch_ew<AxpbyOp<2>>(in, out, n, coef, 2, p.mul, s);
            }
        case 1: return maxpy_group<2>(n, coef, in, p, s);
        case 2: return maxpy_group<3>(n, coef, in, p, s);
        case 3: return maxpy_group<4>(n, coef, in, p, s);
        case 4: return maxpy_group<5>(n, coef, in, p, s);
        case 5: return maxpy_group<6>(n, coef, in, p, s);
        case 6: return maxpy_group<7>(n, coef, in, p, s);
        case 7: return maxpy_group<8>(n, coef, in, p, s);
        default: return fail(WXPY_EINVAL, "bad vector kernel class %d", cls);
    }
}

}  // namespace wx

using namespace wx;

extern "C" {

int wxpy_axpy(int64_t n, double alpha, const double *x, double *y, void *stream) {
    return wxpy(n, alpha, x, y, y, stream);
}

int wxpy_aypx(int64_t n, double alpha, const double *x, double *y, void *stream) {
    return wxpy(n, alpha, y, x, y, stream);
}

int wxpy_axpby(int64_t n, double alpha, double beta, const double *x, double *y, void *stream) {
    const double *in[2] = {x, y};
    const double coef[2] = {alpha, beta};
    return vecops_run(WXPY_VEC_AXPBY, n, coef, in, y, pipes_for(WXPY_VEC_AXPBY),
                      (cudaStream_t)stream);
}

int wxpy_axpbypcz(int64_t n, double alpha, double beta, double gamma, const double *x,
                  const double *y, double *z, void *stream) {
    const double *in[3] = {x, y, z};
    const double coef[3] = {alpha, beta, gamma};
    return vecops_run(WXPY_VEC_AXPBYPCZ, n, coef, in, z, pipes_for(WXPY_VEC_AXPBYPCZ),
                      (cudaStream_t)stream);
}

int wxpy_maxpy(int64_t n, int m, const double *alpha, const double *const *x, double *y,
               void *stream) {
    if (m < 0) return fail(WXPY_EINVAL, "negative m");
    if (m > 0 && (!alpha || !x)) return fail(WXPY_EINVAL, "null alpha or x array");
    if (m == 0 || n == 0) {
        const double *none[1] = {y};
        return validate(n, none, 1, y);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Groups of at most 8 terms, in order: y itself carries the rounded
    // partial sum from one group to the next, as the definition requires.
    for (int j0 = 0; j0 < m; j0 += 8) {
        const int g = std::min(8, m - j0);
        int st;
        if (g == 1) {
            // a single term is y = RN(y + RN(a x)) = RN(RN(a x) + y): wxpy into y
            st = wxpy(n, alpha[j0], x[j0], y, y, stream);
        } else {
            const double *in[9];
            in[0] = y;
            for (int j = 0; j < g; ++j) in[j + 1] = x[j0 + j];
            st = vecops_run(g - 1, n, alpha + j0, in, y, pipes_for(g - 1), s);
        }
        if (st != WXPY_OK) return st;
    }
    return WXPY_OK;
}

int wxpy_pointwise_mult(int64_t n, const double *x, const double *y, double *w, void *stream) {
    const double *in[2] = {x, y};
    return vecops_run(WXPY_VEC_PMULT, n, nullptr, in, w, pipes_for(WXPY_VEC_PMULT),
                      (cudaStream_t)stream);
}

int wxpy_vecops_pipes(int add_offload, int mul_sixteenths) {
    if (add_offload < -1 || add_offload > 2)
        return fail(WXPY_EINVAL, "add offload must be -1, 0, 1 or 2");
    if (mul_sixteenths < -1 || mul_sixteenths > 16)
        return fail(WXPY_EINVAL, "product sixteenths must be in -1..16");
    g_vec_add.store(add_offload);
    g_vec_mul.store(mul_sixteenths);
    return WXPY_OK;
}

int wxpy_vecops_status(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned int fault = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&fault, g_vec_fault, sizeof(fault));
    const unsigned int zero = 0;
    if (e == cudaSuccess && fault) e = cudaMemcpyToSymbol(g_vec_fault, &zero, sizeof(zero));
    if (e != cudaSuccess) return fail_cuda(e, "vector kernel status");
    if (fault)
        return fail(WXPY_ETIMEOUT, "a staged vector kernel's bounded wait ran out (%s)",
                    fault & 1u ? (fault & 2u ? "producer and consumers" : "producer") : "consumers");
    return WXPY_OK;
}

int wxpy_debug_vecops_drop_tile(int64_t tile) {
    if (tile < -1) return fail(WXPY_EINVAL, "tile must be >= -1");
    g_drop_tile.store(tile);
    return WXPY_OK;
}

}  // extern "C"
