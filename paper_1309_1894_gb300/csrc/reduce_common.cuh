// reduce_common.cuh -- what the fused reductions' kernel forms share: the
// tile of the fixed summation tree, the argument block, the per-element
// arithmetic (w = RN(RN(alpha*x) + y) of paper Sec. 3, Fig. 1, then the
// term RN(w*w) or RN(w*z)), the integer-pipeline tree sum of non-negative
// values, the 32-byte accesses, and the last block's sum of the tile sums.
// Included by reduce.cu (register-loaded and staged forms) and
// reduce_warp.cu (warp-tiled form); everything is internal to each.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fp64_addpos.cuh"
#include "fp64_emu.cuh"
#include "fp64_mul.cuh"
#include "internal.h"

namespace wx {

constexpr int kTile = 8192;
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
    int64_t drop_chunk;  // staged path: the producer stops before this chunk (-1: never)
};

// The warp-tiled form (reduce_warp.cu): launches the kernel of `shape`
// (0: two rows per load group, five blocks of 128 threads per SM; 1: four
// rows, four blocks; 2: four rows, three blocks) for kind 0 (norm2, `suml`
// leading tree levels 0..6 in the integer pipelines) or 1 (dot, suml 0) on
// 32-byte co-aligned pointers.
cudaError_t launch_reduce_warp(int kind, int suml, int shape, const ReduceArgs &a,
                               const DeviceProps *dp, cudaStream_t s);

namespace {

__device__ __forceinline__ uint64_t bits_of(double v) { return (uint64_t)__double_as_longlong(v); }
__device__ __forceinline__ double double_of(uint64_t b) { return __longlong_as_double((long long)b); }

static __device__ __noinline__ uint64_t add_rn_hw_bits(uint64_t ua, uint64_t ub) {
    return bits_of(__dadd_rn(double_of(ua), double_of(ub)));
}

// RN(a + b) of two sums of squares (non-negative): the integer-pipeline sum
// when INT, else the FP64 instruction.
template <bool INT>
__device__ __forceinline__ double tree_add(double a, double b) {
    if constexpr (INT) {
        const uint64_t ua = opaque_bits(a), ub = opaque_bits(b);
        bool slow = false;
        uint64_t r = add_pos_core(ua, ub, slow);
        if (slow) r = add_rn_hw_bits(ua, ub);  // out of line
        return double_of(r);
    } else {
        return __dadd_rn(a, b);
    }
}

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
        const uint64_t tb = KIND == 0 ? sqr_rn_bits(wb) : mul_rn_bits(wb, bits_of(z));
        t = double_of(tb);
    } else {
        w = __dadd_rn(__dmul_rn(a.alpha, x), y);
        t = __dmul_rn(w, KIND == 0 ? w : z);
    }
}


// Coherent evict-first 32-byte accesses: w may be one of the inputs.
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

// Terms of the four elements base .. base + 3; w stored.  VEC: one 32-byte
// co-aligned vector of every operand; else element by element with bounds,
// +0 terms past n.
template <int KIND, bool EMU, bool VEC>
__device__ __forceinline__ void vector_terms(const ReduceArgs &a, int64_t base, double (&t)[4]) {
    if constexpr (VEC) {
        double x[4], y[4], z[4], w[4];
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

// The last block to finish (after every tile sum of this grid is written)
// sums the tile sums.  All threads of the block take part.
__device__ __forceinline__ void finish_grid(const ReduceArgs &a, bool &last) {
    __syncthreads();
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

}  // namespace
}  // namespace wx
