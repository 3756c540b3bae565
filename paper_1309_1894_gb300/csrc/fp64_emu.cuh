// fp64_emu.cuh -- IEEE 754 binary64 addition, round to nearest even, computed
// in the integer pipeline.
//
// Why.  w = RN(RN(alpha*x) + y) needs two FP64 instructions per element (the
// two roundings forbid a fused multiply-add), and on GB300 the FP64 pipeline
// issues only about two operations per clock per SM: a 256-bit streaming
// kernel doing DMUL+DADD reaches about 6.0 TB/s, the same kernel with one FP64
// instruction per element 7.2 TB/s.  The integer pipeline is nearly idle in
// this kernel, so part or all of the additions are moved there, which lifts the
// FP64 ceiling above the HBM one.
//
// Method (the definition of a correctly rounded sum, on integer significands).
// For two normal operands, order them by magnitude, |hi| >= |lo|.  Place hi's
// 53-bit significand (hidden bit included) at bits 62..10 of a 64-bit integer
// and lo's likewise, then shift lo's right by the exponent difference d; every
// bit shifted out is OR-ed into bit 0 (a "sticky" or jamming bit).  Add the
// two integers when the signs agree (renormalising a carry into bit 63 by one
// right shift, again jamming) or subtract them when they differ (an exact zero
// gives +0; otherwise shift the leading one back to bit 62).  Round at bit 10:
// up if the ten bits below are more than half, to even on exactly half.
// Correctness of the jamming bit: the bits below the rounding point are only
// approximated when bits were shifted out (d > 10); the approximation is then
// the floor or the ceiling of the exact value on a grid ten bits finer than
// the rounding point, with bit 0 set, so it is never the exact-half pattern and
// compares with one half exactly as the exact value does.  A subtraction with
// d >= 2 renormalises by at most one bit, so nine guard bits stay; with d <= 1
// nothing is shifted out and the result is exact before rounding.
// Operands that are zero, subnormal, infinite or NaN, and sums whose rounded
// result would be subnormal or overflow, take the hardware instruction
// (__dadd_rn) instead; for finite data in the normal range that never happens.
#pragma once

#include <cstdint>

#include "fp64_mul.cuh"

// The sum (add_rn_with) also compiles as plain host C++, so the host can
// check it against its own IEEE addition.
#ifdef __CUDACC__
#define WX_EMU_FN __device__ __forceinline__
#else
#define WX_EMU_FN inline
#endif

namespace wx {

// RN(a + b) on the bit patterns ua, ub of two binary64 values.  Operands and
// results the integer path leaves out go to hw(ua, ub): the hardware
// instruction, out of line, in the kernels (add_rn_bits below); the host's
// check of this function passes a recorder instead.
template <class Hw>
WX_EMU_FN uint64_t add_rn_with(uint64_t ua, uint64_t ub, Hw hw) {
    constexpr uint64_t kSign = 1ull << 63;
    constexpr uint64_t kAbs = kSign - 1;
    constexpr uint64_t kFrac = (1ull << 52) - 1;
    constexpr uint64_t kHidden = 1ull << 52;
    const bool a_big = (ua & kAbs) >= (ub & kAbs);
    const uint64_t hi = a_big ? ua : ub;
    const uint64_t lo = a_big ? ub : ua;
    const int ehi = (int)((hi >> 52) & 0x7FF);
    const int elo = (int)((lo >> 52) & 0x7FF);
    // Inf/NaN, zero or subnormal operands go to the hardware at the end.
    bool slow = ehi == 0x7FF || elo == 0;
    // Branch-free from here to the single fallback test: the lanes of a warp
    // follow one path whatever the signs and exponent gaps of their operands.
    // Every value stays an integer bit pattern until the one reinterpretation
    // at the end: merging several double-valued return paths made the
    // compiler issue FP64-pipeline instructions.
#ifdef __CUDA_ARCH__
    const int dd = min(ehi - elo, 63);  // a gap of 63 or more leaves only the sticky bit
#else
    const int dd = ehi - elo < 63 ? ehi - elo : 63;
#endif
    const uint64_t H = ((hi & kFrac) | kHidden) << 10;
    const uint64_t L0 = ((lo & kFrac) | kHidden) << 10;
    const uint64_t L = (L0 >> dd) | (uint64_t)((L0 & ((1ull << dd) - 1)) != 0);
    // H + L, or H - L (two's complement) when the signs differ
    const uint64_t neg = ((hi ^ lo) & kSign) ? ~0ull : 0ull;
    uint64_t S = H + (L ^ neg) - neg;
    const bool zero = S == 0;  // exact cancellation rounds to +0
    // Leading one back to bit 62: one right shift after a carry (lz == 0, with
    // the jam bit kept), or lz - 1 left shifts after a cancellation.
#ifdef __CUDA_ARCH__
    const int lz = __clzll((long long)S);
#else
    const int lz = S ? __builtin_clzll(S) : 64;
#endif
    const uint64_t right = (S >> 1) | (S & 1);
    const uint64_t left = S << ((lz - 1) & 63);
    S = lz == 0 ? right : left;
    int e = ehi + 1 - lz;
    // Round to nearest, ties to even, at bit 10.
    uint64_t m = S >> 10;
    const uint64_t rem = S & 0x3FF;
    m += (uint64_t)(rem > 0x200 || (rem == 0x200 && (m & 1)));
    const int carry = (int)(m >> 53);  // rounding reached the next binade
    m >>= carry;
    e += carry;
    slow = slow || (!zero && (e <= 0 || e >= 0x7FF));  // subnormal or overflowing result
    uint64_t bits = zero ? 0ull : ((hi & kSign) | ((uint64_t)e << 52) | (m & kFrac));
    if (slow) bits = hw(ua, ub);
    return bits;
}

#ifdef __CUDACC__

// The hardware sum for the rare operands the integer path leaves out, on bit
// patterns.  Kept out of line: an inlined fallback is if-converted by the
// compiler -- issued, predicated off, for every element -- and would occupy the
// FP64 pipeline the integer path exists to relieve; and its arguments and
// result are integers, since the moves that set up double-typed call
// arguments were issued for every element as well.
static __device__ __noinline__ uint64_t add_rn_hw_bits(uint64_t ua, uint64_t ub) {
    return (uint64_t)__double_as_longlong(
        __dadd_rn(__longlong_as_double((long long)ua), __longlong_as_double((long long)ub)));
}

// The bit pattern of a double through an opaque register move.  Handing the
// integer path a value the compiler still sees as a double (for instance the
// product just computed) let it rewrite integer operations on its bits into
// FP64-pipeline instructions.
__device__ __forceinline__ uint64_t opaque_bits(double v) {
    uint64_t b;
    asm volatile("mov.b64 %0, %1;" : "=l"(b) : "d"(v));
    return b;
}

struct AddRnHw {
    __device__ __forceinline__ uint64_t operator()(uint64_t ua, uint64_t ub) const {
        return add_rn_hw_bits(ua, ub);
    }
};

// RN(a + b) on the bit patterns ua, ub of two binary64 values.
__device__ __forceinline__ uint64_t add_rn_bits(uint64_t ua, uint64_t ub) {
    return add_rn_with(ua, ub, AddRnHw{});
}

__device__ __forceinline__ double add_rn_int(double a, double b) {
    return __longlong_as_double((long long)add_rn_bits(opaque_bits(a), opaque_bits(b)));
}

// w = RN(RN(alpha*x) + y) for VW elements; the sum of element k runs in the
// integer pipeline when EMU == 2, or when EMU == 1 and (base + k) is odd.
template <int VW, int EMU>
__device__ __forceinline__ void wxpy_vec_emu(double alpha, const double (&x)[VW],
                                             const double (&y)[VW], double (&w)[VW], int base) {
    static_assert(EMU >= 0 && EMU <= 2, "the product offload needs the coefficient split");
#pragma unroll
    for (int k = 0; k < VW; ++k) {
        const double p = __dmul_rn(alpha, x[k]);
        const bool emu = EMU == 2 || (EMU == 1 && ((base + k) & 1));
        w[k] = emu ? add_rn_int(p, y[k]) : __dadd_rn(p, y[k]);
    }
}

// The same with alpha's split `ca` at hand: EMU == 3 computes every product
// RN(alpha*x) in the integer pipelines (fp64_mul.cuh; operands it leaves out
// take the hardware multiply, out of line) and every sum on the FP64
// pipeline, which then carries one instruction per element.
template <int VW, int EMU>
__device__ __forceinline__ void wxpy_vec_emu(double alpha, const MulCoef &ca, const double (&x)[VW],
                                             const double (&y)[VW], double (&w)[VW], int base) {
    if constexpr (EMU == 3) {
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const uint64_t xb = (uint64_t)__double_as_longlong(x[k]);
            bool slow = false;
            uint64_t pb = mul_rn_core(ca, xb, slow);
            if (slow) pb = mul_rn_hw_bits((uint64_t)__double_as_longlong(alpha), xb);  // out of line
            w[k] = __dadd_rn(__longlong_as_double((long long)pb), y[k]);
        }
    } else {
        wxpy_vec_emu<VW, EMU>(alpha, x, y, w, base);
    }
}

#endif  // __CUDACC__

}  // namespace wx

#undef WX_EMU_FN
