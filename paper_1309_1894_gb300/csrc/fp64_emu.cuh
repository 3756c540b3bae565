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

namespace wx {

__device__ __forceinline__ double add_rn_int(double a, double b) {
    constexpr uint64_t kSign = 1ull << 63;
    constexpr uint64_t kAbs = kSign - 1;
    constexpr uint64_t kFrac = (1ull << 52) - 1;
    constexpr uint64_t kHidden = 1ull << 52;
    const uint64_t ua = (uint64_t)__double_as_longlong(a);
    const uint64_t ub = (uint64_t)__double_as_longlong(b);
    const bool a_big = (ua & kAbs) >= (ub & kAbs);
    const uint64_t hi = a_big ? ua : ub;
    const uint64_t lo = a_big ? ub : ua;
    const int ehi = (int)((hi >> 52) & 0x7FF);
    const int elo = (int)((lo >> 52) & 0x7FF);
    if (ehi == 0x7FF || elo == 0) return __dadd_rn(a, b);  // inf/NaN, zero or subnormal
    const int d = ehi - elo;
    const uint64_t H = ((hi & kFrac) | kHidden) << 10;
    uint64_t L = ((lo & kFrac) | kHidden) << 10;
    if (d >= 64) L = 1;
    else if (d > 0) L = (L >> d) | (uint64_t)((L << (64 - d)) != 0);
    int e = ehi;
    uint64_t S;
    if (((hi ^ lo) & kSign) == 0) {
        S = H + L;
        if (S >> 63) {
            S = (S >> 1) | (S & 1);
            ++e;
        }
    } else {
        S = H - L;
        if (S == 0) return 0.0;  // exact cancellation rounds to +0
        const int lz = __clzll((long long)S) - 1;
        S <<= lz;
        e -= lz;
    }
    uint64_t m = S >> 10;
    const uint64_t rem = S & 0x3FF;
    if (rem > 0x200 || (rem == 0x200 && (m & 1))) ++m;
    if (m >> 53) {
        m >>= 1;
        ++e;
    }
    if (e <= 0 || e >= 0x7FF) return __dadd_rn(a, b);  // subnormal or overflowing result
    return __longlong_as_double((long long)((hi & kSign) | ((uint64_t)e << 52) | (m & kFrac)));
}

// w = RN(RN(alpha*x) + y) for VW elements; the sum of element k runs in the
// integer pipeline when EMU == 2, or when EMU == 1 and (base + k) is odd.
template <int VW, int EMU>
__device__ __forceinline__ void wxpy_vec_emu(double alpha, const double (&x)[VW],
                                             const double (&y)[VW], double (&w)[VW], int base) {
#pragma unroll
    for (int k = 0; k < VW; ++k) {
        const double p = __dmul_rn(alpha, x[k]);
        const bool emu = EMU == 2 || (EMU == 1 && ((base + k) & 1));
        w[k] = emu ? add_rn_int(p, y[k]) : __dadd_rn(p, y[k]);
    }
}

}  // namespace wx
