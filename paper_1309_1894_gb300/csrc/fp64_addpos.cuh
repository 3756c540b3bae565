// fp64_addpos.cuh -- IEEE 754 binary64 addition of two non-negative values,
// round to nearest even, in the integer pipelines.  The operands of a squared
// 2-norm's summation tree are all squares, so every sum of that tree is of
// this kind; it needs about half the integer work of a general sum
// (fp64_emu.cuh), because two non-negative values never cancel.
//
// Method (the definition of a correctly rounded sum).  For non-negative
// binary64 values the bit patterns, read as unsigned integers, order like the
// values, so one integer comparison picks the larger operand a and the smaller
// b.  With exponent fields ea >= eb >= 1 (both normal), d = ea - eb and the
// 53-bit significands A, B (hidden bit included), the exact sum is
// (A + B / 2^d) ulp(a).  B >> d is added to A; the d bits shifted out of B,
// left-aligned in a 64-bit word R, hold the round bit (the top bit) and the
// sticky bits (the rest).  The sum S = A + (B >> d) is below 2^54; when it
// reaches 2^53 (c = 1) the significand is S >> 1, the round bit is bit 0 of S
// and all of R is sticky.  Round to nearest, ties to even, and assemble by
// adding the 53-bit significand, hidden bit included, to (ea + c - 1) << 52,
// so that a rounding carry to 2^53 lands in the exponent field by itself.
// With ea at most 0x7FD the sum stays finite (it can reach the top binade,
// exponent field 0x7FE, but not overflow).  For d >= 64 the clamp to
// 63 leaves B >> d = 0 and a sticky R with a zero round bit: the sum is a.
// A zero or subnormal smaller operand, a larger operand with exponent field
// 0x7FE or more (a possible overflow, infinity, NaN) or a set sign bit is
// flagged for the hardware instruction.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define WX_ADDPOS_FN __host__ __device__ __forceinline__
#else
#define WX_ADDPOS_FN inline
#endif

namespace wx {

// The fast path of RN(a + b) for non-negative a, b given as bit patterns:
// the result's bits, and `slow` set when the operands leave it (the bits are
// then meaningless).
WX_ADDPOS_FN uint64_t add_pos_core(uint64_t ua, uint64_t ub, bool &slow) {
    const bool swap = ub > ua;
    const uint64_t hi = swap ? ub : ua, lo = swap ? ua : ub;
    const uint32_t ea = (uint32_t)(hi >> 52), eb = (uint32_t)(lo >> 52);  // sign bit included
    slow |= (eb == 0u) | (ea >= 0x7FEu);
    uint32_t d = ea - eb;
    d = d > 63u ? 63u : d;
    const uint64_t frac = (1ull << 52) - 1, hidden = 1ull << 52;
    const uint64_t ma = (hi & frac) | hidden, mb = (lo & frac) | hidden;
    const uint64_t s = ma + (mb >> d);
    const uint64_t rem = d == 0u ? 0ull : mb << (64u - d);
    const uint32_t c = (uint32_t)(s >> 53);
    const uint32_t rnd = c ? (uint32_t)(s & 1u) : (uint32_t)(rem >> 63);
    const uint32_t sticky = c ? (uint32_t)(rem != 0) : (uint32_t)((rem << 1) != 0);
    const uint64_t m = s >> c;
    const uint64_t inc = rnd & (sticky | (uint32_t)(m & 1u));
    return ((uint64_t)(ea + c - 1u) << 52) + m + inc;
}

}  // namespace wx

#undef WX_ADDPOS_FN
