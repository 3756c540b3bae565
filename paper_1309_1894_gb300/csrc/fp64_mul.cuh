// fp64_mul.cuh -- IEEE 754 binary64 multiplication, round to nearest even,
// computed in the integer pipelines (the companion of fp64_emu.cuh's
// addition, for kernels with several products per element).
#pragma once

#include <cstdint>

// The cores (mul_coef_of, mul_rn_core, sqr_rn_core) also compile as plain
// host C++, so the host can check them against its own IEEE multiply.
#ifdef __CUDACC__
#define WX_MUL_FN __host__ __device__ __forceinline__
#else
#define WX_MUL_FN inline
#endif

namespace wx {

#ifdef __CUDACC__
static __device__ __noinline__ uint64_t mul_rn_hw_bits(uint64_t ua, uint64_t ub) {
    return (uint64_t)__double_as_longlong(
        __dmul_rn(__longlong_as_double((long long)ua), __longlong_as_double((long long)ub)));
}
#endif

// Bits sh .. sh + 31 of the 64-bit word hi:lo, 0 <= sh < 32.
WX_MUL_FN uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t sh) {
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, sh);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> sh);
#endif
}

// RN(a * b) in the integer pipelines (multiply-adds on the FMA pipeline,
// about thirty ALU operations) -- less than half the ALU cost of add_rn_bits,
// so a product is the cheaper operation to move off the FP64 pipeline.
//
// Method (the definition of a correctly rounded product).  For normal
// operands, split each 53-bit significand (hidden bit included) into a 21-bit
// high and a 32-bit low limb; four 32x32-bit products give the exact 106-bit
// product P = top 2^64 + w1 2^32 + w0, with P in [2^104, 2^106) and t = 1 when
// P >= 2^105.  The unrounded significand is P >> (52 + t), the round bit is
// bit 51 + t of P, and every bit below it is sticky; round to nearest, ties to
// even.  The biased exponent is ea + eb - 1023 + t.  The result is assembled
// by adding the 53-bit significand, hidden bit included, to
// sign | (exponent - 1) << 52, so a rounding carry to 2^53 lands in the
// exponent field by itself.  Operands that are zero, subnormal, infinite or
// NaN, and products whose exponent leaves [1, 0x7FD] (a subnormal, or a
// possible overflow), are flagged for the hardware instruction.

// One operand split once for many products (a coefficient: prepared on the
// host, read from the kernel's parameter space by every product).
struct MulCoef {
    uint32_t hi;  // high significand limb with the hidden bit (21 bits)
    uint32_t lo;  // low significand limb (32 bits)
    int32_t e;    // biased exponent - 1024; 2^20 when the operand is not normal
    uint32_t k;   // sign << 31 plus (biased exponent - 1024) << 20, modulo 2^32
};

WX_MUL_FN MulCoef mul_coef_of(uint64_t ua) {
    const uint32_t ah = (uint32_t)(ua >> 32);
    const uint32_t ea = (ah >> 20) & 0x7FFu;
    MulCoef c;
    c.hi = (ah & 0xFFFFFu) | 0x100000u;
    c.lo = (uint32_t)ua;
    c.e = ea - 1u >= 0x7FEu ? (1 << 20) : (int32_t)ea - 1024;
    c.k = (ah & 0x80000000u) + ((uint32_t)((int32_t)ea - 1024) << 20);
    return c;
}

// The fast path of RN(c * b): the result's bits, and `slow` set when the
// operands or the result leave it (the bits are then meaningless).
WX_MUL_FN uint64_t mul_rn_core(const MulCoef &c, uint64_t ub, bool &slow) {
    const uint32_t bh = (uint32_t)(ub >> 32), bl = (uint32_t)ub;
    const uint32_t eb = (bh >> 20) & 0x7FFu;
    const uint32_t b1 = (bh & 0xFFFFFu) | 0x100000u;
    const uint64_t p00 = (uint64_t)c.lo * bl;
    const uint64_t m1 = (uint64_t)c.hi * bl + (p00 >> 32);              // < 2^53 + 2^32
    const uint64_t m2 = (uint64_t)c.lo * b1 + (uint32_t)m1;             // < 2^53 + 2^32
    const uint64_t top = (uint64_t)c.hi * b1 + (m1 >> 32) + (m2 >> 32);  // P >> 64, < 2^42
    const uint32_t w0 = (uint32_t)p00, w1 = (uint32_t)m2;
    const uint32_t tl = (uint32_t)top, th = (uint32_t)(top >> 32);
    const uint32_t t = th >> 9;                     // bit 105 of P
    const uint32_t sh = 20 + t;                     // significand = (top:w1) >> sh
    const uint32_t m0l = funnel_r(w1, tl, sh);
    const uint32_t m0h = funnel_r(tl, th, sh);  // < 2^21, hidden bit at bit 20
    const uint32_t rnd = (w1 >> (sh - 1)) & 1u;
    const uint32_t stk = (w0 | (w1 << (33 - sh))) != 0u;
    const uint32_t inc = rnd & (stk | m0l);
    const int32_t ebase = c.e + (int32_t)(eb + t);  // result exponent - 1
    slow = slow || (eb - 1u >= 0x7FEu) || ((uint32_t)ebase >= 0x7FDu);
    // sign and exponent: the two signs add modulo 2 in bit 31
    const uint32_t hw = c.k + (bh & 0xFFF00000u) + (t << 20) + m0h;
    return (((uint64_t)hw << 32) | m0l) + inc;
}

// RN(a * a): the same method with both operands one value, so the split is
// taken once and the two cross products are one, doubled: P = A1^2 2^64 +
// 2 A1 A0 2^32 + A0^2 for the limbs A1 (21 bits, hidden bit included) and A0
// (32 bits).  The sign is always clear; the biased exponent is
// 2 ea - 1023 + t.  `slow` as in mul_rn_core.
WX_MUL_FN uint64_t sqr_rn_core(uint64_t ua, bool &slow) {
    const uint32_t ah = (uint32_t)(ua >> 32), a0 = (uint32_t)ua;
    const uint32_t ea = (ah >> 20) & 0x7FFu;
    const uint32_t a1 = (ah & 0xFFFFFu) | 0x100000u;
    const uint64_t p00 = (uint64_t)a0 * a0;
    const uint64_t x = (uint64_t)a1 * a0;                    // < 2^53
    const uint64_t m1 = (x << 1) + (p00 >> 32);              // < 2^54 + 2^32
    const uint64_t top = (uint64_t)a1 * a1 + (m1 >> 32);     // P >> 64, < 2^42
    const uint32_t w0 = (uint32_t)p00, w1 = (uint32_t)m1;
    const uint32_t tl = (uint32_t)top, th = (uint32_t)(top >> 32);
    const uint32_t t = th >> 9;
    const uint32_t sh = 20 + t;
    const uint32_t m0l = funnel_r(w1, tl, sh);
    const uint32_t m0h = funnel_r(tl, th, sh);
    const uint32_t rnd = (w1 >> (sh - 1)) & 1u;
    const uint32_t stk = (w0 | (w1 << (33 - sh))) != 0u;
    const uint32_t inc = rnd & (stk | m0l);
    const int32_t ebase = 2 * (int32_t)ea - 1024 + (int32_t)t;  // result exponent - 1
    slow = slow || (ea - 1u >= 0x7FEu) || ((uint32_t)ebase >= 0x7FDu);
    const uint32_t hw = ((uint32_t)ebase << 20) + m0h;
    return (((uint64_t)hw << 32) | m0l) + inc;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t sqr_rn_bits(uint64_t ua) {
    bool slow = false;
    uint64_t bits = sqr_rn_core(ua, slow);
    if (slow) bits = mul_rn_hw_bits(ua, ua);
    return bits;
}

// RN(a * b) on two bit patterns, the hardware instruction out of line for the
// cases the fast path leaves out.
__device__ __forceinline__ uint64_t mul_rn_bits(uint64_t ua, uint64_t ub) {
    bool slow = false;
    uint64_t bits = mul_rn_core(mul_coef_of(ua), ub, slow);
    if (slow) bits = mul_rn_hw_bits(ua, ub);
    return bits;
}

// Operands here are loaded data or kernel parameters, never the output of an
// FP64 instruction, so their bits are taken directly (no opaque move).
__device__ __forceinline__ double mul_rn_int(double a, double b) {
    return __longlong_as_double((long long)mul_rn_bits((uint64_t)__double_as_longlong(a),
                                                       (uint64_t)__double_as_longlong(b)));
}

#endif  // __CUDACC__

}  // namespace wx

#undef WX_MUL_FN
