// gen.cuh -- the splitmix64 output function, shared by the device-side input
// generators (gen.cu, server.cu).  See gen.cu for the stream convention.
#pragma once

#include <cstdint>

namespace wx {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Key of stream (seed, tag): output number `tag` of the generator at `seed`.
__host__ __device__ __forceinline__ uint64_t stream_key_of(uint64_t seed, uint32_t tag) {
    return mix64(seed + ((uint64_t)tag + 1) * kGolden);
}

// U(-1, 1) value of element i of the stream with key `key`: 2u - 1 with
// u = (b >> 11) * 2^-53, exact.  The value is m * 2^-53 for the even integer
// m = 2k - 2^53 (k = b >> 11), so its binary64 encoding is assembled from m
// with integer operations only: on GB300 the FP64 pipe is the scarce one
// (a conversion, a multiply and an add per value would use it three times).
// More generally, for a range of width 2^(s+1) centred on zero, the value
// lo + width*u = m * 2^(s-53); `uniform_sym(key, i, s)` assembles that.
// Every path stays an integer bit pattern until one opaque move into a double
// register at the end.  Seen through, the sign bit OR-ed into the assembled
// pattern was compiled as an FP64 negation (measured: one DADD per value).
__device__ __forceinline__ double uniform_sym(uint64_t key, int64_t i, int s) {
    const uint64_t b = mix64(key + (uint64_t)(i + 1) * kGolden);
    const int64_t m = (int64_t)((b >> 11) << 1) - ((int64_t)1 << 53);  // [-2^53, 2^53), even
    const uint64_t sign = m < 0 ? (1ull << 63) : 0ull;
    const uint64_t a = (uint64_t)(m < 0 ? -m : m);  // 0 or [2, 2^53]
    const int p = 63 - __clzll((long long)(a | 1));  // a = 1.f * 2^p, p in [1, 53] (a > 0)
    const uint64_t frac = (p <= 52 ? (a << (52 - p)) : (a >> (p - 52))) & ((1ull << 52) - 1);
    const uint64_t expo = (uint64_t)(p - 53 + s + 1023);
    const uint64_t bits = m == 0 ? 0ull : (sign | (expo << 52) | frac);
    double v;
    asm("mov.b64 %0, %1;" : "=d"(v) : "l"(bits));
    return v;
}

__device__ __forceinline__ double uniform_pm1(uint64_t key, int64_t i) {
    return uniform_sym(key, i, 0);
}

}  // namespace wx
