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

// U(-1, 1) value of element i of the stream with key `key`: 2u - 1, exact.
__device__ __forceinline__ double uniform_pm1(uint64_t key, int64_t i) {
    const uint64_t b = mix64(key + (uint64_t)(i + 1) * kGolden);
    return __dadd_rn(-1.0, __dmul_rn(2.0, (double)(b >> 11) * 0x1.0p-53));
}

}  // namespace wx
