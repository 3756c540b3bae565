// gen.cu -- device-side seeded inputs and the bitwise comparison used by the tuner.
//
// The generator is splitmix64 (Steele, Lea & Flood, OOPSLA 2014), written here
// from its published definition and used in counter form: output k of the
// generator seeded with s is mix64(s + (k+1)*0x9E3779B97F4A7C15).  A stream
// (seed, tag) is keyed by output number `tag` of the generator seeded with
// `seed`; element i of the stream is output number i of the generator seeded
// with that key.  A double u = (bits >> 11) * 2^-53 is uniform on [0, 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gen.cuh"
#include "internal.h"

namespace wx {

uint64_t stream_key(uint64_t seed, uint32_t tag) { return stream_key_of(seed, tag); }

// dst[i] = lo + width * u(start + i).  lo + width*u is computed as two
// correctly rounded operations; for the ranges the library uses (width a power
// of two, lo = -width/2) every step is exact.
__global__ void fill_uniform_kernel(double *dst, int64_t n, uint64_t key, int64_t start,
                                    double lo, double width) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t b = mix64(key + (uint64_t)(start + i + 1) * kGolden);
        const double u = (double)(b >> 11) * 0x1.0p-53;
        dst[i] = __dadd_rn(lo, __dmul_rn(width, u));
    }
}

// The same values for a range (-2^s, 2^s), assembled with integer operations
// only (see uniform_sym): no FP64 instruction per element.
__global__ void fill_symmetric_kernel(double *dst, int64_t n, uint64_t key, int64_t start, int s) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = uniform_sym(key, start + i, s);
}

// count += number of i with bits(a[i]) != bits(b[i]).
__global__ void count_mismatch_kernel(const uint64_t *a, const uint64_t *b, int64_t n,
                                      unsigned long long *count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        local += (a[i] != b[i]) ? 1ull : 0ull;
    for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// Reads `n` words and folds them into *sink: evicts the L2 between timed runs
// without leaving dirty lines behind.
__global__ void l2_flush_kernel(const uint64_t *buf, int64_t n, uint64_t *sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint64_t acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        acc ^= buf[i];
    if (acc == 0x5eedf00d5eedf00dull) *sink = acc;  // practically never; keeps the loads
}

int launch_fill_uniform(double *dst, int64_t n, uint64_t seed, uint32_t tag, int64_t start,
                        double lo, double hi, cudaStream_t s) {
    if (n == 0) return WXPY_OK;
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)dp->sm_count * 8);
    cudaError_t e = injected_launch_error();
    if (e == cudaSuccess) {
        // (-2^s, 2^s) with a small s: the integer-only path gives the same bits.
        int sym = -1;
        for (int k = 0; k < 8; ++k)
            if (lo == -std::ldexp(1.0, k) && hi == std::ldexp(1.0, k)) sym = k;
        if (sym >= 0)
            fill_symmetric_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, stream_key(seed, tag),
                                                                   start, sym);
        else
            fill_uniform_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, stream_key(seed, tag),
                                                                 start, lo, hi - lo);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail_cuda(e, "fill kernel launch");
    return WXPY_OK;
}

int launch_count_mismatch(const double *a, const double *b, int64_t n,
                          unsigned long long *count_dev, cudaStream_t s) {
    if (n == 0) return WXPY_OK;
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)dp->sm_count * 4);
    count_mismatch_kernel<<<(unsigned)blocks, 256, 0, s>>>((const uint64_t *)a,
                                                          (const uint64_t *)b, n, count_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "compare kernel launch");
    return WXPY_OK;
}

int launch_l2_flush(const void *buf, int64_t bytes, void *sink, cudaStream_t s) {
    int st = WXPY_OK;
    const DeviceProps *dp = current_device(&st);
    if (!dp) return st;
    l2_flush_kernel<<<(unsigned)dp->sm_count * 4, 512, 0, s>>>((const uint64_t *)buf, bytes / 8,
                                                              (uint64_t *)sink);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, "l2 flush launch");
    return WXPY_OK;
}

__global__ void device_delay_kernel(long long cycles) {
    const long long t0 = clock64();
    while (clock64() - t0 < cycles) __nanosleep(500);
}

void launch_device_delay(long long cycles, cudaStream_t s) {
    device_delay_kernel<<<1, 1, 0, s>>>(cycles);
}

}  // namespace wx

using namespace wx;

extern "C" int wxpy_fill_uniform(int64_t n, uint64_t seed, uint32_t tag, int64_t start, double lo,
                                 double hi, double *dst, void *stream) {
    if (n < 0 || start < 0) return fail(WXPY_EINVAL, "negative n or start");
    if (n > 0 && (!dst || ((uintptr_t)dst & 7u))) return fail(WXPY_EINVAL, "bad destination");
    if (!(hi > lo)) return fail(WXPY_EINVAL, "need hi > lo");
    return launch_fill_uniform(dst, n, seed, tag, start, lo, hi, (cudaStream_t)stream);
}
