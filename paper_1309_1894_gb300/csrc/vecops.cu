// vecops.cu -- the sibling vector kernels of VecWXPY in the same library:
// VecAXPBYPCZ, VecMAXPY and VecPointwiseMult as streaming kernels, and VecAXPY
// / VecAYPX as the in-place special cases of wxpy().
//
// Definitions (PETSc's, every product and sum rounded to nearest-even in
// binary64, left to right, no fused multiply-add):
//   axpy:      y = RN(RN(alpha*x) + y)                       = wxpy(alpha, x, y) into y
//   aypx:      y = RN(x + RN(alpha*y)) = RN(RN(alpha*y) + x) = wxpy(alpha, y, x) into y
//   axpbypcz:  z = RN(RN(RN(alpha*x) + RN(beta*y)) + RN(gamma*z))
//   maxpy:     y = RN(... RN(RN(y + RN(a0*x0)) + RN(a1*x1)) ... + RN(a_{m-1}*x_{m-1}))
//   pmult:     w = RN(x*y)
//
// One element-wise kernel template serves the three streaming operations: a
// grid-stride loop over 32-byte vectors when every pointer shares its offset
// modulo 32 bytes (the head peeled to that boundary and the tail finished
// with scalars), else over single elements.  A pass loads every input before
// it stores, so the output may be exactly one of the inputs.  On GB300 the
// FP64 pipeline is scarce (see fp64_emu.cuh): the sums can run in the integer
// pipeline (offload 1: every other one, 2: all), which these kernels need
// more than wxpy does -- axpbypcz has 3 products and 2 sums per element.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "internal.h"

namespace wx {
namespace {

constexpr int kMaxIn = 9;  // maxpy: y and up to 8 x vectors per launch

template <int NIN>
struct EwArgs {
    const double *in[NIN];
    double *out;
    int64_t n, head, nch;
    double coef[8];
};

template <int OFF>
__device__ __forceinline__ double add_sel(double a, double b, int position) {
    if constexpr (OFF == 2) return add_rn_int(a, b);
    else if constexpr (OFF == 1) return (position & 1) ? add_rn_int(a, b) : __dadd_rn(a, b);
    else return __dadd_rn(a, b);
}

template <int OFF>
struct AxpbypczOp {
    static constexpr int kIn = 3;  // x, y, z
    __device__ __forceinline__ static double apply(const double *c, const double (&e)[kIn]) {
        const double ax = __dmul_rn(c[0], e[0]);
        const double by = __dmul_rn(c[1], e[1]);
        const double cz = __dmul_rn(c[2], e[2]);
        const double s1 = add_sel<OFF>(ax, by, 1);
        return add_sel<OFF>(s1, cz, 0 + (OFF == 1 ? 0 : 1));
    }
};

template <int M, int OFF>
struct MaxpyOp {
    static constexpr int kIn = M + 1;  // y, x0 .. x_{M-1}
    __device__ __forceinline__ static double apply(const double *c, const double (&e)[kIn]) {
        double acc = e[0];
#pragma unroll
        for (int j = 0; j < M; ++j) acc = add_sel<OFF>(acc, __dmul_rn(c[j], e[j + 1]), j + 1);
        return acc;
    }
};

struct PmultOp {
    static constexpr int kIn = 2;
    __device__ __forceinline__ static double apply(const double *, const double (&e)[kIn]) {
        return __dmul_rn(e[0], e[1]);
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
    const double r[1] = {Op::apply(a.coef, e)};
    st_vec<1, 2>(a.out + i, r);
}

template <int VW, class Op>
__global__ void __launch_bounds__(256) ew_kernel(const EwArgs<Op::kIn> a) {
    constexpr int NIN = Op::kIn;
    constexpr int U = NIN <= 3 ? 2 : 1;
    const int64_t tpb = blockDim.x;
    const int64_t stride = (int64_t)gridDim.x * tpb * U;
    for (int64_t c0 = (int64_t)blockIdx.x * tpb * U + threadIdx.x; c0 < a.nch; c0 += stride) {
        double v[U][NIN][VW];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = c0 + u * tpb;
            if (c < a.nch) {
#pragma unroll
                for (int k = 0; k < NIN; ++k) ld_vec<VW, 2>(a.in[k] + a.head + c * VW, v[u][k]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = c0 + u * tpb;
            if (c < a.nch) {
                double r[VW];
#pragma unroll
                for (int q = 0; q < VW; ++q) {
                    double e[NIN];
#pragma unroll
                    for (int k = 0; k < NIN; ++k) e[k] = v[u][k][q];
                    r[q] = Op::apply(a.coef, e);
                }
                st_vec<VW, 2>(a.out + a.head + c * VW, r);
            }
        }
    }
    // head (< VW) and tail (< VW) elements by threads 0..7 of block 0
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        const int t = threadIdx.x;
        const int64_t body_end = a.head + a.nch * VW;
        if (t < 4 && t < a.head) ew_scalar<Op>(a, t);
        if (t >= 4 && body_end + (t - 4) < a.n) ew_scalar<Op>(a, body_end + (t - 4));
    }
}

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
              cudaStream_t s) {
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
    for (int k = 0; k < 8; ++k) a.coef[k] = k < ncoef ? coef[k] : 0.0;
    const bool vec4 = (diff & 31u) == 0;
    const int vw = vec4 ? 4 : 1;
    a.head = vec4 ? std::min<int64_t>((4 - (int64_t)(((uintptr_t)out >> 3) & 3)) & 3, n) : 0;
    a.nch = (n - a.head) / vw;
    constexpr int U = NIN <= 3 ? 2 : 1;
    const int64_t per_block = 256 * U;
    const int64_t grid = std::max<int64_t>(
        1, std::min<int64_t>((int64_t)dp->sm_count * 8, (a.nch + per_block - 1) / per_block));
    cudaError_t e = injected_launch_error();
    if (e == cudaSuccess) {
        if (vec4) ew_kernel<4, Op><<<(unsigned)grid, 256, 0, s>>>(a);
        else ew_kernel<1, Op><<<(unsigned)grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail_cuda(e, "vector kernel launch");
    return WXPY_OK;
}

std::atomic<int> g_vec_offload{2};

template <int M>
int maxpy_group(int64_t n, const double *alpha, const double *const *x, double *y, int off,
                cudaStream_t s) {
    const double *in[M + 1];
    in[0] = y;
    for (int j = 0; j < M; ++j) in[j + 1] = x[j];
    switch (off) {
        case 0: return launch_ew<MaxpyOp<M, 0>>(in, y, n, alpha, M, s);
        case 1: return launch_ew<MaxpyOp<M, 1>>(in, y, n, alpha, M, s);
        default: return launch_ew<MaxpyOp<M, 2>>(in, y, n, alpha, M, s);
    }
}

}  // namespace
}  // namespace wx

using namespace wx;

extern "C" {

int wxpy_axpy(int64_t n, double alpha, const double *x, double *y, void *stream) {
    return wxpy(n, alpha, x, y, y, stream);
}

int wxpy_aypx(int64_t n, double alpha, const double *x, double *y, void *stream) {
    return wxpy(n, alpha, y, x, y, stream);
}

int wxpy_axpbypcz(int64_t n, double alpha, double beta, double gamma, const double *x,
                  const double *y, double *z, void *stream) {
    const double *in[3] = {x, y, z};
    const double coef[3] = {alpha, beta, gamma};
    cudaStream_t s = (cudaStream_t)stream;
    switch (g_vec_offload.load()) {
        case 0: return launch_ew<AxpbypczOp<0>>(in, z, n, coef, 3, s);
        case 1: return launch_ew<AxpbypczOp<1>>(in, z, n, coef, 3, s);
        default: return launch_ew<AxpbypczOp<2>>(in, z, n, coef, 3, s);
    }
}

int wxpy_maxpy(int64_t n, int m, const double *alpha, const double *const *x, double *y,
               void *stream) {
    if (m < 0) return fail(WXPY_EINVAL, "negative m");
    if (m > 0 && (!alpha || !x)) return fail(WXPY_EINVAL, "null alpha or x array");
    if (m == 0 || n == 0) {
        const double *none[1] = {y};
        return validate(n, none, 1, y);
    }
    const int off = g_vec_offload.load();
    cudaStream_t s = (cudaStream_t)stream;
    // Groups of at most 8 terms, in order: y itself carries the rounded
    // partial sum from one group to the next, as the definition requires.
    for (int j0 = 0; j0 < m; j0 += 8) {
        const int g = std::min(8, m - j0);
        int st;
        switch (g) {
            case 1: st = maxpy_group<1>(n, alpha + j0, x + j0, y, off, s); break;
            case 2: st = maxpy_group<2>(n, alpha + j0, x + j0, y, off, s); break;
            case 3: st = maxpy_group<3>(n, alpha + j0, x + j0, y, off, s); break;
            case 4: st = maxpy_group<4>(n, alpha + j0, x + j0, y, off, s); break;
            case 5: st = maxpy_group<5>(n, alpha + j0, x + j0, y, off, s); break;
            case 6: st = maxpy_group<6>(n, alpha + j0, x + j0, y, off, s); break;
            case 7: st = maxpy_group<7>(n, alpha + j0, x + j0, y, off, s); break;
            default: st = maxpy_group<8>(n, alpha + j0, x + j0, y, off, s); break;
        }
        if (st != WXPY_OK) return st;
    }
    return WXPY_OK;
}

int wxpy_pointwise_mult(int64_t n, const double *x, const double *y, double *w, void *stream) {
    const double *in[2] = {x, y};
    return launch_ew<PmultOp>(in, w, n, nullptr, 0, (cudaStream_t)stream);
}

int wxpy_vecops_offload(int offload) {
    if (offload < 0 || offload > 2) return fail(WXPY_EINVAL, "offload must be 0, 1 or 2");
    g_vec_offload.store(offload);
    return WXPY_OK;
}

}  // extern "C"
