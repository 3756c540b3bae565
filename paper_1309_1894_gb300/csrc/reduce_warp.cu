// reduce_warp.cu -- the warp-tiled form of the fused reductions (wxpy_norm2,
// wxpy_dot; reduction variants 4..6): the update of paper Sec. 3, Fig. 1
// (w = RN(RN(alpha*x) + y)) and the terms RN(w*w) or RN(w*z), summed by the
// same fixed tree as the other forms (tiles of 8192 indices, the halving tree
// inside a tile, then over the tile sums), so every form gives the same bits.
//
// One warp sums a whole tile, so a tile needs no shared memory and no block
// barrier.  Lane l takes the 32-byte vectors at 128 r + 4 l of the tile (rows
// r = 0..63, each row 1 KB of every operand, read by the warp at once):
// element i = 128 r + 4 l + q has bits 12..7 = r, 6..2 = l and 1..0 = q.  The
// halving tree reduces bits from the top down: the six levels of bits 12..7
// run inside the thread, bits 6..2 by warp shuffles, bits 1..0 in lane 0.
//
// Inside the thread the rows are visited in sixteen groups (k, j = 0..3):
// group (k, j) holds the rows rho + {0, 32, 16, 48}, rho = 4 rev2(j) + rev2(k)
// (rev2 swaps the two bits of its argument).  Rows rho and rho + 32 differ in
// bit 12, rho and rho + 16 in bit 11, so the group value (e[rho] + e[rho + 32])
// + (e[rho + 16] + e[rho + 48]) is the tree over bits 12 and 11.  The four
// groups of one k differ in bits 10 (j's bit 0) and 9 (j's bit 1), so
// (g0 + g1) + (g2 + g3), in j order, is the tree over those two; the four
// results of k = 0..3 differ in bits 8 and 7 and combine the same way.  Each
// combination keeps its operands in a shift through registers, so the loops
// over j and k stay rolled: the unrolled body is one group, sixteen elements
// per lane, whose loads (two or four rows of every input) are all issued
// before its arithmetic.
//
// Pipes as in the other forms: a share of the tiles (mul_sixteenths, rotated
// over warps and tiles) computes both products in the integer pipelines, and
// for norm2 the first SUML (0..6) tree levels -- every level inside the
// thread, 8064 of a tile's 8191 sums when SUML = 6 -- may run as the integer
// sum of non-negative values (fp64_addpos.cuh).  The last, ragged tile is
// read element by element with FP64 products, +0 terms past n.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "internal.h"
#include "reduce_common.cuh"

namespace wx {
namespace {

constexpr int kWarpThreads = 128;
constexpr int kWarpsPerBlock = kWarpThreads / 32;

// Row offset h of a group: 0, 32, 16, 48.
__device__ __forceinline__ constexpr int group_row(int h) { return ((h & 1) << 5) | ((h & 2) << 3); }

// The terms of one group (rows rho + {0, 32, 16, 48}; `base` = the element of
// row rho for this lane), w stored, and the group value (bits 12 and 11).
// VEC: full tile, LR rows of every input loaded before their arithmetic; else
// element by element with bounds.
template <int KIND, bool EMU, bool VEC, int SUML, int LR>
__device__ __forceinline__ void warp_group(const ReduceArgs &a, int64_t base, double (&g)[4]) {
    static_assert(LR == 2 || LR == 4, "rows loaded together: 2 or 4");
    double e[4][4];
    if constexpr (VEC) {
#pragma unroll
        for (int h = 0; h < 4; h += LR) {
            double x[LR][4], y[LR][4], z[KIND == 1 ? LR : 1][4], w[LR][4];
#pragma unroll
            for (int u = 0; u < LR; ++u) {
                const int64_t b = base + 128 * group_row(h + u);
                ld4(a.x + b, x[u]);
                ld4(a.y + b, y[u]);
                if constexpr (KIND == 1) ld4(a.z + b, z[u]);
            }
#pragma unroll
            for (int u = 0; u < LR; ++u) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    element<KIND, EMU>(a, x[u][q], y[u][q], KIND == 1 ? z[u][q] : 0.0, w[u][q],
                                       e[h + u][q]);
                st4(a.w + base + 128 * group_row(h + u), w[u]);
            }
        }
    } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) vector_terms<KIND, EMU, false>(a, base + 128 * group_row(h), e[h]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        g[q] = tree_add<(SUML >= 2)>(tree_add<(SUML >= 1)>(e[0][q], e[1][q]),
                                     tree_add<(SUML >= 1)>(e[2][q], e[3][q]));
}

// (v0 + v1) + (v2 + v3) elementwise: two tree levels, the first at level L.
template <int SUML, int L>
__device__ __forceinline__ void two_levels(const double (&v0)[4], const double (&v1)[4],
                                           const double (&v2)[4], const double (&v3)[4],
                                           double (&out)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        out[q] = tree_add<(SUML >= L + 1)>(tree_add<(SUML >= L)>(v0[q], v1[q]),
                                           tree_add<(SUML >= L)>(v2[q], v3[q]));
}

__device__ __forceinline__ void shift_in(double (&s0)[4], double (&s1)[4], double (&s2)[4],
                                         double (&s3)[4], const double (&v)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        s0[q] = s1[q];
        s1[q] = s2[q];
        s2[q] = s3[q];
        s3[q] = v[q];
    }
}

// The sum of tile `tile` by one warp; valid in lane 0.
template <int KIND, bool EMU, bool VEC, int SUML, int LR>
__device__ double warp_tile_sum(const ReduceArgs &a, int64_t tile, int lane) {
    static_assert(SUML == 0 || KIND == 0, "integer tree sums need non-negative terms");
    const int64_t t0 = tile * kTile + 4 * lane;
    double k0[4] = {}, k1[4] = {}, k2[4] = {}, k3[4] = {};  // shift over k
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        const int rk = ((k & 1) << 1) | (k >> 1);
        double j0[4] = {}, j1[4] = {}, j2[4] = {}, j3[4] = {};  // shift over j
#pragma unroll 1
        for (int j = 0; j < 4; ++j) {
            const int rj = ((j & 1) << 1) | (j >> 1);
            double g[4];
            warp_group<KIND, EMU, VEC, SUML, LR>(a, t0 + 128 * (4 * rj + rk), g);
            shift_in(j0, j1, j2, j3, g);
        }
        double v[4];
        two_levels<SUML, 3>(j0, j1, j2, j3, v);  // bits 10, 9
        shift_in(k0, k1, k2, k3, v);
    }
    double v[4];
    two_levels<SUML, 5>(k0, k1, k2, k3, v);  // bits 8, 7
    // bits 6..2: lanes L and L + 16, 8, 4, 2, 1
#pragma unroll
    for (int sh = 16; sh >= 1; sh >>= 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(v[q], __shfl_down_sync(0xffffffffu, v[q], sh));
    }
    // bits 1..0 in lane 0: q and q + 2, then q and q + 1
    return __dadd_rn(__dadd_rn(v[0], v[2]), __dadd_rn(v[1], v[3]));
}

template <int KIND, int SUML, int LR, int MINB>
__global__ void __launch_bounds__(kWarpThreads, MINB) wxpy_reduce_warp_kernel(const ReduceArgs a) {
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * kWarpsPerBlock;
    const int64_t gw = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t full = a.n / kTile;  // tiles with every element present
    unsigned slot = (unsigned)(gw * 7) & 15u;  // warp-uniform rotation of the pipe choice
    for (int64_t tile = gw; tile < a.ntiles; tile += warps) {
        double s;
        if (tile >= full) s = warp_tile_sum<KIND, false, false, 0, LR>(a, tile, lane);
        else if ((int)slot < a.mul_sixteenths) s = warp_tile_sum<KIND, true, true, SUML, LR>(a, tile, lane);
        else s = warp_tile_sum<KIND, false, true, SUML, LR>(a, tile, lane);
        if (lane == 0) {
            a.partial[tile] = s;
            __threadfence();
        }
        slot = (slot + 1u) & 15u;
    }
    finish_grid(a, last);
}

template <int KIND, int SUML, int LR, int MINB>
cudaError_t launch_warp(const ReduceArgs &a, const DeviceProps *dp, cudaStream_t s) {
    static std::atomic<int> cached[64];
    const int dev = dp->device;
    int nb = dev >= 0 && dev < 64 ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (nb <= 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, wxpy_reduce_warp_kernel<KIND, SUML, LR, MINB>, kWarpThreads, 0);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        if (dev >= 0 && dev < 64) cached[dev].store(nb, std::memory_order_relaxed);
    }
    const int64_t need = (a.ntiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)dp->sm_count * nb, need));
    wxpy_reduce_warp_kernel<KIND, SUML, LR, MINB><<<(unsigned)grid, kWarpThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KIND, int SUML>
cudaError_t launch_shape(int shape, const ReduceArgs &a, const DeviceProps *dp, cudaStream_t s) {
    switch (shape) {
        case 0: return launch_warp<KIND, SUML, 2, 5>(a, dp, s);
        case 1: return launch_warp<KIND, SUML, 4, 4>(a, dp, s);
        default: return launch_warp<KIND, SUML, 4, 3>(a, dp, s);
    }
}

}  // namespace

cudaError_t launch_reduce_warp(int kind, int suml, int shape, const ReduceArgs &a,
                               const DeviceProps *dp, cudaStream_t s) {
    if (kind == 1) return launch_shape<1, 0>(shape, a, dp, s);
    switch (suml) {
        case 0: return launch_shape<0, 0>(shape, a, dp, s);
        case 1: return launch_shape<0, 1>(shape, a, dp, s);
        case 2: return launch_shape<0, 2>(shape, a, dp, s);
        case 3: return launch_shape<0, 3>(shape, a, dp, s);
        case 4: return launch_shape<0, 4>(shape, a, dp, s);
        case 5: return launch_shape<0, 5>(shape, a, dp, s);
        default: return launch_shape<0, 6>(shape, a, dp, s);
    }
}

}  // namespace wx
