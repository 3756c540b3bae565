// seg_tile.cuh -- one warp computes one tile of a segmented launch.
//
// A tile is a contiguous range of one problem w = RN(RN(alpha*x) + y) (paper
// Sec. 3, Fig. 1 vecwxpy).  When x, y and w share their offset modulo 32
// bytes, the warp peels the head to the 32-byte boundary, streams 256-bit
// vectors with up to kTileMaxU vectors of x and of y per lane in flight (the
// tile's unroll U decides how many), and finishes the tail; otherwise it uses
// coalesced 8-byte accesses.  Loads and stores are evict-first (.cs) and
// coherent, so in-place problems (w == x or w == y) are safe.
//
// One fixed-size body whose unroll is a run-time predicate serves every tile:
// a separately compiled body per (width, unroll) behind a run-time switch made
// the compiler spill registers.
#pragma once

#include "single_kernel.cuh"

namespace wx {

constexpr int kTileMaxU = 4;

__device__ __forceinline__ void tile_scalar(const double *x, const double *y, double *w,
                                            double alpha, int64_t e) {
    double xv[1], yv[1], wv[1];
    ld_vec<1, 2>(x + e, xv);
    ld_vec<1, 2>(y + e, yv);
    wxpy_vec<1>(alpha, xv, yv, wv);
    st_vec<1, 2>(w + e, wv);
}

// EMU: which operations run in the integer pipelines (fp64_emu.cuh): 0 none,
// 1 the sums of the odd positions of every 32-byte vector, 3 every product
// (with alpha's split ca).
template <int EMU>
__device__ __forceinline__ void tile_body4(const double *x, const double *y, double *w,
                                           double alpha, const MulCoef &ca, int64_t nch, int lane,
                                           int U) {
    const int64_t step = 32 * U;
    for (int64_t c0 = lane; c0 < nch; c0 += step) {
        double xv[kTileMaxU][4], yv[kTileMaxU][4], wv[kTileMaxU][4];
#pragma unroll
        for (int u = 0; u < kTileMaxU; ++u) {
            const int64_t c = c0 + 32 * u;
            if (u < U && c < nch) {
                ld_vec<4, 2>(x + c * 4, xv[u]);
                ld_vec<4, 2>(y + c * 4, yv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kTileMaxU; ++u) {
            const int64_t c = c0 + 32 * u;
            if (u < U && c < nch) {
                wxpy_vec_emu<4, EMU>(alpha, ca, xv[u], yv[u], wv[u], 0);
                st_vec<4, 2>(w + c * 4, wv[u]);
            }
        }
    }
}

// The whole tile [x, x+len) by the calling warp (lane = thread index mod 32).
template <int EMU>
__device__ __forceinline__ void tile_wxpy(const double *x, const double *y, double *w,
                                          double alpha, int64_t len, int lane, int U) {
    MulCoef ca{};
    if constexpr (EMU == 3) ca = mul_coef_of((uint64_t)__double_as_longlong(alpha));
    const uintptr_t ax = (uintptr_t)x, ay = (uintptr_t)y, aw = (uintptr_t)w;
    if ((((ax ^ aw) | (ay ^ aw)) & 31u) == 0) {
        const int64_t head = min(len, (int64_t)((4 - (int)((aw >> 3) & 3)) & 3));
        const int64_t nch = (len - head) / 4;
        const int64_t body_end = head + nch * 4;
        if (lane < head) tile_scalar(x, y, w, alpha, lane);
        if (lane >= 4 && body_end + (lane - 4) < len)
            tile_scalar(x, y, w, alpha, body_end + (lane - 4));
        tile_body4<EMU>(x + head, y + head, w + head, alpha, ca, nch, lane, U);
    } else {
        for (int64_t e = lane; e < len; e += 32) tile_scalar(x, y, w, alpha, e);
    }
}

}  // namespace wx
