// mixed_kernel.cuh -- the single-call VecWXPY kernel for pointers whose
// offsets disagree modulo 32 bytes (the mixed-alignment classes).
//
// When x, y and w do not share their offset modulo 32 bytes, no single vector
// width fits all three.  This kernel aligns on w: the head is peeled until w
// reaches a 32-byte boundary, w is stored as 32-byte vectors (4 elements, one
// "chunk"), and each input is loaded for the same chunk at the widest width
// its own offset relative to w allows:
//   KX, KY = 4  the input shares w's offset mod 32: one 32-byte load;
//          = 2  it is 16 bytes off: two 16-byte loads;
//          = 1  it is 8 or 24 bytes off: four 8-byte loads of one 32-byte span.
// The narrower loads of an input never written by the call (classification
// rejects partial overlap, so an input offset from w is disjoint from it) go
// through the non-coherent path with L1 allocation: the first 8-byte load of a
// lane brings the sector into L1 and the three after it hit there, so DRAM sees
// each byte once.  The 32-byte loads and the stores follow CACHE as in the
// single-call family (1: ld.global.nc.L1::no_allocate + st.global.cs; 2:
// coherent evict-first, used under aliasing).  XY: x == y (then KX == KY) is
// loaded once.  The grid either covers the chunks in one pass or strides over
// them (a run-time loop); U chunks per thread per pass, all loads of a pass
// before its stores.
//
// Arithmetic as in the family (paper Sec. 3, Fig. 1, vecwxpy read as PETSc
// VecWXPY): w = RN(RN(alpha*x) + y), never fused; EMU = 1 moves the sums of
// odd element positions to the integer pipeline (fp64_emu.cuh), EMU = 3 every
// product (fp64_mul.cuh).
#pragma once

#include "single_kernel.cuh"

namespace wx {

// One chunk (4 elements) of an input at width K (see above).
template <int K, int CACHE>
__device__ __forceinline__ void ld_chunk(const double *p, double (&r)[4]) {
    if constexpr (K == 4) {
        ld_vec<4, CACHE>(p, r);
    } else if constexpr (K == 2) {
        asm volatile("ld.global.nc.v2.f64 {%0,%1}, [%2];" : "=d"(r[0]), "=d"(r[1]) : "l"(p));
        asm volatile("ld.global.nc.v2.f64 {%0,%1}, [%2];" : "=d"(r[2]), "=d"(r[3]) : "l"(p + 2));
    } else {
        static_assert(K == 1, "K must be 4, 2 or 1");
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(r[k]) : "l"(p + k));
    }
}

template <int KX, int KY, int U, int CACHE, bool XY, int EMU>
__device__ __forceinline__ void mixed_pass(const SingleArgs &a, int64_t c0, int64_t tpb) {
    const double *xb = a.x + a.head;
    const double *yb = a.y + a.head;
    double *wb = a.w + a.head;
    double xv[U][4], yv[U][4], wv[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + u * tpb;
        if (c < a.nchunks) {
            ld_chunk<KX, CACHE>(xb + 4 * c, xv[u]);
            if constexpr (!XY) ld_chunk<KY, CACHE>(yb + 4 * c, yv[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + u * tpb;
        if (c < a.nchunks) {
            if constexpr (XY) wxpy_vec_emu<4, EMU>(a.alpha, a.ca, xv[u], xv[u], wv[u], 0);
            else wxpy_vec_emu<4, EMU>(a.alpha, a.ca, xv[u], yv[u], wv[u], 0);
            st_vec<4, CACHE>(wb + 4 * c, wv[u]);
        }
    }
}

template <int KX, int KY, int U, int CACHE, bool XY, int EMU>
__global__ void __launch_bounds__(max_threads<4, U, 1, XY, EMU>())
    wxpy_mixed_kernel(const SingleArgs a) {
    // the chunks of this thread's first pass, prefetched into L2 before the
    // wait as in the family's kernel (single_kernel.cuh)
    prefetch_first_pass<4, U, XY>(a, (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x, blockDim.x);
    pdl_enter();
    const int64_t tpb = blockDim.x;
    const int64_t stride = (int64_t)gridDim.x * tpb * U;
    for (int64_t c0 = (int64_t)blockIdx.x * tpb * U + threadIdx.x; c0 < a.nchunks; c0 += stride)
        mixed_pass<KX, KY, U, CACHE, XY, EMU>(a, c0, tpb);
    wxpy_edges<CACHE, XY>(a, 4);
}

template <int KX, int KY, int U, int CACHE, bool XY, int EMU>
cudaError_t launch_mixed(unsigned grid, unsigned tpb, const SingleArgs &a, cudaStream_t s) {
    return launch_pdl(&wxpy_mixed_kernel<KX, KY, U, CACHE, XY, EMU>, grid, tpb, s, a);
}

template <int KX, int KY, int U, int CACHE, bool XY, int EMU>
SingleEntry make_mixed_entry() {
    return SingleEntry{(const void *)&wxpy_mixed_kernel<KX, KY, U, CACHE, XY, EMU>,
                       &launch_mixed<KX, KY, U, CACHE, XY, EMU>,
                       max_threads<4, U, 1, XY, EMU>()};
}

// Load width of an input whose offset relative to w, modulo 32 bytes, is
// `rel` bytes (0, 8, 16 or 24).
constexpr int mixed_width(int rel) { return rel == 0 ? 4 : (rel == 16 ? 2 : 1); }

// Instances of one EMU (kernels_mixed_e*.cu).  kx, ky: load widths 4, 2, 1;
// u_idx: log2 U (U = 1, 2, 4); cache: 1 or 2; xy: x == y (then kx == ky).
template <int EMU>
struct MixedTable {
    static SingleEntry get(int kx, int ky, int u_idx, int cache, int xy);
};

}  // namespace wx
