// single_kernel.cuh -- the single-call VecWXPY kernel family (sm_103a).
//
// One template instance per (VW, U, GS, CACHE, XY):
//   VW     elements per vector access: 1, 2, 4 (8-, 16-, 32-byte ld/st; the
//          32-byte form is the sm_100+ 256-bit ld/st.global.v4.f64)
//   U      independent vectors per thread per pass (all loads of a pass are
//          issued before any store, so U*VW*16 bytes per thread are in flight)
//   GS     0: one-shot grid, each thread makes one pass;
//          1: grid-stride loop over a fixed grid
//   CACHE  0: ld/st.global; 1: ld.global.nc.L1::no_allocate + st.global.cs;
//          2: ld/st.global.cs (evict-first, coherent; used under aliasing)
//   XY     x == y: y is not loaded and w = RN(RN(alpha*x) + x)
//   EMU    which roundings run in the integer pipelines instead of FP64
//          instructions: 0 none, 1 half the sums, 2 every sum, 3 every product
// Threads per block and the grid size are launch parameters, not template
// parameters.
//
// Arithmetic (paper Sec. 3, Fig. 1, vecwxpy read as PETSc VecWXPY):
// w = __dadd_rn(__dmul_rn(alpha, x), y) -- two IEEE-correctly-rounded
// operations that the compiler may not fuse into an FMA.
//
// Aliasing: the memory accesses are inline-PTX `asm volatile`, which the
// compiler keeps in program order, and every pass loads all of its vectors
// before storing any.  A thread owns its chunks, so w == x or w == y reads
// each element before writing it.  Pointers are not declared __restrict__.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fp64_mul.cuh"

namespace wx {

struct SingleArgs {
    const double *x;   // unpeeled base pointers
    const double *y;
    double *w;
    double alpha;
    int64_t n;         // total elements
    int64_t head;      // scalar elements before the vector body (< VW)
    int64_t nchunks;   // vector body: chunks of VW elements starting at `head`
    MulCoef ca;        // alpha split for the integer-pipeline product (EMU == 3)
};

template <int VW, int CACHE>
__device__ __forceinline__ void ld_vec(const double *p, double (&r)[VW]) {
    if constexpr (VW == 4) {
        if constexpr (CACHE == 1)
            asm volatile("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3]) : "l"(p));
        else if constexpr (CACHE == 2)
            asm volatile("ld.global.cs.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3]) : "l"(p));
        else
            asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                         : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3]) : "l"(p));
    } else if constexpr (VW == 2) {
        if constexpr (CACHE == 1)
            asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
                         : "=d"(r[0]), "=d"(r[1]) : "l"(p));
        else if constexpr (CACHE == 2)
            asm volatile("ld.global.cs.v2.f64 {%0,%1}, [%2];"
                         : "=d"(r[0]), "=d"(r[1]) : "l"(p));
        else
            asm volatile("ld.global.v2.f64 {%0,%1}, [%2];"
                         : "=d"(r[0]), "=d"(r[1]) : "l"(p));
    } else {
        static_assert(VW == 1, "VW must be 1, 2 or 4");
        if constexpr (CACHE == 1)
            asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(r[0]) : "l"(p));
        else if constexpr (CACHE == 2)
            asm volatile("ld.global.cs.f64 %0, [%1];" : "=d"(r[0]) : "l"(p));
        else
            asm volatile("ld.global.f64 %0, [%1];" : "=d"(r[0]) : "l"(p));
    }
}

template <int VW, int CACHE>
__device__ __forceinline__ void st_vec(double *p, const double (&r)[VW]) {
    if constexpr (VW == 4) {
        if constexpr (CACHE == 0)
            asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};"
                         :: "l"(p), "d"(r[0]), "d"(r[1]), "d"(r[2]), "d"(r[3]) : "memory");
        else
            asm volatile("st.global.cs.v4.f64 [%0], {%1,%2,%3,%4};"
                         :: "l"(p), "d"(r[0]), "d"(r[1]), "d"(r[2]), "d"(r[3]) : "memory");
    } else if constexpr (VW == 2) {
        if constexpr (CACHE == 0)
            asm volatile("st.global.v2.f64 [%0], {%1,%2};"
                         :: "l"(p), "d"(r[0]), "d"(r[1]) : "memory");
        else
            asm volatile("st.global.cs.v2.f64 [%0], {%1,%2};"
                         :: "l"(p), "d"(r[0]), "d"(r[1]) : "memory");
    } else {
        if constexpr (CACHE == 0)
            asm volatile("st.global.f64 [%0], %1;" :: "l"(p), "d"(r[0]) : "memory");
        else
            asm volatile("st.global.cs.f64 [%0], %1;" :: "l"(p), "d"(r[0]) : "memory");
    }
}

// w = RN(RN(alpha*x) + y), element by element, never fused.
template <int VW>
__device__ __forceinline__ void wxpy_vec(double alpha, const double (&x)[VW],
                                         const double (&y)[VW], double (&w)[VW]) {
#pragma unroll
    for (int k = 0; k < VW; ++k) w[k] = __dadd_rn(__dmul_rn(alpha, x[k]), y[k]);
}

}  // namespace wx

#include "fp64_emu.cuh"

namespace wx {

// One pass of one thread: chunks c0, c0 + tpb, ..., c0 + (U-1)*tpb.  EMU
// selects which operations run in the integer pipelines (fp64_emu.cuh): 0
// none; 1 the sums of odd positions of the pass; 2 every sum; 3 every
// product (fp64_mul.cuh), the sums on the FP64 pipeline.  The choice depends
// only on the position, so it is the same for every lane of a warp.
template <int VW, int U, int CACHE, bool XY, int EMU>
__device__ __forceinline__ void wxpy_pass(const SingleArgs &a, int64_t c0, int64_t tpb) {
    const double *xb = a.x + a.head;
    const double *yb = a.y + a.head;
    double *wb = a.w + a.head;
    double xv[U][VW], yv[U][VW], wv[U][VW];
    if (c0 + (U - 1) * tpb < a.nchunks) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = (c0 + u * tpb) * VW;
            ld_vec<VW, CACHE>(xb + e, xv[u]);
            if constexpr (!XY) ld_vec<VW, CACHE>(yb + e, yv[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (XY) wxpy_vec_emu<VW, EMU>(a.alpha, a.ca, xv[u], xv[u], wv[u], u * VW);
            else wxpy_vec_emu<VW, EMU>(a.alpha, a.ca, xv[u], yv[u], wv[u], u * VW);
            st_vec<VW, CACHE>(wb + (c0 + u * tpb) * VW, wv[u]);
        }
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = c0 + u * tpb;
            if (c < a.nchunks) {
                ld_vec<VW, CACHE>(xb + c * VW, xv[u]);
                if constexpr (!XY) ld_vec<VW, CACHE>(yb + c * VW, yv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = c0 + u * tpb;
            if (c < a.nchunks) {
                if constexpr (XY) wxpy_vec_emu<VW, EMU>(a.alpha, a.ca, xv[u], xv[u], wv[u], u * VW);
                else wxpy_vec_emu<VW, EMU>(a.alpha, a.ca, xv[u], yv[u], wv[u], u * VW);
                st_vec<VW, CACHE>(wb + c * VW, wv[u]);
            }
        }
    }
}

// Head (elements [0, head)) and tail (elements after the vector body), at most
// VW-1 each, done with scalar accesses by threads 0..7 of block 0.
template <int CACHE, bool XY>
__device__ __forceinline__ void wxpy_edges(const SingleArgs &a, int64_t vw) {
    if (blockIdx.x != 0 || threadIdx.x >= 8) return;
    const int t = threadIdx.x;
    const int64_t body_end = a.head + a.nchunks * vw;
    int64_t e = -1;
    if (t < 4) {
        if (t < a.head) e = t;
    } else if (body_end + (t - 4) < a.n) {
        e = body_end + (t - 4);
    }
    if (e < 0) return;
    constexpr int C = (CACHE == 1) ? 2 : CACHE;  // scalar edges: coherent path
    double xv[1], yv[1], wv[1];
    ld_vec<1, C>(a.x + e, xv);
    if constexpr (XY) yv[0] = xv[0];
    else ld_vec<1, C>(a.y + e, yv);
    wxpy_vec<1>(a.alpha, xv, yv, wv);
    st_vec<1, C>(a.w + e, wv);
}

// Largest block size of an instance.  A thread keeps U*VW*(XY ? 1 : 2) doubles
// of input live (two registers each) and about three 64-bit addresses per
// unrolled vector, plus the loop state of the grid-stride form; the estimate
// below must fit the per-thread register share 65536 / threads, so that the
// compiler never spills to the stack.  The integer-pipeline sum (EMU > 0)
// needs a handful of 64-bit temporaries more.
template <int VW, int U, int GS, bool XY, int EMU>
constexpr int max_threads() {
    constexpr int regs =
        2 * U * VW * (XY ? 1 : 2) + 6 * U + 20 + (GS ? 16 : 0) + (EMU ? 24 : 0) +
        (EMU == 3 ? 8 : 0);
    return regs <= 64 ? 1024 : (regs <= 128 ? 512 : 256);
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialisation may start while the previous kernel of
// its stream is still running; it waits here until that kernel has completed
// and its memory operations are visible (a no-op for a launch without the
// attribute), and then lets the next launch of the stream be scheduled: once
// every block of this grid has passed this point, the next kernel's blocks
// can take the SMs this grid frees, so its launch overlaps this grid's tail.
// Nothing is read or written before the wait, so any dependence between calls
// (w of one call is x of the next) is kept; only L2 prefetches are issued
// ahead of it (prefetch_first_pass).
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Before the wait: the L2 lines of this thread's first pass of x and y are
// requested, so that a call launched behind another one starts its DRAM
// reads during the other's tail.  A prefetch changes no value, and the L2 is
// where device memory is coherent, so a line the previous call is still
// writing is read with its final contents after the wait.
template <int VW, int U, bool XY>
__device__ __forceinline__ void prefetch_first_pass(const SingleArgs &a, int64_t c0, int64_t tpb) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + u * tpb;
        if (c < a.nchunks) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.x + a.head + c * VW));
            if constexpr (!XY) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.y + a.head + c * VW));
        }
    }
}

template <int VW, int U, int GS, int CACHE, bool XY, int EMU>
__global__ void __launch_bounds__(max_threads<VW, U, GS, XY, EMU>())
    wxpy_single_kernel(const SingleArgs a) {
    prefetch_first_pass<VW, U, XY>(a, (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x, blockDim.x);
    pdl_enter();
    const int64_t tpb = blockDim.x;
    if constexpr (GS == 0) {
        const int64_t c0 = (int64_t)blockIdx.x * tpb * U + threadIdx.x;
        if (c0 < a.nchunks) wxpy_pass<VW, U, CACHE, XY, EMU>(a, c0, tpb);
    } else {
        const int64_t stride = (int64_t)gridDim.x * tpb * U;
        for (int64_t c0 = (int64_t)blockIdx.x * tpb * U + threadIdx.x; c0 < a.nchunks;
             c0 += stride)
            wxpy_pass<VW, U, CACHE, XY, EMU>(a, c0, tpb);
    }
    wxpy_edges<CACHE, XY>(a, VW);
}

// The reference variant of Sec. 2: the plain loop, one element per thread.
__global__ void wxpy_reference_kernel(const SingleArgs a);

using SingleLaunchFn = cudaError_t (*)(unsigned grid, unsigned tpb, const SingleArgs &,
                                       cudaStream_t);

struct SingleEntry {
    const void *func;       // kernel symbol (for cudaFuncSetAttribute)
    SingleLaunchFn launch;  // <<<grid, tpb, 0, stream>>>
    int max_threads;        // launch bound of the instance
};

// Whether launches of the single-call kernels ask for programmatic stream
// serialisation (api.cu; default on, WXPY_PDL=0 or wxpy_launch_pdl(0) off).
bool pdl_enabled();

// <<<grid, tpb, 0, s>>>, with the programmatic-serialisation attribute when on.
template <typename... Args>
cudaError_t launch_pdl(void (*kernel)(Args...), unsigned grid, unsigned tpb, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tpb);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int VW, int U, int GS, int CACHE, bool XY, int EMU>
cudaError_t launch_single(unsigned grid, unsigned tpb, const SingleArgs &a, cudaStream_t s) {
    return launch_pdl(&wxpy_single_kernel<VW, U, GS, CACHE, XY, EMU>, grid, tpb, s, a);
}

template <int VW, int U, int GS, int CACHE, bool XY, int EMU>
SingleEntry make_single_entry() {
    return SingleEntry{(const void *)&wxpy_single_kernel<VW, U, GS, CACHE, XY, EMU>,
                       &launch_single<VW, U, GS, CACHE, XY, EMU>,
                       max_threads<VW, U, GS, XY, EMU>()};
}

// Table of one (VW, EMU): index ((u_idx * 2 + gs) * 3 + cache) * 2 + xy, u_idx = log2 U.
template <int VW, int EMU>
struct SingleTable {
    static SingleEntry get(int u_idx, int gs, int cache, int xy);
};

}  // namespace wx
