// reference.cu -- the reference variant (paper Sec. 2: the plain code whose
// outputs every variant is compared with): one element per thread, plain
// loads and stores, the two hardware-rounded FP64 operations.
#include "single_kernel.cuh"

namespace wx {

__global__ void wxpy_reference_kernel(const SingleArgs a) {
    pdl_enter();  // launched like the family's kernels, so that timings compare
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const double xi = a.x[i];
        const double yi = a.y[i];
        a.w[i] = __dadd_rn(__dmul_rn(a.alpha, xi), yi);
    }
}

cudaError_t launch_reference(unsigned grid, unsigned tpb, const SingleArgs &a, cudaStream_t s) {
    return launch_pdl(&wxpy_reference_kernel, grid, tpb, s, a);
}

}  // namespace wx
