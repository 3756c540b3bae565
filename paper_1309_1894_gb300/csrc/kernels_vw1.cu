// kernels_vw1.cu -- instances of the single-call kernel family with VW = 1
// (8-byte loads and stores).  One translation unit per vector width so
// that the build compiles them in parallel.
#include <array>
#include <utility>

#include "single_kernel.cuh"

namespace wx {
namespace {
// index I = ((u_idx * 2 + gs) * 3 + cache) * 2 + xy
template <std::size_t... I>
std::array<SingleEntry, sizeof...(I)> build_vw1(std::index_sequence<I...>) {
    return {make_single_entry<1, (1 << (I / 12)), int((I / 6) % 2), int((I / 2) % 3),
                              (I % 2) == 1>()...};
}
}  // namespace

template <>
SingleEntry SingleTable<1>::get(int u_idx, int gs, int cache, int xy) {
    static const std::array<SingleEntry, 48> table = build_vw1(std::make_index_sequence<48>{});
    return table[((u_idx * 2 + gs) * 3 + cache) * 2 + xy];
}
}  // namespace wx

namespace wx {
// The reference variant (paper Sec. 2: the plain code whose outputs every
// variant is compared with): one element per thread, plain loads and stores.
__global__ void wxpy_reference_kernel(const SingleArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const double xi = a.x[i];
        const double yi = a.y[i];
        a.w[i] = __dadd_rn(__dmul_rn(a.alpha, xi), yi);
    }
}

cudaError_t launch_reference(unsigned grid, unsigned tpb, const SingleArgs &a, cudaStream_t s) {
    wxpy_reference_kernel<<<grid, tpb, 0, s>>>(a);
    return cudaGetLastError();
}
}  // namespace wx
