// kernels_vw4_e3.cu -- instances of the single-call kernel family with
// VW = 4 (32-byte loads and stores) and EMU = 3 (every product in the integer
// pipelines; the sums on the FP64 pipeline).  One translation unit per (VW, EMU) so
// that the build compiles them in parallel.
#include <array>
#include <utility>

#include "single_kernel.cuh"

namespace wx {
namespace {
// index I = ((u_idx * 2 + gs) * 3 + cache) * 2 + xy
template <std::size_t... I>
std::array<SingleEntry, sizeof...(I)> build_table(std::index_sequence<I...>) {
    return {make_single_entry<4, (1 << (I / 12)), int((I / 6) % 2), int((I / 2) % 3),
                              (I % 2) == 1, 3>()...};
}
}  // namespace

template <>
SingleEntry SingleTable<4, 3>::get(int u_idx, int gs, int cache, int xy) {
    static const std::array<SingleEntry, 48> table = build_table(std::make_index_sequence<48>{});
    return table[((u_idx * 2 + gs) * 3 + cache) * 2 + xy];
}
}  // namespace wx
