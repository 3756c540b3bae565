// kernels_mixed_e3.cu -- instances of the mixed-alignment kernel with EMU = 3
// (every product in the integer pipelines, the sums on the FP64 pipeline).  One
// translation unit per EMU so that the build compiles them in parallel.
#include <array>
#include <utility>

#include "mixed_kernel.cuh"

namespace wx {
namespace {
constexpr int kWidths[3] = {4, 2, 1};

// index I < 54: ((kx_idx * 3 + ky_idx) * 3 + u_idx) * 2 + cache_idx, x != y;
// index I >= 54: I - 54 = (k_idx * 3 + u_idx) * 2 + cache_idx, x == y (kx = ky).
template <std::size_t I>
SingleEntry entry() {
    if constexpr (I < 54)
        return make_mixed_entry<kWidths[I / 18], kWidths[(I / 6) % 3], (1 << ((I / 2) % 3)),
                                1 + int(I % 2), false, 3>();
    else
        return make_mixed_entry<kWidths[(I - 54) / 6], kWidths[(I - 54) / 6],
                                (1 << (((I - 54) / 2) % 3)), 1 + int((I - 54) % 2), true, 3>();
}

template <std::size_t... I>
std::array<SingleEntry, sizeof...(I)> build_table(std::index_sequence<I...>) {
    return {entry<I>()...};
}

int width_index(int k) { return k == 4 ? 0 : (k == 2 ? 1 : 2); }
}  // namespace

template <>
SingleEntry MixedTable<3>::get(int kx, int ky, int u_idx, int cache, int xy) {
    static const std::array<SingleEntry, 72> table = build_table(std::make_index_sequence<72>{});
    const int ci = cache == 2 ? 1 : 0;
    if (xy) return table[54 + (width_index(kx) * 3 + u_idx) * 2 + ci];
    return table[((width_index(kx) * 3 + width_index(ky)) * 3 + u_idx) * 2 + ci];
}
}  // namespace wx
