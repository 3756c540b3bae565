// batch_shape_api.cu -- C ABI of the batched launch's whole-launch knobs.
#include "internal.h"

using namespace wx;

extern "C" int wxpy_batch_launch_get(int *blocks_per_sm, int *fp64_offload) {
    if (!blocks_per_sm || !fp64_offload) return fail(WXPY_EINVAL, "null argument");
    const BatchShape s = current_batch_shape();
    *blocks_per_sm = s.blocks_per_sm;
    *fp64_offload = s.offload;
    return WXPY_OK;
}

extern "C" int wxpy_batch_launch_set(int blocks_per_sm, int fp64_offload) {
    if (blocks_per_sm < 1 || blocks_per_sm > 32 ||
        (fp64_offload != 0 && fp64_offload != 1 && fp64_offload != 3))
        return fail(WXPY_EINVAL, "blocks_per_sm must be 1..32 and fp64_offload 0, 1 or 3");
    BatchShape s = current_batch_shape();
    s.blocks_per_sm = blocks_per_sm;
    s.offload = fp64_offload;
    set_batch_shape(s);
    return WXPY_OK;
}
