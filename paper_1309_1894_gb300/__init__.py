"""GB300 (sm_103a) VecWXPY: FP64 w = alpha*x + y as an autotuned CUDA kernel family.

The paper (Sec. 2) tunes a kernel by generating annotated variants, running
them, checking their outputs against the plain reference code and keeping the
fastest; this package applies that method to the kernel it reports on
(Sec. 3, Fig. 1, "vecwxpy").  The computation lives in ``libwxpy.so``
(C ABI: ``include/wxpy.h``); this package is its ctypes binding.  Importing it
does not load the library; the first call does, and raises if it is missing.
"""
from .binding import (  # noqa: F401
    WxpyError, lib, check, version, strerror,
    wxpy, wxpy_host, wxpy_host_config, wxpy_run_variant,
    wxpy_axpy, wxpy_aypx, wxpy_axpby, wxpy_axpbypcz, wxpy_maxpy, wxpy_pointwise_mult,
    wxpy_vecops_pipes, wxpy_vecops_status, wxpy_vecops_tune, wxpy_vecops_tuned_get,
    wxpy_vecops_tuned_set, wxpy_debug_vecops_drop_tile,
    wxpy_norm2, wxpy_dot, wxpy_reduce_pipes, wxpy_reduce_status, wxpy_reduce_variant, wxpy_reduce_sum_levels,
    wxpy_debug_reduce_drop_chunk, wxpy_reduce_tune, wxpy_reduce_tuned_get, wxpy_reduce_tuned_set,
    reduce_workspace,
    VEC_AXPBYPCZ, VEC_PMULT, VEC_AXPBY, VEC_CLASSES, VEC_CLASS_NAMES,
    wxpy_reference, wxpy_lookup, wxpy_classify,
    wxpy_device_query, wxpy_variant_count, wxpy_variant_describe, wxpy_variant_encode,
    wxpy_set_variant, wxpy_debug_inject_launch_error, wxpy_fill_uniform, wxpy_launch_pdl,
    wxpy_tune, tune, wxpy_tune_get, wxpy_tune_set, wxpy_tune_clear, wxpy_tune_cache_save,
    wxpy_tune_cache_load,
    TUNE_ALIGN16, TUNE_ALIGN8, TUNE_XY, TUNE_WALIAS, TUNE_QUICK, TUNE_RESIDENT,
    desc_table, table_to_device, BatchPlan, wxpy_batch_plan_create, wxpy_batch,
    wxpy_batch_tune, wxpy_batch_shape_get, wxpy_batch_shape_set, wxpy_batch_shape_reset,
    wxpy_batch_launch_get, wxpy_batch_launch_set,
    ALIAS_XY, ALIAS_WX, ALIAS_WY,
    WXPY_OK, WXPY_EINVAL, WXPY_EOVERLAP, WXPY_ENOMEM, WXPY_EBUDGET, WXPY_ECUDA,
    WXPY_ETIMEOUT, WXPY_ENOTFOUND, WXPY_EBUSY, WXPY_EMISMATCH,
)
from .server import Server, SERVE_BATCHED, SERVE_SERIAL, SERVE_FUSED  # noqa: F401,E402
