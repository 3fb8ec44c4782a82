"""GB300-native direct inverse NFFT (Kircheis & Potts, Sec. 3.2.1 and 3.2.2).

Thin Python binding of the C ABI in include/infft.h: argument marshalling only.
Every numerical step runs in the CUDA kernels of libinfft_gb300.so; importing a
function whose library is not built raises InfftError (there is no fallback).
"""
from .binding import (  # noqa: F401
    InfftError, Plan, library, infft_plan, infft_plan_create, infft_set_nodes, infft_precompute,
    infft_apply, nfft_apply, infft_apply_z, nfft_apply_z, plan_destroy, infft_get_info,
    infft_copy_plan_data, infft_profile, infft_profile_read, infft_launch_count, infft_version,
    infft_fft_deconv_noalloc, infft_grad_nodes, infft_plan_create_ansatz, infft_ndft_z, infft_refine_z,
    infft_nfft_kb_z, infft_apply_sorted, infft_sort_values, infft_apply_configs, infft_set_apply_config,
    infft_get_apply_config, infft_tune_apply, infft_fp64_fma_probe, infft_fp64_fma_probe_sink_len,
    Batch, infft_batch_create, infft_batch_set_nodes, infft_batch_precompute, infft_batch_apply,
    infft_batch_get_info, infft_batch_copy_problem, infft_apply_many, infft_apply_many_workspace,
    infft_batch_tile_shapes, infft_batch_set_tile_shape, infft_batch_get_tile_shape, infft_batch_tune_apply,
    EXPORTED_SYMBOLS, KERNEL_FULL, KERNEL_SYM, ANSATZ_UNDERDETERMINED, ANSATZ_OVERDETERMINED,
    Plan2D, infft2d_plan_create, infft2d_set_nodes, infft2d_precompute, infft2d_apply, infft2d_apply_z,
    infft2d_get_info, infft2d_copy_plan_data,
)
from .autograd import InverseNFFT, inverse_nfft  # noqa: F401
from .tuning import batch_workload_key, autotune_batch  # noqa: F401
