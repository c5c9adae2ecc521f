"""GB300-native communication-avoiding LU and QR (CALU / CAQR with TSLU and
TSQR reduction trees), after Grigori, Jacquelin and Khabou, "Multilevel
communication optimal LU and QR factorizations for hierarchical platforms".

The compute path is ``libcagb300.so`` (CUDA for sm_103a, C-ABI in
``include/ca_gb300.h``); this package holds its build script, the thin
ctypes binding (same names as the C-ABI) and the seeded input generators.
"""
_BINDING_NAMES = {
    "calu_factor", "tslu", "calu_getrs", "caqr_factor", "tsqr", "caqr_geqrs",
    "ca_calu_workspace", "ca_caqr_workspace", "ca_geqrs_workspace", "make_tree", "colmajor",
    "ca_tree_t", "CaError", "BINARY", "FLAT", "load", "lib_path",
    "ca_prof_enable", "ca_prof_read", "ca_launch_count", "ca_kernel_class_name", "KERNEL_CLASSES",
    "ca_gemm_mixed_workspace", "ca_gemm_minus_mixed", "tslu_noalloc", "ca_calu_mixed_workspace",
    "calu_factor_mixed", "ca_gesv_mixed_workspace", "calu_gesv_mixed", "ca_caqr_mixed_workspace",
    "caqr_factor_mixed", "ca_batched_plan", "ca_batched_factor", "BatchedFactor", "ca_batch_item_t",
    "CA_BATCH_CALU", "CA_BATCH_CAQR", "CA_DTYPE_F64", "CA_DTYPE_F32", "ca_solve_status",
    "ca_getrs_workspace", "ca_test_solve_hook", "CA_REFINE_CLASSIC", "CA_REFINE_GMRES", "CA_REFINE_AUTO",
    "CA_STATUS_SOLVE_TIMEOUT", "CA_STATUS_REFACTORED", "ca_peak_probe", "ca_gels_mixed_workspace",
    "caqr_gels_mixed",
}


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
