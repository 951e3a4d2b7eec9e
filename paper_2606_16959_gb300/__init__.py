"""Diagonal-budgeted Trotterization on one GB300 GPU (arxiv 2606.16959 hot path).

The compute path is libhs.so (CUDA, sm_103a) behind the C ABI in include/hs.h
(grouped rotation factors) and include/hs_dia.h (single-factor Taylor mode);
``paper_2606_16959_gb300.hs`` is its thin Python binding (same names).
"""
from .hs import (  # noqa: F401
    HS_C64, HS_C128, HS_METHOD_AUTO, HS_METHOD_FUSED, HS_METHOD_PLAIN, Batch, Factors, HSError,
    hs_batch_create, hs_batch_launch,
    hs_apply_factor, hs_autotune, hs_build_factors, hs_build_factors_masks, hs_evolve, hs_evolve_ex, hs_evolve_plan, hs_fidelity,
    hs_inner_device, hs_plan_factors,
    Dia, hs_dia_convert, hs_dia_create, hs_dia_evolve, hs_dia_from_masks, hs_dia_from_terms, hs_estimate_timesteps,
    hs_spgemm, hs_spme, hs_spmv, hs_expectation, hs_kernel_launches,
    hs_build_factors_td, hs_evolve_td, hs_factors_set_drive, hs_dia_evolve_td,
)
