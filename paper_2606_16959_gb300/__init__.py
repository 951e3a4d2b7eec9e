"""Diagonal-budgeted Trotterization on one GB300 GPU (arxiv 2606.16959 hot path).

The compute path is libhs.so (CUDA, sm_103a) behind the C ABI in include/hs.h;
``paper_2606_16959_gb300.hs`` is its thin Python binding (same names).
"""
from .hs import (  # noqa: F401
    HS_C64, HS_C128, HS_METHOD_AUTO, HS_METHOD_FUSED, HS_METHOD_PLAIN, Batch, Factors, HSError,
    hs_batch_create, hs_batch_launch,
    hs_apply_factor, hs_autotune, hs_build_factors, hs_build_factors_masks, hs_evolve, hs_evolve_ex, hs_evolve_plan, hs_fidelity,
    hs_inner_device, hs_plan_factors,
)
