"""GB300-native spectrum sweeping (RESS-DGC) DOS estimator.

The computation lives in libssm.so (CUDA for sm_103a, C ABI in
include/ssm.h); this package builds it (``build.build``) and binds it
(``api``).  There is no CPU fallback: calls fail when the library is missing.
"""
from .api import (Plan, ssm_coefficients, ssm_dos, ssm_gram_pair, ssm_kpm_adjoint, ssm_moments, ssm_moments_adjoint,
                  ssm_plan_create, ssm_plan_destroy, ssm_plan_info, ssm_plan_set_diag, ssm_stats_get, ssm_stats_reset,
                  ssm_timing_enable, ssm_trace_f, ssm_trace_weights, ssm_plan_create_batched, ssm_batch_info,
                  ssm_debug_fail_alloc, ssm_selftest_wait, ssm_batch_tuning, ssm_dos_explicit,
                  ssm_debug_explicit_chunk)
from ._native import SSMError

__all__ = ["Plan", "SSMError", "ssm_coefficients", "ssm_dos", "ssm_gram_pair", "ssm_moments", "ssm_plan_create",
           "ssm_plan_destroy", "ssm_plan_info", "ssm_stats_get", "ssm_stats_reset", "ssm_timing_enable",
           "ssm_trace_f", "ssm_trace_weights", "ssm_plan_set_diag", "ssm_kpm_adjoint", "ssm_moments_adjoint",
           "ssm_plan_create_batched", "ssm_batch_info", "ssm_debug_fail_alloc", "ssm_selftest_wait",
           "ssm_batch_tuning", "ssm_dos_explicit", "ssm_debug_explicit_chunk", "KPMDensity"]
from .autograd import KPMDensity  # noqa: E402
