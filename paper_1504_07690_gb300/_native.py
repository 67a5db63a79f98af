"""ctypes declarations of the C ABI in include/ssm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libssm.so")

SSM_OK = 0
STATUS_NAMES = {0: "SSM_OK", 1: "SSM_EINVAL", 2: "SSM_ENOMEM", 3: "SSM_ECUDA", 4: "SSM_ETIMEOUT",
                5: "SSM_ENONFINITE", 6: "SSM_ENOTSYM", 7: "SSM_EDOMAIN", 8: "SSM_ESTATE",
                9: "SSM_ENOCONV"}
SSM_FP64 = 0
SSM_MIXED = 1
SSM_FP64_TC = 2  # float64 recurrence, tensor-core Gram products from exact bf16 slices
PRECISIONS = {"fp64": SSM_FP64, "mixed": SSM_MIXED, "fp64_tc": SSM_FP64_TC}
SSM_DAMP_NONE, SSM_DAMP_JACKSON, SSM_DAMP_LORENTZ = 0, 1, 2
SSM_OPT_CUDA_CORE_GRAM = 1
SSM_OPT_ADJOINT = 2
SSM_OPT_FUSED_STEP = 4  # mixed stencil plans: recurrence step and Gram products in one launch
SSM_OPT_PINV = 8  # per-point estimate Tr[K_W^+ K_Z] (pseudo-inverse form, no range filter)


class ssm_stencil(C.Structure):
    _fields_ = [("dims", C.c_int64 * 3), ("periodic", C.c_int32 * 3), ("diag", C.c_void_p),
                ("offdiag", C.c_double * 3)]


class ssm_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("val", C.c_void_p)]


class ssm_params(C.Structure):
    _fields_ = [("n_v", C.c_int32), ("n_vh", C.c_int32), ("degree", C.c_int32), ("precision", C.c_int32),
                ("lo", C.c_double), ("hi", C.c_double), ("tau", C.c_double), ("kappa", C.c_double),
                ("n_theta", C.c_int32), ("options", C.c_int32), ("eps_floor", C.c_double),
                ("damping", C.c_int32), ("damping_lambda", C.c_double)]


class ssm_stats(C.Structure):
    _fields_ = [("ms_coeffs", C.c_double), ("ms_recurrence", C.c_double), ("ms_gram", C.c_double),
                ("ms_reduce", C.c_double), ("ms_assemble", C.c_double), ("ms_solve", C.c_double),
                ("ms_kpm", C.c_double), ("ms_trace", C.c_double), ("ms_adjoint", C.c_double),
                ("recurrence_launches", C.c_int64),
                ("gram_launches", C.c_int64), ("launches", C.c_int64)]


TRACE_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)

# name -> (restype, argtypes), mirroring include/ssm.h
SIGNATURES = {
    "ssm_plan_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(ssm_stencil), C.POINTER(ssm_csr),
                                  C.POINTER(ssm_params), C.c_void_p]),
    "ssm_plan_create_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(ssm_csr),
                                          C.POINTER(ssm_params), C.c_void_p]),
    "ssm_batch_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "ssm_plan_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
    "ssm_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "ssm_dos": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p,
                          C.c_void_p]),
    "ssm_trace_f": (C.c_int, [C.c_void_p, TRACE_FN, C.c_void_p, C.c_int64, C.c_double, C.c_double,
                              C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ssm_trace_weights": (C.c_int, [C.c_void_p, TRACE_FN, C.c_void_p, C.c_int64, C.c_double, C.c_double,
                                    C.c_double, C.c_void_p, C.c_void_p]),
    "ssm_plan_set_diag": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ssm_kpm_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p]),
    "ssm_moments_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "ssm_coefficients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                   C.c_void_p]),
    "ssm_gram_pair": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int64, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "ssm_gram_pair_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int64,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssm_timing_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "ssm_debug_fail_alloc": (C.c_int, [C.c_int32]),
    "ssm_debug_explicit_chunk": (C.c_int, [C.c_int32]),
    "ssm_batch_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ssm_dos_explicit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                                   C.c_void_p, C.c_void_p]),
    "ssm_selftest_wait": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p]),
    "ssm_stats_get": (C.c_int, [C.c_void_p, C.POINTER(ssm_stats)]),
    "ssm_stats_reset": (C.c_int, [C.c_void_p]),
    "ssm_plan_destroy": (None, [C.c_void_p]),
    "ssm_last_error": (C.c_char_p, [C.c_void_p]),
    "ssm_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libssm.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SSMError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.name}: {message}")
