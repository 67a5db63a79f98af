"""The C ABI library loads and exports what include/ssm.h declares (no GPU).

Argument checks that precede any CUDA call are exercised too.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ssm.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ssm_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_07690_gb300 import _native as N

    if not os.path.exists(N.LIB_PATH):
        from paper_1504_07690_gb300 import build as B

        B.build()
    return N.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("ssm_plan_create", "ssm_moments", "ssm_dos", "ssm_trace_f", "ssm_plan_destroy",
                 "ssm_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1504_07690_gb300 import _native as N

    assert set(_declared_functions()) == set(N.SIGNATURES)


def test_struct_layouts_match_header_sizes():
    from paper_1504_07690_gb300 import _native as N

    assert C.sizeof(N.ssm_stencil) == 3 * 8 + 3 * 4 + 4 + 8 + 3 * 8
    assert C.sizeof(N.ssm_csr) == 5 * 8
    # ..., eps_floor, then damping (int32, padded to 8) and damping_lambda
    assert C.sizeof(N.ssm_params) == 4 * 4 + 4 * 8 + 2 * 4 + 8 + 8 + 8
    assert N.ssm_params.damping_lambda.offset == 72
    assert C.sizeof(N.ssm_stats) == 9 * 8 + 3 * 8


def test_status_strings(lib):
    assert lib.ssm_status_string(0) == b"SSM_OK"
    assert lib.ssm_status_string(8) == b"SSM_ESTATE"


@pytest.mark.parametrize("field,value", [("degree", 7), ("degree", 0), ("n_v", 0), ("precision", 5),
                                         ("n_theta", 3), ("options", 16), ("damping", 3), ("damping", -1),
                                         ("precision", 3)])
def test_parameter_validation_before_any_cuda_call(lib, field, value):
    from paper_1504_07690_gb300 import _native as N

    p = N.ssm_params(n_v=4, n_vh=0, degree=10, precision=0, lo=0, hi=0, tau=0, kappa=-1, n_theta=0, options=0)
    setattr(p, field, value)
    diag = (C.c_double * 8)(*([2.0] * 8))
    st = N.ssm_stencil((C.c_int64 * 3)(8, 1, 1), (C.c_int32 * 3)(0, 0, 0), C.cast(diag, C.c_void_p),
                       (C.c_double * 3)(-1.0, 0, 0))
    h = C.c_void_p()
    status = lib.ssm_plan_create(C.byref(h), C.byref(st), None, C.byref(p), None)
    assert status == 1  # SSM_EINVAL
    assert not h.value
    assert lib.ssm_last_error(None)


def test_both_or_no_operator_is_rejected(lib):
    from paper_1504_07690_gb300 import _native as N

    p = N.ssm_params(n_v=4, n_vh=0, degree=10, precision=0, lo=0, hi=0, tau=0, kappa=-1, n_theta=0, options=0)
    h = C.c_void_p()
    assert lib.ssm_plan_create(C.byref(h), None, None, C.byref(p), None) == 1


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.ssm_moments(None, None, 0, None) == 1
    assert lib.ssm_dos(None, None, 0, 1.0, None, None, None) == 1
    assert lib.ssm_moments_adjoint(None, None, 1, None, None) == 1
    assert lib.ssm_kpm_adjoint(None, None, 0, 1.0, None, None) == 1
    assert lib.ssm_plan_set_diag(None, None) == 1
    lib.ssm_plan_destroy(None)
