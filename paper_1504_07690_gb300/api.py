"""Python binding of the spectrum sweeping library (include/ssm.h).

The functions carry the C names and only marshal arguments: every step of
the computation runs in the CUDA kernels of libssm.so.  Arrays may be numpy
arrays (host memory) or torch tensors (host or CUDA); outputs live where the
main input lives (CUDA tensors in, CUDA tensors out).  PyTorch, when present,
supplies the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from typing import Callable, Optional, Tuple

import numpy as np

from . import _native as N

try:  # torch is plumbing only (device memory and streams)
    import torch
except Exception:  # pragma: no cover
    torch = None


def _is_cuda(x) -> bool:
    return torch is not None and isinstance(x, torch.Tensor) and x.is_cuda


def _as_buffer(x, dtype):
    """(keepalive, pointer) for a float64/int array that the library reads."""
    if torch is not None and isinstance(x, torch.Tensor):
        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        t = x.detach().to(tdt).contiguous()
        return t, t.data_ptr()
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a, a.ctypes.data


def _empty_like_input(ref, shape, dtype):
    if _is_cuda(ref):
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        t = torch.empty(shape, dtype=tdt, device=ref.device)
        return t, t.data_ptr()
    a = np.empty(shape, dtype=dtype)
    return a, a.ctypes.data


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    if torch is not None and torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _check(lib, status: int, handle):
    if status != N.SSM_OK:
        msg = lib.ssm_last_error(handle)
        raise N.SSMError(status, msg.decode() if msg else "")


class Plan:
    """Owns one ssm_plan_t (destroyed with the object)."""

    def __init__(self, handle, params: N.ssm_params, is_stencil: bool = True):
        self.handle = handle
        self.params = params
        self.is_stencil = is_stencil
        self._lib = N.load()
        n, nnz = C.c_int64(), C.c_int64()
        self._lib.ssm_plan_info(handle, None, None, None, None, C.byref(n), C.byref(nnz))
        self.n = n.value
        self.nnz = nnz.value

    @property
    def n_v(self) -> int:
        return self.params.n_v

    @property
    def n_vh(self) -> int:
        return self.params.n_vh

    @property
    def n_tot(self) -> int:
        return self.params.n_v + self.params.n_vh

    @property
    def degree(self) -> int:
        return self.params.degree

    def close(self):
        if self.handle:
            self._lib.ssm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_DAMPING = {None: 0, "none": 0, "jackson": 1, "lorentz": 2, 0: 0, 1: 1, 2: 2}


def _params(n_v, n_vh, degree, precision, lo, hi, tau, kappa, n_theta, options, eps_floor, damping,
            damping_lambda):
    # names are translated; other integers go to the library unchanged (it rejects them)
    code = _DAMPING[damping] if damping in _DAMPING else int(damping)
    return N.ssm_params(n_v=n_v, n_vh=n_vh, degree=degree, precision=N.PRECISIONS[precision], lo=lo, hi=hi,
                        tau=tau, kappa=kappa, n_theta=n_theta, options=options, eps_floor=eps_floor,
                        damping=code, damping_lambda=damping_lambda)


def ssm_plan_create(stencil=None, csr=None, *, n_v: int, degree: int, n_vh: int = 0,
                    precision: str = "fp64", lo: float = 0.0, hi: float = 0.0, tau: float = 0.0,
                    kappa: float = -1.0, n_theta: int = 0, eps_floor: float = 0.0, options: int = 0,
                    damping=None, damping_lambda: float = 0.0, stream=None) -> Plan:
    """ssm_plan_create: operator (stencil descriptor or CSR) + parameters -> Plan."""
    lib = N.load()
    p = _params(n_v, n_vh, degree, precision, lo, hi, tau, kappa, n_theta, options, eps_floor, damping,
                damping_lambda)
    keep = []
    st_p = None
    csr_p = None
    if stencil is not None:
        d, dptr = _as_buffer(stencil.diag, np.float64)
        keep.append(d)
        dims = list(stencil.dims) + [1] * (3 - len(stencil.dims))
        per = list(stencil.periodic) + [0] * (3 - len(stencil.periodic))
        off = list(stencil.offdiag) + [0.0] * (3 - len(stencil.offdiag))
        st = N.ssm_stencil((C.c_int64 * 3)(*dims), (C.c_int32 * 3)(*[int(bool(v)) for v in per]), dptr,
                           (C.c_double * 3)(*off))
        st_p = C.byref(st)
    if csr is not None:
        rp, rpp = _as_buffer(csr.rowptr, np.int64)
        ci, cip = _as_buffer(csr.colind, np.int32)
        va, vap = _as_buffer(csr.val, np.float64)
        keep += [rp, ci, va]
        cs = N.ssm_csr(int(csr.n), int(len(csr.val)), rpp, cip, vap)
        csr_p = C.byref(cs)
    h = C.c_void_p()
    status = lib.ssm_plan_create(C.byref(h), st_p, csr_p, C.byref(p), _stream(stream))
    _check(lib, status, None)
    return Plan(h, p, is_stencil=stencil is not None)


def ssm_plan_create_batched(csrs, *, n_v: int, degree: int, n_vh: int = 0, precision: str = "mixed",
                            lo: float = 0.0, hi: float = 0.0, tau: float = 0.0, kappa: float = -1.0,
                            n_theta: int = 0, eps_floor: float = 0.0, options: int = 0, damping=None,
                            damping_lambda: float = 0.0, stream=None) -> Plan:
    """ssm_plan_create_batched: B CSR operators of uneven size in one plan."""
    lib = N.load()
    p = _params(n_v, n_vh, degree, precision, lo, hi, tau, kappa, n_theta, options, eps_floor, damping,
                damping_lambda)
    keep = []
    arr = (N.ssm_csr * len(csrs))()
    for k, c in enumerate(csrs):
        rp, rpp = _as_buffer(c.rowptr, np.int64)
        ci, cip = _as_buffer(c.colind, np.int32)
        va, vap = _as_buffer(c.val, np.float64)
        keep += [rp, ci, va]
        arr[k] = N.ssm_csr(int(c.n), int(len(c.val)), rpp, cip, vap)
    h = C.c_void_p()
    _check(lib, lib.ssm_plan_create_batched(C.byref(h), len(csrs), arr, C.byref(p), _stream(stream)), None)
    plan = Plan(h, p, is_stencil=False)
    plan.batch = len(csrs)
    return plan


def ssm_batch_info(plan: Plan, b: int) -> dict:
    lib = N.load()
    a, bb, lo, hi = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    _check(lib, lib.ssm_batch_info(plan.handle, int(b), C.byref(a), C.byref(bb), C.byref(lo), C.byref(hi),
                                   C.byref(n)), plan.handle)
    return dict(a=a.value, b=bb.value, lo=lo.value, hi=hi.value, n=n.value)


def ssm_batch_tuning(plan: Plan) -> dict:
    """ssm_batch_tuning: the autotuned CSR CTA size and Gram slab count of a batched plan."""
    lib = N.load()
    ct, gs = C.c_int32(), C.c_int32()
    _check(lib, lib.ssm_batch_tuning(plan.handle, C.byref(ct), C.byref(gs)), plan.handle)
    return {"csr_threads": ct.value, "gram_slabs": gs.value}


def ssm_plan_info(plan: Plan) -> dict:
    lib = N.load()
    a, b, lo, hi = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    n, nnz = C.c_int64(), C.c_int64()
    _check(lib, lib.ssm_plan_info(plan.handle, C.byref(a), C.byref(b), C.byref(lo), C.byref(hi),
                                  C.byref(n), C.byref(nnz)), plan.handle)
    return dict(a=a.value, b=b.value, lo=lo.value, hi=hi.value, n=n.value, nnz=nnz.value)


def ssm_moments(plan: Plan, W, return_moments: bool = False):
    """ssm_moments: X_l = W^T T_l(A~) W for l = 0..M; returns them if asked."""
    lib = N.load()
    Wb, Wp = _as_buffer(W, np.float64)
    ldw = Wb.shape[1]
    out = None
    optr = None
    if return_moments:
        shp = (plan.degree + 1, plan.n_tot, plan.n_tot)
        if getattr(plan, "batch", 0):
            shp = (plan.batch,) + shp
        out, optr = _empty_like_input(W, shp, np.float64)
    _check(lib, lib.ssm_moments(plan.handle, Wp, ldw, optr), plan.handle)
    return out


def ssm_dos(plan: Plan, t, sigma: float, want_ss: bool = True, want_kpm: bool = True,
            want_rank: bool = True):
    """ssm_dos: (dos_ss, dos_kpm, rank) at the sweep points t."""
    lib = N.load()
    tb, tp = _as_buffer(t, np.float64)
    n_t = int(tb.shape[0])
    ss, ssp = _empty_like_input(t, (n_t,), np.float64) if want_ss else (None, None)
    kp, kpp = _empty_like_input(t, (n_t,), np.float64) if want_kpm else (None, None)
    rk, rkp = _empty_like_input(t, (n_t, 2), np.int32) if want_rank else (None, None)
    _check(lib, lib.ssm_dos(plan.handle, tp, n_t, float(sigma), ssp, kpp, rkp), plan.handle)
    return ss, kp, rk


def ssm_dos_explicit(plan: Plan, W, t, sigma: float, want_rank: bool = True):
    """ssm_dos_explicit: (dos, rank) of SS-DGC (Alg. 5) with probes W at the sweep points t."""
    lib = N.load()
    Wb, Wp = _as_buffer(W, np.float64)
    tb, tp = _as_buffer(t, np.float64)
    n_t = int(tb.shape[0])
    ds, dsp = _empty_like_input(t, (n_t,), np.float64)
    rk, rkp = _empty_like_input(t, (n_t, 2), np.int32) if want_rank else (None, None)
    _check(lib, lib.ssm_dos_explicit(plan.handle, Wp, Wb.shape[1], tp, n_t, float(sigma), dsp, rkp), plan.handle)
    return ds, rk


def ssm_coefficients(plan: Plan, t, sigma: float):
    """ssm_coefficients: (mu, nu), each n_t x (M+1)."""
    lib = N.load()
    tb, tp = _as_buffer(t, np.float64)
    n_t = int(tb.shape[0])
    mu, mup = _empty_like_input(t, (n_t, plan.degree + 1), np.float64)
    nu, nup = _empty_like_input(t, (n_t, plan.degree + 1), np.float64)
    _check(lib, lib.ssm_coefficients(plan.handle, tp, n_t, float(sigma), mup, nup), plan.handle)
    return mu, nu


def ssm_trace_f(plan: Plan, f: Callable[[float], float], n_t: int, sigma: float,
                sigma_tilde: float = 0.016, a: float = 0.93) -> Tuple[float, float]:
    """ssm_trace_f: (Tr f(A) from the RESS-DGC DOS, from the KPM DOS)."""
    lib = N.load()
    cb = N.TRACE_FN(lambda x, ctx: float(f(x)))
    tr_ss, tr_kpm = C.c_double(), C.c_double()
    _check(lib, lib.ssm_trace_f(plan.handle, cb, None, int(n_t), float(sigma), float(sigma_tilde), float(a),
                                C.byref(tr_ss), C.byref(tr_kpm)), plan.handle)
    return tr_ss.value, tr_kpm.value


def ssm_trace_weights(plan: Plan, f: Callable[[float], float], n_t: int, sigma: float,
                      sigma_tilde: float = 0.016, a: float = 0.93, device=None):
    """ssm_trace_weights: (x, w) with Tr f(A) ~= sum_i w_i phi_KPM(x_i) (Alg. 8's quadrature)."""
    lib = N.load()
    cb = N.TRACE_FN(lambda x, ctx: float(f(x)))
    ref = torch.empty(0, device=device) if (device is not None and torch is not None) else None
    x, xp = _empty_like_input(ref, (int(n_t),), np.float64)
    w, wp = _empty_like_input(ref, (int(n_t),), np.float64)
    _check(lib, lib.ssm_trace_weights(plan.handle, cb, None, int(n_t), float(sigma), float(sigma_tilde), float(a),
                                      xp, wp), plan.handle)
    return x, w


def ssm_plan_set_diag(plan: Plan, diag):
    """ssm_plan_set_diag: replace a stencil operator's diagonal (the interval (a, b) stays)."""
    lib = N.load()
    db, dp = _as_buffer(diag, np.float64)
    _check(lib, lib.ssm_plan_set_diag(plan.handle, dp), plan.handle)


def ssm_kpm_adjoint(plan: Plan, t, sigma: float, w):
    """ssm_kpm_adjoint: g_l = sum_i w_i mu_l(t_i) / n_tot (dL/dX_l = g_l I), M+1 values."""
    lib = N.load()
    tb, tp = _as_buffer(t, np.float64)
    wb, wp = _as_buffer(w, np.float64)
    n_t = int(tb.shape[0])
    if int(wb.shape[0]) != n_t:
        raise ValueError("t and w must have the same length")
    g, gp = _empty_like_input(t, (plan.degree + 1,), np.float64)
    _check(lib, lib.ssm_kpm_adjoint(plan.handle, tp, n_t, float(sigma), wp, gp), plan.handle)
    return g


def ssm_moments_adjoint(plan: Plan, dL_dX):
    """ssm_moments_adjoint: (dL/d diag, dL/d offdiag) from dL/dX_l.

    dL_dX of shape (M+1,) means G_l = dL_dX[l] I (kind 1); shape (M+1, n_tot, n_tot)
    gives the matrices (kind 0).  dL/d offdiag has 3 entries for a stencil plan
    (per axis) and nnz entries for a CSR plan (per stored entry).
    """
    lib = N.load()
    gb, gp = _as_buffer(dL_dX, np.float64)
    shp = tuple(gb.shape)
    if shp == (plan.degree + 1,):
        kind = 1
    elif shp == (plan.degree + 1, plan.n_tot, plan.n_tot):
        kind = 0
    else:
        raise ValueError(f"dL_dX must have shape ({plan.degree + 1},) or "
                         f"({plan.degree + 1}, {plan.n_tot}, {plan.n_tot}), got {shp}")
    dd, ddp = _empty_like_input(dL_dX, (plan.n,), np.float64)
    do, dop = _empty_like_input(dL_dX, (3 if plan.is_stencil else plan.nnz,), np.float64)
    _check(lib, lib.ssm_moments_adjoint(plan.handle, gp, kind, ddp, dop), plan.handle)
    return dd, do


def ssm_gram_pair(A, B=None, stream=None):
    """ssm_gram_pair: (A^T A, A^T B) of CUDA float64 blocks (rows x cols, row-major)."""
    lib = N.load()
    if not (_is_cuda(A) and (B is None or _is_cuda(B))):
        raise ValueError("ssm_gram_pair takes CUDA tensors")
    A = A.contiguous()
    n_rows, n_cols = A.shape
    gaa = torch.empty((n_cols, n_cols), dtype=torch.float64, device=A.device)
    gab = None
    bptr = None
    if B is not None:
        B = B.contiguous()
        if B.shape != A.shape:
            raise ValueError("A and B must have the same shape")
        gab = torch.empty_like(gaa)
        bptr = B.data_ptr()
    _check(lib, lib.ssm_gram_pair(A.data_ptr(), bptr, n_rows, n_cols, n_cols, gaa.data_ptr(),
                                  None if gab is None else gab.data_ptr(), _stream(stream)), None)
    return gaa, gab


def ssm_debug_explicit_chunk(max_points: int):
    """ssm_debug_explicit_chunk: cap on the sweep points ssm_dos_explicit holds at a time (0: none)."""
    lib = N.load()
    _check(lib, lib.ssm_debug_explicit_chunk(int(max_points)), None)


def ssm_debug_fail_alloc(after: int):
    """ssm_debug_fail_alloc: the device allocation that finds `after` earlier ones counted
    down fails with SSM_ENOMEM (-1 disables)."""
    lib = N.load()
    _check(lib, lib.ssm_debug_fail_alloc(int(after)), None)


def ssm_selftest_wait(polls: int, arrive: bool, stream=None):
    """ssm_selftest_wait: the library's bounded mbarrier wait on its own (raises SSMError
    with SSM_ETIMEOUT when the wait gives up)."""
    lib = N.load()
    _check(lib, lib.ssm_selftest_wait(int(polls), 1 if arrive else 0, _stream(stream)), None)


def ssm_timing_enable(plan: Plan, on: bool = True):
    lib = N.load()
    _check(lib, lib.ssm_timing_enable(plan.handle, 1 if on else 0), plan.handle)


def ssm_stats_get(plan: Plan) -> dict:
    lib = N.load()
    s = N.ssm_stats()
    _check(lib, lib.ssm_stats_get(plan.handle, C.byref(s)), plan.handle)
    return {name: getattr(s, name) for name, _ in N.ssm_stats._fields_}


def ssm_stats_reset(plan: Plan):
    lib = N.load()
    _check(lib, lib.ssm_stats_reset(plan.handle), plan.handle)


def ssm_plan_destroy(plan: Plan):
    plan.close()
