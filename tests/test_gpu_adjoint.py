"""Adjoint of the moment recurrence on the GPU vs the adjoint oracle.

ssm_moments_adjoint (reverse of the doubling loop, checkpointed) against
oracle/adjoint_oracle.py (reverse of the paper's M-step loop, everything
stored), element by element:
* float64: dL/d diag, dL/d offdiag (stencil, per axis) and dL/dA_ij (CSR,
  per stored entry) within 1e-10 of the largest entry, for general G_l and
  for G_l = g_l I;
* float32 recurrence (mixed plans, separate or fused recurrence + Gram steps):
  within 1e-4 of the largest entry;
* the dense-eigh closed form (W = sqrt(N) I, G_l = g_l I);
* the autograd Function against central finite differences of its own
  float64 forward pass (KPM loss plus Tr exp(-A) by Alg. 8's weights).
Segments of ceil(sqrt(S)) steps with a ragged last one are covered by S = 13.
"""
import dataclasses
import math

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import adjoint_oracle as AO  # noqa: E402
from oracle import ssm_oracle as O  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1504_07690_gb300 as S

    return S


def _stencil_pattern(st):
    """A's pattern plus every axis's couplings (for axes whose coupling is zero)."""
    n = st.n
    P = abs(_csr(wl.stencil_to_csr(st))) + sp.identity(n, format="csr")
    for d in range(3):
        off = [0.0, 0.0, 0.0]
        off[d] = 1.0
        P = P + abs(_csr(wl.stencil_to_csr(dataclasses.replace(st, diag=np.zeros(n), offdiag=tuple(off)))))
    P = sp.csr_matrix(P)
    P.data[:] = 1.0
    return P


def _csr(c):
    return O.csr_matrix(c.n, c.rowptr, c.colind, c.val)


def _oracle_stencil(st, W, M, G, a, b):
    A = _csr(wl.stencil_to_csr(st))
    At = O.transform(A, a, b)
    d, pat = AO.moments_adjoint_direct(At, W, M, G, pattern=_stencil_pattern(st))
    gd, go = AO.stencil_parameter_grad(AO.grad_wrt_a(pat, a, b), AO.grad_wrt_a(d, a, b), st, wl.stencil_to_csr)
    return gd, go


def _gpu(S, plan, W, G):
    S.ssm_moments(plan, torch.from_numpy(W).cuda())
    dd, do = S.ssm_moments_adjoint(plan, torch.from_numpy(np.ascontiguousarray(G)).cuda())
    return dd.cpu().numpy(), do.cpu().numpy()


STENCILS = [
    ("dirichlet_2d", lambda: wl.Stencil(dims=(1, 9, 11), periodic=(False, False, False),
                                        diag=4.0 + np.random.default_rng(1).uniform(-1, 1, 99),
                                        offdiag=(0.0, -1.0, -1.0))),
    ("periodic_3d_mixed", lambda: wl.Stencil(dims=(2, 5, 6), periodic=(True, False, True),
                                             diag=6.0 + np.random.default_rng(2).uniform(-1, 1, 60),
                                             offdiag=(-0.8, -1.0, -1.2))),
    ("self_loop_axis", lambda: wl.Stencil(dims=(1, 7, 8), periodic=(True, True, False),
                                          diag=np.random.default_rng(3).uniform(-1, 1, 56),
                                          offdiag=(-0.5, -1.0, -1.0))),
]


@pytest.mark.parametrize("name,make", STENCILS, ids=[s[0] for s in STENCILS])
@pytest.mark.parametrize("kind", ["matrices", "scalars"])
def test_stencil_adjoint_fp64(S, name, make, kind):
    st = make()
    n_tot, M = 6, 26
    rng = np.random.default_rng(11)
    W = rng.standard_normal((st.n, n_tot))
    if kind == "matrices":
        G = rng.standard_normal((M + 1, n_tot, n_tot))
        Gin = G
    else:
        g = rng.standard_normal(M + 1)
        G = g[:, None, None] * np.eye(n_tot)[None]
        Gin = g
    plan = S.ssm_plan_create(stencil=st, n_v=n_tot, degree=M, precision="fp64", options=2)
    info = S.ssm_plan_info(plan)
    dd, do = _gpu(S, plan, W, Gin)
    gd, go = _oracle_stencil(st, W, M, G, info["a"], info["b"])
    scale = max(np.max(np.abs(gd)), np.max(np.abs(go)))
    assert np.max(np.abs(dd - gd)) <= 1e-10 * scale
    assert np.max(np.abs(do - go)) <= 1e-10 * scale, (do, go)


def test_csr_adjoint_fp64_per_entry(S):
    csr = wl.er_normalized_laplacian(300, 6.0, 5)
    n_tot, M = 5, 22
    rng = np.random.default_rng(12)
    W = rng.standard_normal((csr.n, n_tot))
    G = rng.standard_normal((M + 1, n_tot, n_tot))
    plan = S.ssm_plan_create(csr=csr, n_v=n_tot, degree=M, precision="fp64", options=2)
    info = S.ssm_plan_info(plan)
    dd, dval = _gpu(S, plan, W, G)
    A = _csr(csr)
    At = O.transform(A, info["a"], info["b"])
    d, pat = AO.moments_adjoint_direct(At, W, M, G)
    gd = AO.grad_wrt_a(d, info["a"], info["b"])
    gp = AO.grad_wrt_a(AO.symmetric_part(pat), info["a"], info["b"])
    # the oracle's pattern is A's (sorted, duplicates summed) = the input CSR order
    assert np.array_equal(gp.indptr, csr.rowptr) and np.array_equal(gp.indices, csr.colind)
    scale = max(np.max(np.abs(gd)), np.max(np.abs(gp.data)))
    assert np.max(np.abs(dd - gd)) <= 1e-10 * scale
    assert np.max(np.abs(dval - gp.data)) <= 1e-10 * scale


@pytest.mark.parametrize("options", [2, 6], ids=["separate", "fused-step"])
def test_stencil_adjoint_mixed(S, options):
    st = STENCILS[1][1]()
    n_tot, M = 8, 26
    rng = np.random.default_rng(13)
    W = rng.standard_normal((st.n, n_tot))
    G = rng.standard_normal((M + 1, n_tot, n_tot))
    plan = S.ssm_plan_create(stencil=st, n_v=n_tot, degree=M, precision="mixed", options=options)
    info = S.ssm_plan_info(plan)
    dd, do = _gpu(S, plan, W, G)
    gd, go = _oracle_stencil(st, W, M, G, info["a"], info["b"])
    scale = max(np.max(np.abs(gd)), np.max(np.abs(go)))
    assert np.max(np.abs(dd - gd)) <= 1e-4 * scale
    assert np.max(np.abs(do - go)) <= 1e-4 * scale


def test_adjoint_dense_eigh_closed_form(S):
    st = wl.Stencil(dims=(1, 6, 6), periodic=(False, True, False),
                    diag=np.random.default_rng(4).uniform(-1, 1, 36), offdiag=(0.0, -1.0, -1.0))
    n = st.n
    M = 30
    W = math.sqrt(n) * np.eye(n)
    g = np.random.default_rng(6).standard_normal(M + 1)
    plan = S.ssm_plan_create(stencil=st, n_v=n, degree=M, precision="fp64", options=2)
    info = S.ssm_plan_info(plan)
    dd, _ = _gpu(S, plan, W, g)
    At = O.transform(_csr(wl.stencil_to_csr(st)), info["a"], info["b"]).toarray()
    lam, Q = np.linalg.eigh(At)
    dp = np.polynomial.chebyshev.chebval(lam, np.polynomial.chebyshev.chebder(g))
    ref = n * np.einsum("ij,j,ij->i", Q, dp, Q) * (2.0 / (info["b"] - info["a"]))
    assert np.max(np.abs(dd - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_adjoint_requires_option_and_moments(S):
    st = STENCILS[0][1]()
    plan = S.ssm_plan_create(stencil=st, n_v=4, degree=10, precision="fp64")
    S.ssm_moments(plan, torch.ones(st.n, 4, dtype=torch.float64, device="cuda"))
    with pytest.raises(S.SSMError, match="ESTATE"):
        S.ssm_moments_adjoint(plan, np.zeros(11))
    plan2 = S.ssm_plan_create(stencil=st, n_v=4, degree=10, precision="fp64", options=2)
    with pytest.raises(S.SSMError, match="ESTATE"):
        S.ssm_moments_adjoint(plan2, np.zeros(11))
    S.ssm_moments(plan2, torch.ones(st.n, 4, dtype=torch.float64, device="cuda"))
    bad = np.zeros(11)
    bad[3] = np.nan
    with pytest.raises(S.SSMError, match="ENONFINITE"):
        S.ssm_moments_adjoint(plan2, bad)


def test_set_diag_rejects_leaving_the_interval(S):
    st = STENCILS[0][1]()
    plan = S.ssm_plan_create(stencil=st, n_v=4, degree=10, precision="fp64")
    with pytest.raises(S.SSMError, match="EDOMAIN"):
        S.ssm_plan_set_diag(plan, st.diag + 100.0)
    bad = st.diag.copy()
    bad[0] = np.inf
    with pytest.raises(S.SSMError, match="ENONFINITE"):
        S.ssm_plan_set_diag(plan, bad)


def test_autograd_kpm_and_trace_vs_finite_differences(S):
    base = wl.Stencil(dims=(1, 8, 9), periodic=(False, True, False), diag=np.full(72, 4.0),
                      offdiag=(0.0, -1.0, -1.0))
    rng = np.random.default_rng(21)
    v0 = rng.normal(0.0, 0.3, base.n)
    # interval wide enough for every potential the finite differences visit
    plan = S.ssm_plan_create(stencil=dataclasses.replace(base, diag=base.diag + v0), n_v=16, degree=40,
                             precision="fp64", lo=-3.0, hi=12.0, options=2)
    W = torch.from_numpy(wl.random_block(base.n, 16, 7, "gaussian")).cuda()
    sigma = 0.3
    t = torch.linspace(0.5, 8.5, 60, dtype=torch.float64, device="cuda")
    dt = float(t[1] - t[0])
    target = torch.from_numpy(0.01 * np.exp(-((np.linspace(0.5, 8.5, 60) - 4.0) ** 2) / 4.0)).cuda()
    xw, ww = S.ssm_trace_weights(plan, lambda x: math.exp(-x), 128, 0.05, 0.016, 0.93, device="cuda")
    tt = torch.cat([t, xw])

    def loss_of(v):
        phi = S.KPMDensity.apply(v, plan, W, tt, sigma)
        return ((phi[:60] - target) ** 2).sum() * dt + (ww * phi[60:]).sum()

    v = torch.from_numpy(base.diag + v0).cuda().requires_grad_(True)
    L = loss_of(v)
    L.backward()
    grad = v.grad.detach().cpu().numpy()
    with torch.no_grad():
        for i in (0, 17, 40, 71):
            h = 1e-4
            e = torch.zeros_like(v)
            e[i] = h
            fd = (float(loss_of(v + e)) - float(loss_of(v - e))) / (2 * h)
            assert abs(grad[i] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(grad))), (i, grad[i], fd)
