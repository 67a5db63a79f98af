"""SS-DGC with explicit filtered blocks (Alg. 5): CUDA path vs the CPU oracle.

ssm_dos_explicit forms Z(t_i) = sum_{l<=M} mu_l(t_i) T_l(A~) W in float64 and
solves (Z^T Z, W^T Z) at every point by Alg. 4.  As for RESS-DGC, Alg. 4
divides by eigenvalues of K_W(t) down to tau = 1e-7 of the largest, so
rounding differences are amplified; the tolerance is max(1e-10, 10 x spread),
spread = the relative L1 difference between two float64 evaluations of the
same estimator by the oracle: Alg. 5 at degree M and RESS-DGC at degree 2M,
which form the same pencil (K_W of degree M, K_Z = its square) in exact
arithmetic.  Kept ranks must agree on the points neither oracle run flags as
within 1e-8 of an Alg. 4 threshold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import ssm_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1504_07690_gb300 as S

    return S


def _A(op):
    c = wl.stencil_to_csr(op) if isinstance(op, wl.Stencil) else op
    return O.csr_matrix(c.n, c.rowptr, c.colind, c.val)


def _gpu(S, op, W, M, sigma, t=None, n_t=0, kind="stencil", **kw):
    key = "stencil" if kind == "stencil" else "csr"
    plan = S.ssm_plan_create(**{key: op}, n_v=W.shape[1], degree=M, precision="fp64", **kw)
    info = S.ssm_plan_info(plan)
    if t is None:
        t = np.linspace(info["lo"], info["hi"], n_t)
    dos, rank = S.ssm_dos_explicit(plan, torch.from_numpy(W).cuda(), torch.from_numpy(t).cuda(), sigma)
    plan.close()
    return dos.cpu().numpy(), rank.cpu().numpy(), t, info


def _check(op, W, M, sigma, t, info, dos, rank, estimator="alg4", damping=0):
    A = _A(op)
    iv = (info["a"], info["b"])
    r = O.ss_dgc(A, W, t, M, sigma, interval=iv, flag_eps=1e-8, estimator=estimator, damping=damping)
    r2 = O.ress_dgc(A, W, W.shape[1], t, 2 * M, sigma, interval=iv, flag_eps=1e-8, estimator=estimator,
                    damping=damping, moments="doubling") if damping == 0 else None
    ok = ~r["flagged"]
    if r2 is not None:
        ok &= ~r2["flagged"]
        spread = O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok])
    else:
        spread = 0.0
    tol = max(1e-10, 10.0 * spread)
    assert ok.mean() >= 0.9
    assert np.array_equal(rank[ok, 0], r["rank_s"][ok])
    if estimator == "alg4":
        assert np.array_equal(rank[ok, 1], r["rank_xi"][ok])
    err = O.relative_l1_error(dos[ok], r["dos_ss"][ok])
    assert err <= tol, (err, tol)
    return err


def test_config1_shape_matches_oracle(S):
    # the 32 x 32 Dirichlet Laplacian with potential: N = 1024, N_v = 40, M = 200, 101 points
    c = wl.CONFIGS["lap2d_dirichlet_32"]
    st = wl.make_operator("lap2d_dirichlet_32")
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    dos, rank, t, info = _gpu(S, st, W, c["M"], c["sigma"], n_t=c["n_t"])
    _check(st, W, c["M"], c["sigma"], t, info, dos, rank)


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_ragged_shapes_match_oracle(S, kind):
    # odd grid and odd N_v (the block's padded leading dimension), M not a multiple
    # of the eight blocks one accumulation takes, points outside the spectrum too
    st = wl.laplacian2d_dirichlet_potential(23, 77)
    op = st if kind == "stencil" else wl.stencil_to_csr(st)
    W = wl.random_block(st.n, 13, 78)
    M, sigma = 62, 0.15
    info_plan = S.ssm_plan_create(stencil=st, n_v=13, degree=M, precision="fp64")
    info = S.ssm_plan_info(info_plan)
    info_plan.close()
    t = np.linspace(info["lo"] - 0.5, info["hi"] + 0.5, 37)
    dos, rank, _, info = _gpu(S, op, W, M, sigma, t=t, kind=kind)
    _check(op, W, M, sigma, t, info, dos, rank)


def test_pinv_and_damping_match_oracle(S):
    st = wl.laplacian2d_dirichlet_potential(16, 81)
    W = wl.random_block(st.n, 24, 82)
    M, sigma = 120, 0.1
    dos, rank, t, info = _gpu(S, st, W, M, sigma, n_t=41, options=8)
    _check(st, W, M, sigma, t, info, dos, rank, estimator="pinv")
    dos, rank, t, info = _gpu(S, st, W, M, sigma, n_t=41, damping="jackson")
    _check(st, W, M, sigma, t, info, dos, rank, damping=1)


def test_host_buffers_and_single_point(S):
    st = wl.laplacian2d_dirichlet_potential(12, 83)
    W = wl.random_block(st.n, 9, 84)
    plan = S.ssm_plan_create(stencil=st, n_v=9, degree=40, precision="fp64")
    info = S.ssm_plan_info(plan)
    t = np.array([0.5 * (info["lo"] + info["hi"])])
    dos_h, rank_h = S.ssm_dos_explicit(plan, W, t, 0.2)  # host arrays in, host arrays out
    dos_d, rank_d = S.ssm_dos_explicit(plan, torch.from_numpy(W).cuda(), torch.from_numpy(t).cuda(), 0.2)
    plan.close()
    assert isinstance(dos_h, np.ndarray)
    assert np.array_equal(dos_h, dos_d.cpu().numpy())
    assert np.array_equal(rank_h, rank_d.cpu().numpy())
    _check(st, W, 40, 0.2, t, info, dos_h, rank_h)


def test_chunks_of_points_give_the_same_result(S):
    # the filtered blocks of 3 points at a time (the recurrence reruns per chunk): every
    # point's arithmetic is the same as with all points at once, so the results agree
    # bit for bit; then against the oracle
    st = wl.laplacian2d_dirichlet_potential(14, 86)
    W = wl.random_block(st.n, 11, 87)
    M, sigma = 50, 0.15
    plan = S.ssm_plan_create(stencil=st, n_v=11, degree=M, precision="fp64")
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], 11)
    Wd, td = torch.from_numpy(W).cuda(), torch.from_numpy(t).cuda()
    d_all, r_all = S.ssm_dos_explicit(plan, Wd, td, sigma)
    try:
        S.ssm_debug_explicit_chunk(3)
        d_chk, r_chk = S.ssm_dos_explicit(plan, Wd, td, sigma)
    finally:
        S.ssm_debug_explicit_chunk(0)
    plan.close()
    assert torch.equal(d_all, d_chk) and torch.equal(r_all, r_chk)
    _check(st, W, M, sigma, t, info, d_chk.cpu().numpy(), r_chk.cpu().numpy())


def test_rejects_plans_it_does_not_serve(S):
    st = wl.laplacian2d_dirichlet_potential(12, 85)
    W = torch.zeros((st.n, 8), dtype=torch.float64, device="cuda")
    t = torch.zeros(3, dtype=torch.float64, device="cuda")
    for kw in (dict(precision="mixed", n_v=8), dict(precision="fp64_tc", n_v=8),
               dict(precision="fp64", n_v=4, n_vh=4)):
        plan = S.ssm_plan_create(stencil=st, degree=20, **kw)
        with pytest.raises(S.SSMError):
            S.ssm_dos_explicit(plan, W, t, 0.1)
        plan.close()


def test_benchmark_shape_sampled_points(S):
    # the 2D Anderson model of the benchmark (N = 65536, N_v = 200 Rademacher,
    # M = 1000) at the 16 sweep points the bench times; three of them are
    # recomputed by the oracle, which forms every point independently.  The
    # tolerance is that of the float64 RESS-DGC DOS at this shape (its measured
    # oracle spread is ~1e-10 and its GPU error ~1e-9) with a margin of ten.
    c = wl.CONFIGS["anderson2d_256"]
    st = wl.make_operator("anderson2d_256")
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    plan = S.ssm_plan_create(stencil=st, n_v=c["n_v"], degree=c["M"], precision="fp64")
    info = S.ssm_plan_info(plan)
    plan.close()
    t = wl.explicit_points(info["lo"], info["hi"])
    dos, rank, _, info = _gpu(S, st, W, c["M"], c["sigma"], t=t)
    pick = np.array([3, 8, 12])
    r = O.ss_dgc(_A(st), W, t[pick], c["M"], c["sigma"], interval=(info["a"], info["b"]), flag_eps=1e-8)
    ok = ~r["flagged"]
    assert ok.sum() >= 2
    assert np.array_equal(rank[pick][ok, 0], r["rank_s"][ok])
    err = O.relative_l1_error(dos[pick][ok], r["dos_ss"][ok])
    assert err <= 1e-8, err
    assert np.all(np.isfinite(dos)) and np.all(dos >= -1e-12)
