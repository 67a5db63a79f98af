"""Float64-accuracy plans with tensor-core Gram products (SSM_FP64_TC) against
the oracle.

The Gram products are exact sums of bf16 slice products (six 8-bit digits of
a per-column fixed point, about 2^-48 of each column's largest entry), so the
moments must agree with the oracle as closely as the CUDA-core float64
plan's do: 1e-11 of max |X| (the doubling products and the paper's M-step
loop differ by rounding only).  The DOS lines use the float64 plan's
tolerances: KPM 1e-10 relative L1; RESS-DGC max(1e-10, 10 x the spread
between the oracle's own two float64 evaluations) on unflagged points, with
equal kept ranks.
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


# n_tot: one tile below 128 (ragged), exactly 128, three tiles just past 128, the
# benchmark's 200, the largest 256; N not a multiple of the 16-row stage
SHAPES = [(12, 0, 23), (37, 0, 31), (128, 0, 40), (100, 29, 33), (150, 50, 45), (256, 0, 37), (5, 3, 3)]


@pytest.mark.parametrize("nv,nvh,nx", SHAPES, ids=[f"{a}+{b}-N{c * c}" for a, b, c in SHAPES])
def test_fp64tc_moments_match_oracle(S, nv, nvh, nx):
    st = wl.anderson2d(nx, 700 + nx)
    n_tot = nv + nvh
    W = wl.random_block(st.n, n_tot, 701 + nx, "rademacher")
    M = 40
    plan = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M, precision="fp64_tc")
    info = S.ssm_plan_info(plan)
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    ref = O.moments_direct(O.transform(_A(st), info["a"], info["b"]), W, M)
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(X - ref)) / scale
    assert err <= 1e-11, err
    assert np.array_equal(X, np.transpose(X, (0, 2, 1)))
    # repeatable to the bit
    X2 = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    assert np.array_equal(X, X2)


def test_fp64tc_gaussian_probes_with_large_entries(S):
    # Gaussian probes scaled by 1e3 in some columns and 1e-3 in others: the per-column
    # scales keep every column at the same relative accuracy
    st = wl.make_operator("lap2d_dirichlet_32", nx=24)
    W = wl.random_block(st.n, 40, 55)
    W[:, :10] *= 1e3
    W[:, 30:] *= 1e-3
    M = 30
    plan = S.ssm_plan_create(stencil=st, n_v=40, degree=M, precision="fp64_tc")
    info = S.ssm_plan_info(plan)
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    ref = O.moments_direct(O.transform(_A(st), info["a"], info["b"]), W, M)
    d = np.sqrt(np.abs(np.diagonal(ref[0])))
    rel = np.abs(X - ref) / (d[None, :, None] * d[None, None, :])
    assert np.max(rel) <= 1e-11, np.max(rel)


def test_fp64tc_config1_dos(S):
    st = wl.make_operator("lap2d_dirichlet_32")
    c = wl.CONFIGS["lap2d_dirichlet_32"]
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    plan = S.ssm_plan_create(stencil=st, n_v=c["n_v"], degree=c["M"], precision="fp64_tc")
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], c["n_t"])
    S.ssm_moments(plan, torch.from_numpy(W).cuda())
    ss, kpm, rank = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(t).cuda(), c["sigma"]))
    A = _A(st)
    kw = dict(interval=(info["a"], info["b"]), flag_eps=1e-8)
    r = O.ress_dgc(A, W, c["n_v"], t, c["M"], c["sigma"], **kw)
    r2 = O.ress_dgc(A, W, c["n_v"], t, c["M"], c["sigma"], moments="doubling", **kw)
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= 1e-10
    ok = ~r["flagged"] & ~r2["flagged"]
    assert ok.sum() >= 0.9 * ok.size
    spread = O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok])
    err = O.relative_l1_error(ss[ok], r["dos_ss"][ok])
    print(f"config 1 fp64_tc: ss err {err:.3e} oracle spread {spread:.3e}")
    assert err <= 1e-7
    assert np.array_equal(rank[ok, 0], r["rank_s"][ok])


def test_fp64tc_csr_hybrid(S):
    csr = wl.er_normalized_laplacian(3000, 8.0, 1104)
    W = wl.random_block(csr.n, 160, 2104)
    M, sigma = 80, 0.05
    plan = S.ssm_plan_create(csr=csr, n_v=120, n_vh=40, degree=M, precision="fp64_tc")
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], 41)
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    ss, kpm, rank = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(t).cuda(), sigma))
    A = _A(csr)
    kw = dict(interval=(info["a"], info["b"]), flag_eps=1e-8)
    r = O.ress_dgc(A, W, 120, t, M, sigma, **kw)
    r2 = O.ress_dgc(A, W, 120, t, M, sigma, moments="doubling", **kw)
    assert np.max(np.abs(X - r["X"])) <= 1e-11 * np.max(np.abs(r["X"]))
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= 1e-10
    ok = ~r["flagged"] & ~r2["flagged"]
    tol = max(1e-10, 10.0 * O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok]))
    assert O.relative_l1_error(ss[ok], r["dos_ss"][ok]) <= tol


def test_fp64tc_rejects_wide_blocks(S):
    st = wl.make_operator("lap2d_dirichlet_32", nx=8)
    with pytest.raises(S.SSMError) as e:
        S.ssm_plan_create(stencil=st, n_v=200, n_vh=57, degree=10, precision="fp64_tc")
    assert e.value.name == "SSM_EINVAL"
