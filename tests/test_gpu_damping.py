"""Jackson / Lorentz damping of the series (options of the KPM literature the
paper's KPM remark cites; the paper uses none): CUDA path vs the oracle.

Tolerances as in test_gpu_parity.py: coefficient tables 1e-12 of their max,
KPM DOS 1e-10 relative L1, RESS-DGC DOS max(1e-10, 10 x the oracle's own
direct-vs-doubling spread) on unflagged points, kept ranks equal.
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


@pytest.mark.parametrize("damping,kind", [("jackson", 1), ("lorentz", 2)])
def test_damped_coefficients_kpm_and_ss_fp64(S, damping, kind):
    st = wl.make_operator("lap2d_dirichlet_32")
    c = wl.CONFIGS["lap2d_dirichlet_32"]
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    plan = S.ssm_plan_create(stencil=st, n_v=c["n_v"], degree=c["M"], damping=damping)
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], c["n_t"])
    mu, nu = S.ssm_coefficients(plan, t, c["sigma"])
    S.ssm_moments(plan, torch.from_numpy(W).cuda())
    ss, kpm, rank = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(t).cuda(), c["sigma"]))
    csr = wl.stencil_to_csr(st)
    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    kw = dict(interval=(info["a"], info["b"]), flag_eps=1e-8, damping=kind)
    r = O.ress_dgc(A, W, c["n_v"], t, c["M"], c["sigma"], **kw)
    assert np.max(np.abs(mu - r["mu_full"])) <= 1e-12 * np.max(np.abs(r["mu_full"]))
    assert np.max(np.abs(nu - r["nu"])) <= 1e-12 * np.max(np.abs(r["nu"]))
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= 1e-10
    r2 = O.ress_dgc(A, W, c["n_v"], t, c["M"], c["sigma"], moments="doubling", **kw)
    ok = ~r["flagged"] & ~r2["flagged"]
    assert ok.sum() >= 0.9 * ok.size
    tol = max(1e-10, 10.0 * O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok]))
    assert O.relative_l1_error(ss[ok], r["dos_ss"][ok]) <= tol
    assert np.array_equal(rank[ok, 0], r["rank_s"][ok])
    # damping changes the estimate (the factors reach the kernels)
    r0 = O.ress_dgc(A, W, c["n_v"], t, c["M"], c["sigma"], interval=(info["a"], info["b"]))
    assert O.relative_l1_error(kpm, r0["dos_kpm"]) > 1e-6


def test_bad_damping_is_rejected(S):
    st = wl.make_operator("lap2d_dirichlet_32", nx=8)
    with pytest.raises(S.SSMError) as e:
        S.ssm_plan_create(stencil=st, n_v=4, degree=10, damping=3)
    assert e.value.name == "SSM_EINVAL"
