"""The per-point assembly of mixed and float64-accurate plans on the tensor cores.

Single-operator plans of these precisions form K(t) = sum_l mu_l(t) X_l and
K_Z(t) = sum_l nu_l(t) X_l on the tensor cores, as exact products of bf16
slices of the moments and of the coefficients (six slices on mixed plans,
about 2^-47 of each entry's and each point's largest term; seven on SSM_FP64_TC
plans, 2^-55).  To test that step and the solve after it apart
from the rounding of the recurrence, the RESS-DGC line of a plan is compared
with the oracle's Alg. 7 loop run on the plan's own moments (returned by
ssm_moments) with the plan's rounding floor: relative L1 1e-7 on the points the
oracle does not flag as within 1e-8 of an Alg. 4 threshold, equal kept ranks.
Shapes: ragged N_v (odd, below and above one 128-entry tile of the packed
triangle), hybrid blocks (K_Z is a prefix of the packed entries), sweep points
outside the spectrum, more points than one 64-point tile.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import ssm_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu

FLOOR = {"mixed": 2.0 ** -36, "fp64_tc": 2.0 ** -52}


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1504_07690_gb300 as S

    return S


CASES = [("mixed", 13, 0, 120, 70), ("mixed", 40, 0, 200, 101), ("mixed", 21, 10, 80, 130),
         ("mixed", 150, 0, 60, 33), ("mixed", 24, 9, 60, 200), ("fp64_tc", 37, 0, 100, 65),
         ("fp64_tc", 24, 9, 60, 33), ("fp64_tc", 140, 0, 40, 80)]


@pytest.mark.parametrize("precision,nv,nvh,M,n_t", CASES,
                         ids=[f"{p}-{a}+{b}-M{m}-t{t}" for p, a, b, m, t in CASES])
def test_tensor_core_assembly_against_oracle_on_own_moments(S, precision, nv, nvh, M, n_t):
    st = wl.laplacian2d_dirichlet_potential(20, 90 + nv)
    W = wl.random_block(st.n, nv + nvh, 91 + nv, "gaussian")
    sigma = 0.08
    plan = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M, precision=precision)
    info = S.ssm_plan_info(plan)
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    t = np.linspace(info["lo"] - 0.3, info["hi"] + 0.3, n_t)
    ss, kpm, rk = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(t).cuda(), sigma))
    plan.close()
    tab = O.coefficient_tables(t, M, sigma, st.n, info["a"], info["b"])
    r = O.ress_from_moments(X, tab, nv, O.g_max(sigma, st.n), flag_eps=1e-8, eps_floor=FLOOR[precision])
    ok = ~r["flagged"]
    assert ok.mean() >= 0.9
    assert np.array_equal(rk[ok, 0], r["rank_s"][ok])
    assert O.relative_l1_error(ss[ok], r["dos_ss"][ok]) <= 1e-7
    assert O.relative_l1_error(kpm, O.kpm_dos(tab["mu_full"], X)) <= 1e-12
