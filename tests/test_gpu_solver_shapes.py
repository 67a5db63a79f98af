"""Per-point solver (Alg. 4 + Alg. 6) at the probe counts where its CTA shape
changes, against the oracle.

The solver runs 64-thread CTAs up to n_v = 64, 128 threads up to 128 and 256
above; tile products, bisection lane groups and the back-transform take a
different shape in each.  These cases run n_v = 100, 128, 129, 200 and 256
(and 150 + 50 hybrid columns) on a 48 x 48 periodic Anderson model with
sweep points from well below to well above the spectrum, so that every route
occurs: nothing kept (outside the spectrum), everything kept (inside it, more
eigenvalues under the Gaussian than probes), part kept with many or few
directions dropped (duplicated probe columns make two directions exactly
null), and the step-by-step route with the hybrid correction.  A two-band
operator with a resolved expansion adds points inside a spectral gap, where
nothing is kept.

Tolerance (float64 plans): max(1e-10, 10 x the relative L1 spread between the
oracle's own two float64 evaluations, the paper's M-step loop and the
doubling products), on the points the oracle does not flag as within 1e-8 of
an Alg. 4 threshold; kept ranks must be equal there.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402
from oracle import ssm_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [(100, 0, False), (128, 0, True), (129, 0, False), (200, 0, False), (256, 0, True),
         (200, 0, True), (150, 50, False)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1504_07690_gb300 as S

    return S


@pytest.mark.parametrize("nv,nvh,dup", CASES, ids=[f"{a}+{b}{'-dup' if d else ''}" for a, b, d in CASES])
def test_solver_routes_at_large_probe_counts(S, nv, nvh, dup):
    st = wl.anderson2d(48, 4800 + nv)
    csr = wl.stencil_to_csr(st)
    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    W = wl.random_block(csr.n, nv + nvh, 4900 + nv, "rademacher")
    if dup:
        W[:, 1] = W[:, 0]
        W[:, 3] = W[:, 2]
    M, sigma = 80, 0.3
    plan = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M)
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"] - 2.5, info["hi"] + 2.5, 71)
    S.ssm_moments(plan, torch.from_numpy(W).cuda())
    ss, kpm, rank = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(t).cuda(), sigma))
    kw = dict(interval=(info["a"], info["b"]), flag_eps=1e-8)
    r = O.ress_dgc(A, W, nv, t, M, sigma, **kw)
    r2 = O.ress_dgc(A, W, nv, t, M, sigma, moments="doubling", **kw)
    ok = ~r["flagged"] & ~r2["flagged"]
    assert ok.sum() >= 0.9 * ok.size
    rs = r["rank_s"]
    # the routes this case is meant to reach
    assert np.sum((rs > 0) & (rs < nv)) > 0
    if not dup:
        assert np.sum(rs == nv) > 0
    if dup:
        assert np.sum((rs > 0) & (3 * (nv - rs) < rs)) > 0
    tol = max(1e-10, 10.0 * O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok]))
    assert tol <= 1e-7
    err = O.relative_l1_error(ss[ok], r["dos_ss"][ok])
    assert err <= tol, (err, tol)
    assert np.array_equal(rank[ok, 0], rs[ok])
    assert np.array_equal(rank[ok, 1], r["rank_xi"][ok])
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= 1e-10


def test_solver_keeps_nothing_inside_a_spectral_gap(S):
    # Two bands (on-site energies near -4 and +4, weak hopping) with a gap of width
    # ~6 between them and a resolved expansion (M/2 sigma~ ~ 13): inside the gap
    # K_W(t) is rounding noise and the solver keeps nothing; at the band centres it
    # keeps every direction or part of them.
    rng = np.random.default_rng(4801)
    nx = 32
    diag = np.where(rng.uniform(size=nx * nx) < 0.5, -4.0, 4.0) + rng.uniform(-0.5, 0.5, nx * nx)
    st = wl.Stencil(dims=(nx, nx, 1), periodic=(True, True, False), diag=diag, offdiag=(-0.25, -0.25, 0.0))
    csr = wl.stencil_to_csr(st)
    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    nv = 200
    W = wl.random_block(csr.n, nv, 4902, "rademacher")
    M, sigma = 1600, 0.1
    plan = S.ssm_plan_create(stencil=st, n_v=nv, degree=M)
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], 41)
    S.ssm_moments(plan, torch.from_numpy(W).cuda())
    ss, kpm, rank = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(t).cuda(), sigma))
    kw = dict(interval=(info["a"], info["b"]), flag_eps=1e-8)
    r = O.ress_dgc(A, W, nv, t, M, sigma, **kw)
    r2 = O.ress_dgc(A, W, nv, t, M, sigma, moments="doubling", **kw)
    ok = ~r["flagged"] & ~r2["flagged"]
    assert ok.sum() >= 0.6 * ok.size  # the band edges sit near the rounding floor
    rs = r["rank_s"]
    assert np.sum(rs[ok] == 0) >= 5 and np.sum((rs > 0) & (rs < nv)) > 0
    tol = max(1e-10, 10.0 * O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok]))
    assert tol <= 1e-6
    assert O.relative_l1_error(ss[ok], r["dos_ss"][ok]) <= tol
    assert np.array_equal(rank[ok, 0], rs[ok])
    assert np.all(ss[ok & (rs == 0)] == 0.0)
