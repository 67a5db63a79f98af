"""Batched plans (many operators of uneven size in one graph-captured
recurrence) against the oracle run matrix by matrix, and against single-
operator plans of the GPU path.

* float64: every matrix's moments within 1e-11 of max|X| of the oracle's
  M-step loop, KPM DOS within 1e-10 relative L1, RESS-DGC DOS within the
  conditioning-aware tolerance of test_gpu_parity (max(1e-10, 10 x the
  oracle's direct-vs-doubling spread) on unflagged points), kept ranks equal
  to the oracle's there.
* mixed: moments within 2e-5 of max|X| of the float64 oracle (split-bf16
  Gram error) and KPM within 1e-4 relative L1.
Sizes are ragged (not multiples of the 32-row panel) and include an
isolated vertex (an empty row of the normalised Laplacian).
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


def _graphs():
    sizes = [300, 517, 64, 1000, 45]
    return [wl.er_normalized_laplacian(n, 6.0, 40 + k) for k, n in enumerate(sizes)]


def _run(S, csrs, n_v, M, sigma, n_tp, precision):
    plan = S.ssm_plan_create_batched(csrs, n_v=n_v, degree=M, precision=precision)
    Ws = [wl.random_block(c.n, n_v, 77 + k, "rademacher") for k, c in enumerate(csrs)]
    W = np.vstack(Ws)
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    infos = [S.ssm_batch_info(plan, b) for b in range(len(csrs))]
    t = np.concatenate([np.linspace(i["lo"], i["hi"], n_tp) for i in infos])
    ss, kpm, rk = S.ssm_dos(plan, torch.from_numpy(t).cuda(), sigma)
    return plan, Ws, X, infos, t, ss.cpu().numpy(), kpm.cpu().numpy(), rk.cpu().numpy()


def test_batched_fp64_matches_oracle_per_matrix(S):
    csrs = _graphs()
    n_v, M, sigma, n_tp = 8, 40, 0.05, 24
    plan, Ws, X, infos, t, ss, kpm, rk = _run(S, csrs, n_v, M, sigma, n_tp, "fp64")
    assert X.shape == (len(csrs), M + 1, n_v, n_v)
    for b, c in enumerate(csrs):
        A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
        tb = t[b * n_tp:(b + 1) * n_tp]
        r = O.ress_dgc(A, Ws[b], n_v, tb, M, sigma, interval=(infos[b]["a"], infos[b]["b"]), flag_eps=1e-8)
        assert np.max(np.abs(X[b] - r["X"])) <= 1e-11 * np.max(np.abs(r["X"]))
        assert O.relative_l1_error(kpm[b * n_tp:(b + 1) * n_tp], r["dos_kpm"]) <= 1e-10
        r2 = O.ress_dgc(A, Ws[b], n_v, tb, M, sigma, interval=(infos[b]["a"], infos[b]["b"]), flag_eps=1e-8,
                        moments="doubling")
        ok = ~r["flagged"] & ~r2["flagged"]
        tol = max(1e-10, 10.0 * O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok]))
        if np.sum(np.abs(r["dos_ss"][ok])) > 0:
            assert O.relative_l1_error(ss[b * n_tp:(b + 1) * n_tp][ok], r["dos_ss"][ok]) <= tol
        assert np.array_equal(rk[b * n_tp:(b + 1) * n_tp, 0][ok], r["rank_s"][ok])


def test_batched_intervals_are_per_matrix(S):
    csrs = _graphs()
    plan = S.ssm_plan_create_batched(csrs, n_v=4, degree=10, precision="fp64")
    for b, c in enumerate(csrs):
        A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
        lo, hi = O.gershgorin(A)
        a, bb = O.spectral_interval(A)
        i = S.ssm_batch_info(plan, b)
        assert i["n"] == c.n
        assert abs(i["lo"] - lo) <= 1e-14 * max(1.0, abs(lo)) and abs(i["hi"] - hi) <= 1e-14 * max(1.0, abs(hi))
        assert abs(i["a"] - a) <= 1e-14 * max(1.0, abs(a)) and abs(i["b"] - bb) <= 1e-14 * max(1.0, abs(bb))


def test_batched_mixed_tensor_core(S):
    csrs = _graphs()
    n_v, M, sigma, n_tp = 16, 40, 0.05, 16
    plan, Ws, X, infos, t, ss, kpm, rk = _run(S, csrs, n_v, M, sigma, n_tp, "mixed")
    for b, c in enumerate(csrs):
        A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
        At = O.transform(A, infos[b]["a"], infos[b]["b"])
        Xr = O.moments_direct(At, Ws[b], M)
        assert np.max(np.abs(X[b] - Xr)) <= 2e-5 * np.max(np.abs(Xr)), b
        tb = t[b * n_tp:(b + 1) * n_tp]
        tab = O.coefficient_tables(tb, M, sigma, c.n, infos[b]["a"], infos[b]["b"])
        assert O.relative_l1_error(kpm[b * n_tp:(b + 1) * n_tp], O.kpm_dos(tab["mu_full"], Xr)) <= 1e-4


@pytest.mark.parametrize("n_v,n_tp", [(16, 16), (21, 70)])
def test_batched_mixed_ss_per_matrix_from_its_moments(S, n_v, n_tp):
    # The RESS-DGC line of a mixed batched plan, matrix by matrix, against the oracle's
    # Alg. 7 loop run on the plan's own moments (so the float32 recurrence's rounding,
    # which the SS line amplifies, is not what is compared): each matrix's interval,
    # size (g_max, the 1/N_b of g_sigma), rounding floor (the mixed plan's 2^-36 unit
    # with its own X_0) and coefficient tables must be the right ones.  The assembly
    # runs on the tensor cores as exact products of six bf16 slices (~2^-47 of the
    # largest term), all matrices in one launch: (21, 70) gives two entry tiles and two
    # point tiles a matrix, the second ragged.  1e-7 on unflagged points.
    csrs = _graphs()
    M, sigma = 40, 0.05
    plan, Ws, X, infos, t, ss, kpm, rk = _run(S, csrs, n_v, M, sigma, n_tp, "mixed")
    for b, c in enumerate(csrs):
        tb = t[b * n_tp:(b + 1) * n_tp]
        tab = O.coefficient_tables(tb, M, sigma, c.n, infos[b]["a"], infos[b]["b"])
        r = O.ress_from_moments(X[b], tab, n_v, O.g_max(sigma, c.n), flag_eps=1e-8, eps_floor=2.0 ** -36)
        ok = ~r["flagged"]
        assert ok.mean() >= 0.8, b
        got = ss[b * n_tp:(b + 1) * n_tp]
        assert np.array_equal(rk[b * n_tp:(b + 1) * n_tp][ok, 0], r["rank_s"][ok]), b
        assert O.relative_l1_error(got[ok], r["dos_ss"][ok]) <= 1e-7, b


def test_batched_autotuner_reports_its_choices(S):
    csrs = _graphs()
    plan = S.ssm_plan_create_batched(csrs, n_v=16, degree=20, precision="mixed")
    assert S.ssm_batch_tuning(plan) == {"csr_threads": 0, "gram_slabs": 0}  # before the first moments
    W = np.vstack([wl.random_block(c.n, 16, 5 + k) for k, c in enumerate(csrs)])
    S.ssm_moments(plan, W)
    tuned = S.ssm_batch_tuning(plan)
    assert tuned["csr_threads"] in (64, 128, 256, 512)
    # at least one Ge and one Go slab per matrix
    assert tuned["gram_slabs"] >= 2 * len(csrs)
    plan.close()


def test_batched_repeat_and_single(S):
    # the captured graph replays with new probe contents; B = 1 is a plain batch
    csrs = _graphs()[:1]
    plan = S.ssm_plan_create_batched(csrs, n_v=4, degree=12, precision="fp64")
    c = csrs[0]
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    i = S.ssm_batch_info(plan, 0)
    At = O.transform(A, i["a"], i["b"])
    for seed in (1, 2):
        W = wl.random_block(c.n, 4, seed)
        X = S.ssm_moments(plan, W, return_moments=True)
        Xr = O.moments_direct(At, W, 12)
        assert np.max(np.abs(X[0] - Xr)) <= 1e-11 * np.max(np.abs(Xr))
    with pytest.raises(S.SSMError, match="EINVAL"):
        S.ssm_trace_f(plan, lambda x: 1.0, 64, 0.05)
    plan2 = S.ssm_plan_create_batched(_graphs()[:2], n_v=4, degree=12, precision="fp64")
    S.ssm_moments(plan2, np.vstack([wl.random_block(c.n, 4, 3) for c in _graphs()[:2]]))
    with pytest.raises(S.SSMError, match="EINVAL"):
        S.ssm_dos(plan2, np.zeros(3), 0.1)  # 3 points do not split into B = 2 equal blocks


@pytest.mark.parametrize("damping,kind", [(None, 0), ("jackson", 1)])
def test_batched_shared_interval_coefficients_fp64(S, damping, kind):
    # Matrices with one interval (here the normalised Laplacians' [0, 2], padded by 1e-3 of its
    # width) and the same sweep points share one coefficient table scaled by each matrix's
    # norm 1/(N_b sqrt(2 pi sigma^2)) (nu: its square).  Matrix 2 gets other points, so two
    # tables are built; every matrix is checked against the oracle run on it alone.
    csrs = _graphs()
    n_v, M, sigma, n_tp = 8, 40, 0.05, 24
    lo, hi = -2e-3, 2.0 + 2e-3
    plan = S.ssm_plan_create_batched(csrs, n_v=n_v, degree=M, precision="fp64", lo=lo, hi=hi, damping=damping)
    Ws = [wl.random_block(c.n, n_v, 177 + k, "rademacher") for k, c in enumerate(csrs)]
    S.ssm_moments(plan, torch.from_numpy(np.vstack(Ws)).cuda())
    base = np.linspace(0.0, 2.0, n_tp)
    ts = [base if b != 2 else base * 0.9 + 0.05 for b in range(len(csrs))]
    ss, kpm, rk = (x.cpu().numpy() for x in S.ssm_dos(plan, torch.from_numpy(np.concatenate(ts)).cuda(), sigma))
    for b, c in enumerate(csrs):
        i = S.ssm_batch_info(plan, b)
        assert (i["a"], i["b"]) == (lo, hi)
        A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
        kw = dict(interval=(lo, hi), flag_eps=1e-8, damping=kind)
        r = O.ress_dgc(A, Ws[b], n_v, ts[b], M, sigma, **kw)
        r2 = O.ress_dgc(A, Ws[b], n_v, ts[b], M, sigma, moments="doubling", **kw)
        sl = slice(b * n_tp, (b + 1) * n_tp)
        assert O.relative_l1_error(kpm[sl], r["dos_kpm"]) <= 1e-10, b
        ok = ~r["flagged"] & ~r2["flagged"]
        assert ok.mean() >= 0.8, b
        tol = max(1e-10, 10.0 * O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok]))
        assert O.relative_l1_error(ss[sl][ok], r["dos_ss"][ok]) <= tol, b
        assert np.array_equal(rk[sl, 0][ok], r["rank_s"][ok]), b
    plan.close()
