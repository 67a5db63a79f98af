"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances:
* float64 path: moments to 1e-11 of max|X| (doubling vs the paper's M-step
  loop differ only by rounding), coefficient tables to 1e-12 of their max,
  KPM DOS to 1e-10 relative L1 (Eq. error).
* RESS-DGC DOS (float64): Alg. 4 divides by eigenvalues of K_W(t) down to
  tau = 1e-7 of the largest, so rounding-level differences in the moments
  are amplified by up to ~1/tau.  The tolerance is therefore
  max(1e-10, 10 x spread), spread = the relative L1 difference between the
  oracle's own two float64 evaluations (the paper's M-step loop and the
  doubling products), measured on the sweep points the oracle does not flag
  as within 1e-8 of an Alg. 4 threshold.
* mixed path (float32 recurrence, float32-accumulated Gram): KPM DOS within
  1e-4 relative L1 of the float64 oracle.  Its RESS-DGC DOS misses that
  target (an expected failure, kept as an assertion): K_W(t) is a sum of
  moments with coefficients that cancel by orders of magnitude, which
  float32 moments cannot resolve.
"""
import math

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


def _csr_A(st_or_csr):
    c = wl.stencil_to_csr(st_or_csr) if isinstance(st_or_csr, wl.Stencil) else st_or_csr
    return O.csr_matrix(c.n, c.rowptr, c.colind, c.val)


def _run(S, op, W, n_v, n_vh, M, sigma, t=None, precision="fp64", n_t=101, kind="stencil",
         moments=True, **kw):
    if kind == "stencil":
        plan = S.ssm_plan_create(stencil=op, n_v=n_v, n_vh=n_vh, degree=M, precision=precision, **kw)
    else:
        plan = S.ssm_plan_create(csr=op, n_v=n_v, n_vh=n_vh, degree=M, precision=precision, **kw)
    info = S.ssm_plan_info(plan)
    if t is None:
        t = np.linspace(info["lo"], info["hi"], n_t)
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=moments)
    ss, kpm, rank = S.ssm_dos(plan, torch.from_numpy(t).cuda(), sigma)
    out = dict(plan=plan, info=info, t=t, X=None if X is None else X.cpu().numpy(), ss=ss.cpu().numpy(),
               kpm=kpm.cpu().numpy(), rank=rank.cpu().numpy())
    return out


def _oracle(op, W, n_v, t, M, sigma, info, flag_eps=1e-8, **kw):
    A = _csr_A(op)
    return O.ress_dgc(A, W, n_v, t, M, sigma, interval=(info["a"], info["b"]), flag_eps=flag_eps, **kw)


def _ss_tolerance(op, W, n_v, t, M, sigma, info, r, ok):
    """max(1e-10, 10 x the oracle's own direct-vs-doubling spread) on the points `ok`."""
    r2 = _oracle(op, W, n_v, t, M, sigma, info, moments="doubling")
    ok = ok & ~r2["flagged"]
    spread = O.relative_l1_error(r2["dos_ss"][ok], r["dos_ss"][ok])
    return max(1e-10, 10.0 * spread), ok


# ------------------------------------------------------------------ config 1

@pytest.fixture(scope="module")
def cfg1(S):
    st = wl.make_operator("lap2d_dirichlet_32")
    c = wl.CONFIGS["lap2d_dirichlet_32"]
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    g = _run(S, st, W, c["n_v"], 0, c["M"], c["sigma"], n_t=c["n_t"])
    r = _oracle(st, W, c["n_v"], g["t"], c["M"], c["sigma"], g["info"])
    return st, W, c, g, r


def test_interval_matches_oracle_gershgorin(cfg1):
    st, W, c, g, r = cfg1
    a, b = O.spectral_interval(_csr_A(st))
    assert abs(g["info"]["a"] - a) <= 1e-12 * (b - a)
    assert abs(g["info"]["b"] - b) <= 1e-12 * (b - a)


def test_coefficients_fp64(S, cfg1):
    st, W, c, g, r = cfg1
    mu, nu = S.ssm_coefficients(g["plan"], g["t"], c["sigma"])
    assert np.max(np.abs(mu - r["mu_full"])) <= 1e-12 * np.max(np.abs(r["mu_full"]))
    assert np.max(np.abs(nu - r["nu"])) <= 1e-12 * np.max(np.abs(r["nu"]))


def test_moments_fp64(cfg1):
    st, W, c, g, r = cfg1
    scale = np.max(np.abs(r["X"]))
    assert np.max(np.abs(g["X"] - r["X"])) <= 1e-11 * scale


def test_kpm_dos_fp64(cfg1):
    st, W, c, g, r = cfg1
    assert O.relative_l1_error(g["kpm"], r["dos_kpm"]) <= 1e-10


def test_ress_dos_fp64(cfg1):
    st, W, c, g, r = cfg1
    ok = ~r["flagged"]
    assert ok.sum() >= 0.9 * ok.size
    tol, ok = _ss_tolerance(st, W, c["n_v"], g["t"], c["M"], c["sigma"], g["info"], r, ok)
    assert tol <= 1e-8
    assert O.relative_l1_error(g["ss"][ok], r["dos_ss"][ok]) <= tol
    assert np.array_equal(g["rank"][ok, 0], r["rank_s"][ok])
    assert np.array_equal(g["rank"][ok, 1], r["rank_xi"][ok])


def test_duplicated_probe_columns_few_dropped_directions(S):
    # Two pairs of equal probe columns: K_W(t) has two exactly null directions at every
    # sweep point, so inside the spectrum all but two directions are kept and the solver
    # works in the complement of the two dropped eigenvectors (Householder reflections of
    # K_W and K_Z) instead of a basis of the 38 kept ones.
    st = wl.make_operator("lap2d_dirichlet_32")
    c = wl.CONFIGS["lap2d_dirichlet_32"]
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    W[:, 1] = W[:, 0]
    W[:, 3] = W[:, 2]
    sigma = 0.3  # ~200 eigenvalues under the Gaussian: K_W(t) has full rank but for the pairs
    g = _run(S, st, W, c["n_v"], 0, c["M"], sigma, n_t=61)
    r = _oracle(st, W, c["n_v"], g["t"], c["M"], sigma, g["info"])
    ok = ~r["flagged"]
    assert np.sum(ok & (r["rank_s"] == c["n_v"] - 2)) >= 0.9 * ok.size  # the route is exercised
    tol, ok = _ss_tolerance(st, W, c["n_v"], g["t"], c["M"], sigma, g["info"], r, ok)
    assert O.relative_l1_error(g["ss"][ok], r["dos_ss"][ok]) <= tol
    assert np.array_equal(g["rank"][ok, 0], r["rank_s"][ok])
    assert np.array_equal(g["rank"][ok, 1], r["rank_xi"][ok])


def test_hybrid_fp64_ragged_columns(S):
    # 20 + 17 columns: n_tot not a multiple of the vector width; Alg. 6 correction on.
    st = wl.make_operator("lap2d_dirichlet_32", nx=23)
    W = wl.random_block(st.n, 37, 77)
    M, sigma = 120, 0.08
    g = _run(S, st, W, 20, 17, M, sigma, n_t=53)
    r = _oracle(st, W, 20, g["t"], M, sigma, g["info"])
    assert np.max(np.abs(g["X"] - r["X"])) <= 1e-11 * np.max(np.abs(r["X"]))
    assert O.relative_l1_error(g["kpm"], r["dos_kpm"]) <= 1e-10
    tol, ok = _ss_tolerance(st, W, 20, g["t"], M, sigma, g["info"], r, ~r["flagged"])
    assert O.relative_l1_error(g["ss"][ok], r["dos_ss"][ok]) <= tol


def test_csr_operator_fp64(S):
    csr = wl.er_normalized_laplacian(1500, 8.0, 1004)
    W = wl.random_block(csr.n, 24, 2004)
    M, sigma = 80, 0.05
    g = _run(S, csr, W, 16, 8, M, sigma, n_t=41, kind="csr")
    r = _oracle(csr, W, 16, g["t"], M, sigma, g["info"])
    assert np.max(np.abs(g["X"] - r["X"])) <= 1e-11 * np.max(np.abs(r["X"]))
    assert O.relative_l1_error(g["kpm"], r["dos_kpm"]) <= 1e-10
    tol, ok = _ss_tolerance(csr, W, 16, g["t"], M, sigma, g["info"], r, ~r["flagged"])
    assert O.relative_l1_error(g["ss"][ok], r["dos_ss"][ok]) <= tol


def test_3d_periodic_prime_and_self_loop_axes(S):
    # 3D periodic 7x5x3 (odd extents), then a 1-D prime-length chain whose
    # periodic unit axes fold into the diagonal.
    rng = np.random.default_rng(5)
    st = wl.Stencil(dims=(7, 5, 3), periodic=(True, True, True), diag=6 + rng.normal(0, .3, 105),
                    offdiag=(-1.0, -0.7, -1.3))
    W = wl.random_block(105, 9, 6)
    g = _run(S, st, W, 9, 0, 40, 0.2, n_t=21)
    r = _oracle(st, W, 9, g["t"], 40, 0.2, g["info"])
    assert np.max(np.abs(g["X"] - r["X"])) <= 1e-11 * np.max(np.abs(r["X"]))
    st2 = wl.Stencil(dims=(1009, 1, 1), periodic=(False, True, True), diag=rng.uniform(-1, 1, 1009),
                     offdiag=(-1.0, 0.25, 0.5))
    W2 = wl.random_block(1009, 5, 7)
    g2 = _run(S, st2, W2, 5, 0, 30, 0.1, n_t=11)
    r2 = _oracle(st2, W2, 5, g2["t"], 30, 0.1, g2["info"])
    assert np.max(np.abs(g2["X"] - r2["X"])) <= 1e-11 * np.max(np.abs(r2["X"]))
    assert O.relative_l1_error(g2["kpm"], r2["dos_kpm"]) <= 1e-10


def test_minimal_degree_and_host_buffers(S):
    st = wl.make_operator("lap2d_dirichlet_32", nx=6)
    W = wl.random_block(36, 3, 8)
    plan = S.ssm_plan_create(stencil=st, n_v=3, degree=2)
    info = S.ssm_plan_info(plan)
    X = S.ssm_moments(plan, W, return_moments=True)  # host W, host output
    t = np.linspace(info["lo"], info["hi"], 5)
    ss, kpm, rank = S.ssm_dos(plan, t, 0.5)
    r = _oracle(st, W, 3, t, 2, 0.5, info)
    assert isinstance(X, np.ndarray) and X.shape == (3, 3, 3)
    assert np.max(np.abs(X - r["X"])) <= 1e-12 * np.max(np.abs(r["X"]))
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= 1e-12


# ------------------------------------------------------------------ mixed path

@pytest.fixture(scope="module")
def mixed1(S, cfg1):
    st, W, c, g64, r = cfg1
    return _run(S, st, W, c["n_v"], 0, c["M"], c["sigma"], t=g64["t"], precision="mixed")


def test_mixed_precision_config1_kpm(cfg1, mixed1):
    # against the plain float64 oracle
    r = cfg1[4]
    assert O.relative_l1_error(mixed1["kpm"], r["dos_kpm"]) <= 1e-4


@pytest.mark.xfail(strict=True, reason="K_W(t) = sum_l mu_l X_l cancels by orders of magnitude; float32 "
                                       "moments do not resolve it (measured 1.6e-2); the float64 plans do")
def test_mixed_precision_config1_ss_meets_1e4(cfg1, mixed1):
    # against the plain float64 oracle (its own rounding floor, flag_eps 1e-8)
    r = cfg1[4]
    ok = ~r["flagged"]
    assert ok.sum() >= 0.9 * ok.size
    assert O.relative_l1_error(mixed1["ss"][ok], r["dos_ss"][ok]) <= 1e-4


# ------------------------------------------------------------------ errors

def test_error_paths(S):
    st = wl.make_operator("lap2d_dirichlet_32", nx=8)
    plan = S.ssm_plan_create(stencil=st, n_v=4, degree=10)
    with pytest.raises(S.SSMError) as e:
        S.ssm_dos(plan, np.zeros(3), 0.1)
    assert e.value.name == "SSM_ESTATE"
    W = wl.random_block(64, 4, 1)
    W[3, 2] = np.nan
    with pytest.raises(S.SSMError) as e:
        S.ssm_moments(plan, W)
    assert e.value.name == "SSM_ENONFINITE"
    W[3, 2] = 0.0
    S.ssm_moments(plan, W)
    ss, kpm, rk = S.ssm_dos(plan, np.zeros(0), 0.1)
    assert ss.shape == (0,)
    with pytest.raises(S.SSMError) as e:
        S.ssm_dos(plan, np.zeros(3), -1.0)
    assert e.value.name == "SSM_EINVAL"
    bad = wl.er_normalized_laplacian(200, 5.0, 3)
    bad.val = bad.val.copy()
    rows = np.repeat(np.arange(bad.n), np.diff(bad.rowptr))
    e = int(np.nonzero(bad.colind != rows)[0][0])
    bad.val[e] += 1e-3  # an off-diagonal entry: breaks numerical symmetry
    with pytest.raises(S.SSMError) as e:
        S.ssm_plan_create(csr=bad, n_v=4, degree=10)
    assert e.value.name == "SSM_ENOTSYM"
    st2 = wl.make_operator("lap2d_dirichlet_32", nx=8)
    st2.diag = st2.diag.copy()
    st2.diag[5] = np.inf
    with pytest.raises(S.SSMError) as e:
        S.ssm_plan_create(stencil=st2, n_v=4, degree=10)
    assert e.value.name == "SSM_ENONFINITE"


# ------------------------------------------------------------------ trace

def test_trace_f_fp64(S):
    st = wl.make_operator("lap2d_dirichlet_32", nx=12)
    W = wl.random_block(st.n, 24, 12)
    M, sigma, n_t = 400, 0.05, 256
    plan = S.ssm_plan_create(stencil=st, n_v=16, n_vh=8, degree=M)
    info = S.ssm_plan_info(plan)
    S.ssm_moments(plan, torch.from_numpy(W).cuda())
    f = lambda x: math.exp(-0.5 * x)  # noqa: E731
    tr_ss, tr_kpm = S.ssm_trace_f(plan, f, n_t, sigma, 0.016, 0.93)
    A = _csr_A(st)
    x, dx, ft, h = O.deconvolve_h(lambda v: np.exp(-0.5 * v), n_t, info["lo"], info["hi"], sigma, 0.016, 0.93)
    r = O.ress_dgc(A, W, 16, x, M, sigma, interval=(info["a"], info["b"]), flag_eps=1e-8)
    r2 = O.ress_dgc(A, W, 16, x, M, sigma, interval=(info["a"], info["b"]), moments="doubling")
    ref_ss = st.n * dx * np.sum(ft * r["dos_ss"])
    ref_kpm = st.n * dx * np.sum(ft * r["dos_kpm"])
    spread = abs(st.n * dx * np.sum(ft * r2["dos_ss"]) - ref_ss)
    assert abs(tr_kpm - ref_kpm) <= 1e-9 * abs(ref_kpm)
    assert abs(tr_ss - ref_ss) <= max(1e-9 * abs(ref_ss), 10.0 * spread)
    # both estimates are close to the exact trace of the function
    ev = np.linalg.eigvalsh(A.toarray())
    exact = np.sum(np.exp(-0.5 * ev))
    assert abs(tr_kpm - exact) < 0.05 * exact


# ------------------------------------------------------------------ Gram pair

def test_gram_pair_fp64_matches_definition_and_repeats(S):
    rng = np.random.default_rng(17)
    A = rng.standard_normal((5003, 70))
    B = rng.standard_normal((5003, 70))
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    gaa, gab = S.ssm_gram_pair(Ad, Bd)
    ref_aa, ref_ab = A.T @ A, A.T @ B
    assert np.max(np.abs(gaa.cpu().numpy() - ref_aa)) <= 1e-13 * np.max(np.abs(ref_aa))
    assert np.max(np.abs(gab.cpu().numpy() - ref_ab)) <= 1e-13 * np.max(np.abs(ref_ab))
    assert np.array_equal(gaa.cpu().numpy(), gaa.cpu().numpy().T)
    gaa2, gab2 = S.ssm_gram_pair(Ad, Bd)
    assert torch.equal(gaa, gaa2) and torch.equal(gab, gab2)
    g1, none = S.ssm_gram_pair(Ad[:1])
    assert none is None and np.allclose(g1.cpu().numpy(), np.outer(A[0], A[0]), rtol=1e-15, atol=0)


# ------------------------------------------------------------------ tensor-core Gram (mixed path)

@pytest.mark.parametrize("nv,nvh,nx", [(150, 50, 61), (37, 0, 33), (128, 0, 40), (100, 29, 47)])
def test_mixed_tensor_core_moments(S, nv, nvh, nx):
    # n_tot = 200 (two M blocks), 37 (ragged, one block), 128 (exactly one), 129 (just over)
    st = wl.anderson2d(nx, 900 + nx)
    n_tot = nv + nvh
    W = wl.random_block(st.n, n_tot, 901 + nx, "rademacher")
    M = 60
    plan_tc = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M, precision="mixed")
    plan_cc = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M, precision="mixed", options=1)
    Wd = torch.from_numpy(W).cuda()
    Xtc = S.ssm_moments(plan_tc, Wd, return_moments=True).cpu().numpy()
    Xcc = S.ssm_moments(plan_cc, Wd, return_moments=True).cpu().numpy()
    info = S.ssm_plan_info(plan_tc)
    A = _csr_A(st)
    X64 = O.moments_direct(O.transform(A, info["a"], info["b"]), W, M)
    scale = np.max(np.abs(X64))
    # float32 recurrence: both mixed variants within 2e-5 of the float64 oracle
    assert np.max(np.abs(Xcc - X64)) <= 2e-5 * scale
    assert np.max(np.abs(Xtc - X64)) <= 2e-5 * scale
    # split-bf16 tensor products vs float32 CUDA-core products on the same blocks
    assert np.max(np.abs(Xtc - Xcc)) <= 1e-5 * scale
    assert np.array_equal(Xtc, np.transpose(Xtc, (0, 2, 1)))


# ------------------------------------------------------------------ row-group stencil step

MARCH_SHAPES = [
    # (dims, periodic, offdiag): float32 grids whose axis 0 is inactive once trailing
    # extent-1 axes are dropped run the row-group kernel.  Lines of 3 and 2 rows (a row pair
    # straddles lines, wrapped neighbours), a 1D ring, a 1D chain given as (n, 1, 1), an
    # open axis next to a periodic one, a ragged last panel
    ((5, 3, 1), (True, True, False), (-1.0, -0.7, 0.0)),
    ((1, 4, 2), (False, True, True), (0.0, -1.0, -0.5)),
    ((1, 1, 10), (False, False, True), (0.0, 0.0, -1.0)),
    ((9, 1, 1), (False, False, False), (-1.0, 0.0, 0.0)),
    ((1, 33, 7), (False, False, True), (0.0, -1.0, -1.3)),
    ((17, 6, 1), (True, False, False), (-0.9, -1.1, 0.0)),
]


@pytest.mark.parametrize("dims,per,off", MARCH_SHAPES, ids=[f"{d[0]}x{d[1]}x{d[2]}" for d, _, _ in MARCH_SHAPES])
def test_row_group_stencil_geometries(S, dims, per, off):
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(n + 5)
    st = wl.Stencil(dims=dims, periodic=per, diag=rng.uniform(-2, 2, n), offdiag=off)
    nv, M = 13, 40
    W = wl.random_block(n, nv, 31 + n, "gaussian")
    plan = S.ssm_plan_create(stencil=st, n_v=nv, degree=M, precision="mixed")
    X = S.ssm_moments(plan, torch.from_numpy(W).cuda(), return_moments=True).cpu().numpy()
    info = S.ssm_plan_info(plan)
    X64 = O.moments_direct(O.transform(_csr_A(st), info["a"], info["b"]), W, M)
    assert np.max(np.abs(X - X64)) <= 2e-5 * np.max(np.abs(X64))


# ------------------------------------------------------------------ fused recurrence + Gram step

FUSED_SHAPES = [
    # (dims, periodic, offdiag, n_v, n_vh): 2D periodic with two accumulator tiles and
    # ~10 panels per CTA (every pipeline barrier wraps), ragged N, 3D with four stride
    # blocks, a periodic extent-1 axis (self coupling), N < 16, an inactive middle axis,
    # the largest n_tot
    ((1, 128, 128), (False, True, True), (0.0, -1.0, -1.0), 150, 50),
    ((1, 47, 47), (False, True, True), (0.0, -1.0, -1.0), 200, 0),
    ((5, 6, 7), (True, False, True), (-0.8, -1.0, -1.2), 100, 36),
    ((1, 7, 8), (True, True, False), (-0.5, -1.0, -1.0), 8, 0),
    ((1, 1, 11), (False, False, True), (0.0, 0.0, -1.0), 20, 0),
    ((3, 1, 33), (True, False, False), (-1.0, 0.0, -1.0), 129, 0),
    ((1, 64, 64), (False, True, True), (0.0, -1.0, -1.0), 256, 0),
]


@pytest.mark.parametrize("dims,per,off,nv,nvh", FUSED_SHAPES,
                         ids=[f"{d[0]}x{d[1]}x{d[2]}-{n + h}" for d, _, _, n, h in FUSED_SHAPES])
def test_fused_step_matches_separate_kernels_and_oracle(S, dims, per, off, nv, nvh):
    n = dims[0] * dims[1] * dims[2]
    rng = np.random.default_rng(sum(dims) + nv)
    st = wl.Stencil(dims=dims, periodic=per, diag=rng.uniform(-2, 2, n), offdiag=off)
    n_tot = nv + nvh
    W = wl.random_block(n, n_tot, 77 + n_tot, "rademacher")
    M = 40
    fused = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M, precision="mixed", options=4)
    sep = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=M, precision="mixed")
    Wd = torch.from_numpy(W).cuda()
    Xf = S.ssm_moments(fused, Wd, return_moments=True).cpu().numpy()
    Xs = S.ssm_moments(sep, Wd, return_moments=True).cpu().numpy()
    info = S.ssm_plan_info(fused)
    X64 = O.moments_direct(O.transform(_csr_A(st), info["a"], info["b"]), W, M)
    scale = np.max(np.abs(X64))
    ef, es, efs = (np.max(np.abs(a - b)) / scale for a, b in ((Xf, X64), (Xs, X64), (Xf, Xs)))
    # identical float32 blocks; only the grouping of the float32 Gram sums differs
    assert efs <= 2e-6, (ef, es, efs)
    # split-bf16 products (~2^-17 relative per term, doubled by the doubling identities)
    # on float32 blocks: within 5e-5 of the float64 oracle, as the separate kernels are
    assert ef <= 5e-5 and es <= 5e-5, (ef, es, efs)
    assert np.array_equal(Xf, np.transpose(Xf, (0, 2, 1)))
    # a second call on the same plan repeats bit for bit
    Xf2 = S.ssm_moments(fused, Wd, return_moments=True).cpu().numpy()
    assert np.array_equal(Xf, Xf2)


def test_solver_schedule_repeats_bit_for_bit(S):
    # The second and later DOS calls over the same number of points run the points in an
    # order taken from the routes of the call before (points that keep part of the
    # directions on SMs of their own).  Each point's arithmetic does not depend on the CTA
    # that runs it: every call gives the same bits, and at least two routes occur.
    st = wl.make_operator("lap2d_dirichlet_32")
    c = wl.CONFIGS["lap2d_dirichlet_32"]
    W = wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])
    for precision in ("fp64", "mixed"):
        plan = S.ssm_plan_create(stencil=st, n_v=c["n_v"], n_vh=0, degree=c["M"], precision=precision)
        info = S.ssm_plan_info(plan)
        # sigma = 0.3: full rank inside the spectrum, part of the directions towards and
        # past its ends (checked on the oracle)
        t = torch.from_numpy(np.linspace(info["lo"] - 3.0, info["hi"] + 3.0, 157)).cuda()
        S.ssm_moments(plan, torch.from_numpy(W).cuda())
        runs = [S.ssm_dos(plan, t, 0.3) for _ in range(3)]
        r0 = runs[0][2].cpu().numpy()[:, 0]
        classes = {int(np.sum(r0 == 0) > 0), 2 * int(np.sum((r0 > 0) & (r0 < c["n_v"])) > 0),
                   4 * int(np.sum(r0 == c["n_v"]) > 0)} - {0}
        assert len(classes) >= 2, np.unique(r0)
        for ss, kp, rk in runs[1:]:
            assert torch.equal(ss, runs[0][0]) and torch.equal(rk, runs[0][2]) and torch.equal(kp, runs[0][1])
