"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks one oracle function against something the paper or the
mathematics fixes: a number the paper prints, a closed-form spectrum, an
independent quadrature, dense eigendecomposition, or an exact identity.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.sparse as sp

import workloads as wl
from oracle import ssm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_sym(n, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(lo, hi, n))
    return Q @ np.diag(lam) @ Q.T, lam, Q


# ---------------------------------------------------------------- worked example

def test_range_bound_matches_printed_worked_example():
    with open(os.path.join(GOLDEN, "worked_example_range_filter.json")) as f:
        g = json.load(f)
    gm = O.g_max(g["sigma"], g["N"])
    assert abs(gm - g["range_bound_printed"]) <= 0.5 * 10 ** (-g["printed_decimals"])
    # the printed spurious eigenvalue is outside the filter range and is dropped
    K_W = np.array([[1.0]])
    K_Z = np.array([[g["spurious_xi_printed"]]])
    xi, C, info = O.geneig(K_W, K_Z, gm)
    assert xi.size == 0 and info["rank_xi"] == 0
    K_Z = np.array([[0.5 * gm]])
    xi, C, info = O.geneig(K_W, K_Z, gm)
    assert xi.size == 1 and abs(xi[0] - 0.5 * gm) < 1e-18


# ---------------------------------------------------------------- operators

@pytest.mark.parametrize("nx,periodic", [(7, False), (8, True)])
def test_stencil_csr_matches_closed_form_laplacian_spectrum(nx, periodic):
    st = wl.Stencil(dims=(nx, nx, 1), periodic=(periodic, periodic, False),
                    diag=np.full(nx * nx, 4.0), offdiag=(-1.0, -1.0, 0.0))
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val).toarray()
    assert np.array_equal(A, A.T)
    k = np.arange(nx)
    if periodic:
        lam1 = 2.0 - 2.0 * np.cos(2.0 * math.pi * k / nx)
    else:
        lam1 = 2.0 - 2.0 * np.cos(math.pi * (k + 1) / (nx + 1))
    exact = np.sort((lam1[:, None] + lam1[None, :]).ravel())
    assert np.allclose(np.linalg.eigvalsh(A), exact, atol=1e-12)


def test_stencil_3d_periodic_closed_form():
    nx = 5
    st = wl.Stencil(dims=(nx, nx, nx), periodic=(True, True, True),
                    diag=np.full(nx ** 3, 6.0), offdiag=(-1.0, -1.0, -1.0))
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val).toarray()
    lam1 = 2.0 - 2.0 * np.cos(2.0 * math.pi * np.arange(nx) / nx)
    exact = np.sort((lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]).ravel())
    assert np.allclose(np.linalg.eigvalsh(A), exact, atol=1e-12)


def test_gershgorin_hand_example_and_containment():
    A = sp.csr_matrix(np.array([[2.0, -1.0, 0.5], [-1.0, 0.0, 0.25], [0.5, 0.25, -3.0]]))
    lo, hi = O.gershgorin(A)
    # rows: 2 +- 1.5, 0 +- 1.25, -3 +- 0.75
    assert (lo, hi) == (-3.75, 3.5)
    for name in ("lap2d_dirichlet_32",):
        st = wl.make_operator(name, nx=12)
        c = wl.stencil_to_csr(st)
        A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
        a, b = O.spectral_interval(A)
        ev = np.linalg.eigvalsh(A.toarray())
        assert a < ev[0] and ev[-1] < b
        At = O.transform(A, a, b)
        evt = np.linalg.eigvalsh(At.toarray())
        assert np.allclose(evt, (2 * ev - (a + b)) / (b - a), atol=1e-13)
        assert -1 < evt[0] and evt[-1] < 1


# ---------------------------------------------------------------- coefficients

@pytest.mark.parametrize("t,l", [(0.3, 0), (0.3, 1), (-0.7, 5), (0.05, 17)])
def test_mu_matches_independent_quadrature_of_integral_definition(t, l):
    # mu_l(t) = (2 - delta_l0)/pi int_0^pi g(t - x(cos th)) cos(l th) dth (Eq. mucoef2)
    a, b, sigma, N, M = -1.5, 2.0, 0.2, 10, 40
    mu = O.dgc_coefficients(t, M, sigma, N, a, b)

    def integrand(th):
        x = 0.5 * (a + b) + 0.5 * (b - a) * math.cos(th)
        return O.g_sigma(t - x, sigma, N) * math.cos(l * th)

    val, err = si.quad(integrand, 0.0, math.pi, limit=400, epsabs=1e-15, epsrel=1e-13)
    ref = (2.0 - (l == 0)) / math.pi * val
    assert abs(mu[l] - ref) <= 1e-12 * O.g_max(sigma, N)


def test_mu_series_reconstructs_gaussian_within_theorem2_regime():
    a, b, sigma, N, M = -1.0, 1.0, 0.1, 1, 400
    s = np.linspace(-0.999, 0.999, 301)
    for t in (-0.5, 0.0, 0.8):
        mu = O.dgc_coefficients(t, M, sigma, N, a, b)
        T = np.cos(np.outer(np.arccos(s), np.arange(M + 1)))
        approx = T @ mu
        exact = O.g_sigma(t - s, sigma, N)
        assert np.max(np.abs(approx - exact)) < 1e-12


def test_nu_is_the_square_of_the_half_degree_series():
    a, b, sigma, N, M = -2.0, 3.0, 0.15, 7, 64
    rng = np.random.default_rng(0)
    s = rng.uniform(-1, 1, 50)
    for t in (-1.0, 0.4, 2.5):
        mh = O.dgc_coefficients(t, M // 2, sigma, N, a, b, n_theta=2 * M)
        nu = O.squared_coefficients(mh, M)
        Th = np.cos(np.outer(np.arccos(s), np.arange(M // 2 + 1)))
        Tf = np.cos(np.outer(np.arccos(s), np.arange(M + 1)))
        lhs = (Th @ mh) ** 2
        rhs = Tf @ nu
        assert np.max(np.abs(lhs - rhs)) <= 1e-14 * max(1.0, np.max(np.abs(lhs)))
        # the product rule T_p T_q = (T_{p+q} + T_|p-q|)/2 gives the same nu
        nu2 = np.zeros(M + 1)
        for p in range(M // 2 + 1):
            for q in range(M // 2 + 1):
                nu2[p + q] += 0.5 * mh[p] * mh[q]
                nu2[abs(p - q)] += 0.5 * mh[p] * mh[q]
        assert np.max(np.abs(nu - nu2)) <= 1e-14 * np.max(np.abs(nu2))


# ---------------------------------------------------------------- moments

def test_moments_match_dense_eigendecomposition_and_doubling():
    A, lam, Q = _dense_sym(30, 3, -2.0, 5.0)
    A = sp.csr_matrix(A)
    a, b = -2.5, 5.5
    At = O.transform(A, a, b)
    W = wl.random_block(30, 5, 4)
    M = 24
    X = O.moments_direct(At, W, M)
    lt = (2 * lam - (a + b)) / (b - a)
    Y = Q.T @ W
    for l in (0, 1, 2, 7, 24):
        ref = Y.T @ (np.cos(l * np.arccos(lt))[:, None] * Y)
        assert np.allclose(X[l], ref, atol=1e-12 * np.abs(ref).max())
    Xd = O.moments_doubling(At, W, M)
    assert np.max(np.abs(X - Xd)) <= 1e-12 * np.max(np.abs(X))


# ---------------------------------------------------------------- KPM line

def test_kpm_with_identity_probes_is_exact_dos_when_resolved():
    # W = sqrt(N) I gives zeta_l = sum_i T_l(lambda~_i): the KPM line is the exact
    # degree-M expansion; with M sigma~ large it equals the exact phi_sigma.
    A, lam, Q = _dense_sym(40, 5, -1.0, 2.0)
    A = sp.csr_matrix(A)
    N = 40
    W = math.sqrt(N) * np.eye(N)
    t = np.linspace(-1.2, 2.2, 37)
    r = O.ress_dgc(A, W, N, t, 400, 0.15)
    ex = O.exact_dos(lam, t, 0.15)
    assert np.max(np.abs(r["dos_kpm"] - ex)) < 1e-10 * np.max(ex)


def test_kpm_integrates_to_one_for_rademacher_probes():
    st = wl.make_operator("lap2d_dirichlet_32", nx=10)
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    W = wl.random_block(c.n, 8, 9, "rademacher")
    a, b = O.spectral_interval(A)
    sigma = 0.3
    t = np.linspace(a - 12 * sigma, b + 12 * sigma, 3001)
    r = O.ress_dgc(A, W, 8, t, 60, sigma)
    integral = np.trapezoid(r["dos_kpm"], t)
    assert abs(integral - 1.0) < 1e-10


# ---------------------------------------------------------------- SS estimate

def test_ss_with_identity_probes_recovers_exact_dos():
    # W = I: K_W = P, K_Z = P^2, so Alg. 4 returns the eigenvalues of P within
    # [tau max, g_max]; with a resolved expansion this is phi_sigma(t).
    A, lam, Q = _dense_sym(36, 6, -1.0, 1.0)
    A = sp.csr_matrix(A)
    N = 36
    t = np.linspace(-0.9, 0.9, 19)
    sigma = 0.12
    r = O.ress_dgc(A, np.eye(N), N, t, 800, sigma, interval=(-1.05, 1.05))
    ex = O.exact_dos(lam, t, sigma)
    assert np.max(np.abs(r["dos_ss"] - ex)) < 1e-6 * np.max(ex)


def test_ss_recovers_low_rank_trace_theorem3_regime():
    # r eigenvalues within a few sigma of t, the rest far away: with
    # N_v = r + 10 Gaussian probes the estimate matches the exact trace.
    rng = np.random.default_rng(11)
    N, r, sigma = 120, 6, 0.05
    lam = np.concatenate([rng.uniform(-0.1, 0.1, r), rng.uniform(0.7, 0.95, N - r)])
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    A = sp.csr_matrix(Q @ np.diag(lam) @ Q.T)
    W = wl.random_block(N, r + 10, 12)
    t = np.array([-0.05, 0.0, 0.04])
    res = O.ress_dgc(A, W, r + 10, t, 1200, sigma, interval=(-1.0, 1.0))
    ex = O.exact_dos(lam, t, sigma)
    assert np.max(np.abs(res["dos_ss"] - ex)) < 1e-8 * np.max(ex)
    # the same probes through the KPM line carry O(1/sqrt(N_v)) noise
    assert np.max(np.abs(res["dos_kpm"] - ex)) > 1e-4 * np.max(ex)


def test_hybrid_correction_is_unbiased_over_second_block():
    # For fixed W, E_{W~}[phi_SS] = Tr g^{M/2}(tI - A) (Theorem 4, Eq. 4.x
    # consistency): average over many W~ and compare with the exact trace of
    # the degree-M/2 series, computed from the eigenvalues.
    N, nv, nvh, M, sigma = 24, 3, 4, 80, 0.2
    A, lam, Q = _dense_sym(N, 21, -1.0, 1.0)
    A = sp.csr_matrix(A)
    t = np.array([0.1])
    a, b = -1.1, 1.1
    W = wl.random_block(N, nv, 22)
    mh = O.dgc_coefficients(t[0], M // 2, sigma, N, a, b, n_theta=2 * M)
    lt = (2 * lam - (a + b)) / (b - a)
    exact = float(np.sum(np.cos(np.outer(np.arccos(lt), np.arange(M // 2 + 1))) @ mh))
    At = O.transform(A, a, b)
    tab = O.coefficient_tables(t, M, sigma, N, a, b)
    vals = []
    for s in range(600):
        Wt = wl.random_block(N, nvh, 10_000 + s)
        Wall = np.hstack([W, Wt])
        X = O.moments_direct(At, Wall, M)
        K = O.assemble(tab["mu_half"][0], tab["nu"][0], X, nv)
        phi, _ = O.ress_dos_point(*K, O.g_max(sigma, N))
        vals.append(phi)
    vals = np.array(vals)
    se = vals.std(ddof=1) / math.sqrt(vals.size)
    assert abs(vals.mean() - exact) < 4.0 * se + 1e-12
    # without the correction the low-rank part alone is biased low here
    X = O.moments_direct(At, W, M)
    K = O.assemble(tab["mu_half"][0], tab["nu"][0], X, nv)
    phi0, _ = O.ress_dos_point(*K, O.g_max(sigma, N))
    assert exact - phi0 > 10.0 * se


# ---------------------------------------------------------------- trace of f(A)

@pytest.mark.parametrize("kind", ["one", "x", "x2", "exp"])
def test_trace_from_exact_dos_matches_closed_forms(kind):
    A, lam, Q = _dense_sym(50, 31, -3.0, 4.0)
    N = 50
    f = {"one": lambda x: np.ones_like(x), "x": lambda x: x, "x2": lambda x: x * x,
         "exp": lambda x: np.exp(-0.3 * x)}[kind]
    exact = {"one": N, "x": np.trace(A), "x2": np.sum(A * A),
             "exp": np.sum(np.exp(-0.3 * lam))}[kind]
    lo, hi = lam[0], lam[-1]
    # sigma small enough that h's spectrum decays faster than the Gaussian's
    # (the condition of Section 5) and that the smeared DOS stays inside the
    # periodic cell; sigma~ = 0.016 as in the paper's trace experiment.
    sigma = 0.02
    tr = O.trace_f(f, N, lambda x: O.exact_dos(lam, x, sigma), 1024, lo, hi, sigma,
                   sigma_tilde=0.016)
    assert abs(tr - exact) < 1e-9 * max(1.0, abs(exact))


def test_relative_l1_error_definition():
    assert O.relative_l1_error(np.array([1.0, 2.0, 3.5]), np.array([1.0, 2.0, 3.0])) == 0.5 / 6.0


def test_ss_identity_probes_underresolved_selects_filtered_eigenvalues():
    # Under-resolved expansion (M/2 sigma~ ~ 1): P = g^{M/2}(tI - A) has
    # negative and tiny eigenvalues.  With W = I, K_W = P and K_Z = P^2, so
    # Alg. 4 must return exactly the eigenvalues p(lambda_i) of P that pass the
    # truncation (p >= tau max p) and the range filter (p <= g_max).
    A, lam, Q = _dense_sym(30, 41, -1.0, 1.0)
    A = sp.csr_matrix(A)
    N, M, sigma = 30, 16, 0.08
    a, b = -1.05, 1.05
    t = np.linspace(-0.8, 0.8, 9)
    r = O.ress_dgc(A, np.eye(N), N, t, M, sigma, interval=(a, b))
    lt = (2 * lam - (a + b)) / (b - a)
    T = np.cos(np.outer(np.arccos(lt), np.arange(M // 2 + 1)))
    gm = O.g_max(sigma, N)
    for i, ti in enumerate(t):
        mh = O.dgc_coefficients(ti, M // 2, sigma, N, a, b, n_theta=2 * M)
        p = T @ mh
        assert np.any(p < 0)  # the truncated series does oscillate below zero
        keep = (p >= 1e-7 * p.max()) & (p <= (1 + 1e-6) * gm) & (p >= -1e-6 * gm)
        assert abs(r["dos_ss"][i] - p[keep].sum()) < 1e-12 * gm
        # the KPM line with W = I is the trace of the degree-M series
        Tf = np.cos(np.outer(np.arccos(lt), np.arange(M + 1)))
        mf = O.dgc_coefficients(ti, M, sigma, N, a, b, n_theta=2 * M)
        assert abs(r["dos_kpm"][i] - (Tf @ mf).sum() / N) < 1e-12 * gm


def test_rounding_floor_drops_noise_only():
    # A spectral gap: at sweep points more than 12 sigma from every eigenvalue
    # g_sigma(tI - A) is below 1e-31 of its peak, so K_W(t) is rounding noise;
    # the floor must keep nothing there (phi = 0), while inside the spectrum
    # it must not change the estimate.
    rng = np.random.default_rng(7)
    N, sigma, M = 60, 0.03, 600
    lam = np.concatenate([rng.uniform(-0.9, -0.4, N // 2), rng.uniform(0.4, 0.9, N // 2)])
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    A = sp.csr_matrix(Q @ np.diag(lam) @ Q.T)
    W = wl.random_block(N, 12, 8)
    gap = np.linspace(-0.02, 0.02, 5)
    r = O.ress_dgc(A, W, 12, gap, M, sigma, interval=(-1.0, 1.0))
    assert np.all(r["dos_ss"] == 0.0) and np.all(r["rank_s"] == 0)
    inside = np.linspace(-0.85, -0.45, 7)
    r1 = O.ress_dgc(A, W, 12, inside, M, sigma, interval=(-1.0, 1.0))
    r0 = O.ress_dgc(A, W, 12, inside, M, sigma, interval=(-1.0, 1.0), eps_floor=0.0)
    assert np.array_equal(r1["dos_ss"], r0["dos_ss"])
    # the floor is far below tau * max s inside the spectrum
    tab = O.coefficient_tables(inside, M, sigma, N, -1.0, 1.0)
    for i in range(inside.size):
        K = O.assemble(tab["mu_half"][i], tab["nu"][i], r1["X"], 12)
        s = np.linalg.eigvalsh(K[0])
        assert O.rounding_floor(tab["mu_half"][i], r1["X"], 12, O.EPS_FP64) < 1e-3 * 1e-7 * s.max()


# ---------------------------------------------------------------- damping (KPM literature)

@pytest.mark.parametrize("L", [1, 2, 7, 64, 501])
def test_jackson_closed_form_is_autocorrelation_of_sine_sequence(L):
    # The Jackson kernel is |sum_nu a_nu e^{i nu phi}|^2 / sum a_nu^2 with
    # a_nu = sin(pi (nu + 1) / (L + 1)); its Fourier coefficients are the
    # normalised autocorrelations of a, an independent route to the factors.
    a = np.sin(math.pi * (np.arange(L) + 1) / (L + 1))
    ac = np.array([np.dot(a[: L - k], a[k:]) for k in range(L)]) / np.dot(a, a)
    g = O.jackson_factors(L)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert np.max(np.abs(g - ac)) < 1e-13


@pytest.mark.parametrize("kind", [1, 2])
def test_damping_kernels_are_nonnegative(kind):
    # Both kernels K(phi) = g_0 + 2 sum_n g_n cos(n phi) are nonnegative (the
    # Jackson one touches zero), which is what makes damped expansions of
    # nonnegative functions nonnegative.
    L = 50
    g = O.damping_factors(kind, L, 4.0)
    phi = np.linspace(0.0, math.pi, 4001)
    K = g[0] + 2.0 * np.cos(np.outer(phi, np.arange(1, L))) @ g[1:]
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert np.min(K) > -1e-12 * np.max(K)
    if kind == 2:
        lam = 4.0
        assert g[10] == pytest.approx(math.sinh(lam * (1 - 10 / L)) / math.sinh(lam), rel=1e-14)


def test_jackson_damped_gaussian_expansion_is_nonnegative():
    # An under-resolved truncated series of g_sigma(t - x) has negative Gibbs
    # lobes; the Jackson-damped one is a convolution of g_sigma with a
    # nonnegative kernel and stays nonnegative on the whole interval.
    M, sigma, a, b, N = 40, 0.02, -1.0, 1.0, 100
    t = np.array([0.1])
    s = np.linspace(-1.0, 1.0, 4001)
    T = np.cos(np.outer(np.arccos(s), np.arange(M + 1)))
    plain = T @ O.coefficient_tables(t, M, sigma, N, a, b)["mu_full"][0]
    damped = T @ O.coefficient_tables(t, M, sigma, N, a, b, damping=1)["mu_full"][0]
    assert np.min(plain) < -1e-3 * np.max(plain)
    assert np.min(damped) > -1e-12 * np.max(damped)


@pytest.mark.parametrize("kind", [1, 2])
def test_damped_kpm_with_identity_probes_matches_eigenvalue_sum(kind):
    # W = sqrt(N) I: the KPM line is sum_i sum_l g_l mu_l(t) T_l(lambda~_i) with the
    # factors of M+1 terms, evaluated here from the eigenvalues; the SS line's
    # nu is the square of the half-degree series damped with M/2+1 factors.
    A, lam, Q = _dense_sym(30, 11, -1.0, 2.0)
    A = sp.csr_matrix(A)
    N, M, sigma = 30, 60, 0.2
    a, b = O.spectral_interval(A)
    t = np.linspace(-1.0, 2.0, 13)
    r = O.ress_dgc(A, math.sqrt(N) * np.eye(N), N, t, M, sigma, damping=kind)
    lt = (2 * lam - (a + b)) / (b - a)
    T = np.cos(np.outer(np.arange(M + 1), np.arccos(lt)))   # (M+1) x N
    g = O.damping_factors(kind, M + 1)
    ref = np.array([np.sum((g * O.dgc_coefficients(ti, M, sigma, N, a, b)) @ T) for ti in t])
    assert np.max(np.abs(r["dos_kpm"] - ref)) < 1e-11 * np.max(np.abs(ref))
    gh = O.damping_factors(kind, M // 2 + 1)
    tab = O.coefficient_tables(t, M, sigma, N, a, b, damping=kind)
    s = np.linspace(-1.0, 1.0, 257)
    Th = np.cos(np.outer(np.arccos(s), np.arange(M // 2 + 1)))
    Tf = np.cos(np.outer(np.arccos(s), np.arange(M + 1)))
    for i in (0, 6, 12):
        ph = Th @ (gh * O.dgc_coefficients(t[i], M // 2, sigma, N, a, b, 2 * M))
        assert np.max(np.abs(Tf @ tab["nu"][i] - ph * ph)) < 1e-12 * np.max(ph * ph)


def test_damped_kpm_integrates_to_one():
    st = wl.make_operator("lap2d_dirichlet_32", nx=10)
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    W = wl.random_block(c.n, 8, 9, "rademacher")
    a, b = O.spectral_interval(A)
    sigma = 0.3
    t = np.linspace(a - 12 * sigma, b + 12 * sigma, 3001)
    r = O.ress_dgc(A, W, 8, t, 60, sigma, damping=1)
    assert abs(np.trapezoid(r["dos_kpm"], t) - 1.0) < 1e-10


# ---------------------------------------------------------------- log-determinant reference

def test_logdet_shifted_matches_dense_eigenvalues():
    # the sparse-LU log det used as the exact Tr log(A + I) of the 3D log-normal workload
    st = wl.make_operator("lap3d_lognormal_64", nx=7)
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    ev = np.linalg.eigvalsh(A.toarray())
    assert np.min(ev) > -1.0
    assert abs(O.logdet_shifted(A, 1.0) - np.sum(np.log(ev + 1.0))) <= 1e-11 * abs(np.sum(np.log(ev + 1.0)))


def test_trace_of_log_from_exact_dos_matches_logdet():
    # Alg. 8 on the exact regularised DOS of a 3D log-normal operator (f(t) = log(t + 1),
    # sigma = 0.06 as in the 64^3 workload) against the sparse-LU log det
    st = wl.make_operator("lap3d_lognormal_64", nx=10)
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    ev = np.linalg.eigvalsh(A.toarray())
    lo, hi = O.gershgorin(A)
    n_t = 2048
    x, dx, ft, _ = O.deconvolve_h(lambda v: np.log(v + 1.0), n_t, lo, hi, 0.06, 0.016, 0.93)
    tr = c.n * dx * np.sum(ft * O.exact_dos(ev, x, 0.06))
    ld = O.logdet_shifted(A, 1.0)
    assert abs(tr - ld) <= 1e-6 * abs(ld), (tr, ld)


# ---------------------------------------------------------------- pseudo-inverse form (Section 3.2)

def test_pinv_trace_hand_example_and_printed_spurious_value():
    # K_W = diag(1, 1e-6), K_Z = diag(0.5, 1e-3): both directions clear tau = 1e-7 and
    # Tr[K_W^+ K_Z] = 0.5 + 1e-3 / 1e-6; tau = 1e-5 drops the second; Alg. 4 with the
    # range [0, 1] keeps only xi = 0.5.  Rotated, the values are the same.
    KW, KZ = np.diag([1.0, 1e-6]), np.diag([0.5, 1e-3])
    v, info = O.pinv_trace(KW, KZ)
    assert v == pytest.approx(1000.5, rel=1e-12) and info["rank_s"] == 2
    assert O.pinv_trace(KW, KZ, tau=1e-5)[0] == pytest.approx(0.5, rel=1e-15)
    assert np.sum(O.geneig(KW, KZ, 1.0)[0]) == pytest.approx(0.5, rel=1e-12)
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((2, 2)))
    assert O.pinv_trace(Q @ KW @ Q.T, Q @ KZ @ Q.T)[0] == pytest.approx(1000.5, rel=1e-9)
    # the paper's printed spurious eigenvalue (Section 3.2): the pseudo-inverse form keeps
    # it, Alg. 4's range filter drops it
    with open(os.path.join(GOLDEN, "worked_example_range_filter.json")) as f:
        g = json.load(f)
    gm = O.g_max(g["sigma"], g["N"])
    xi = g["spurious_xi_printed"]
    assert O.pinv_trace(np.array([[1.0]]), np.array([[xi]]))[0] == pytest.approx(xi, rel=1e-15)
    assert O.geneig(np.array([[1.0]]), np.array([[xi]]), gm)[0].size == 0


def test_pinv_equals_alg4_when_every_xi_is_in_range():
    # identity probes with a resolved expansion: every generalised eigenvalue is a value
    # of the polynomial in [0, g_max], so the filter removes nothing and both forms agree
    A, lam, Q = _dense_sym(36, 6, -1.0, 1.0)
    A = sp.csr_matrix(A)
    t = np.linspace(-0.9, 0.9, 7)
    kw = dict(interval=(-1.05, 1.05))
    r4 = O.ress_dgc(A, np.eye(36), 36, t, 800, 0.12, **kw)
    rp = O.ress_dgc(A, np.eye(36), 36, t, 800, 0.12, estimator="pinv", **kw)
    assert np.all(r4["rank_xi"] == r4["rank_s"])
    assert np.max(np.abs(rp["dos_ss"] - r4["dos_ss"])) <= 1e-9 * np.max(np.abs(r4["dos_ss"]))


# ---------------------------------------------------------------- SS-DGC (Alg. 5)

def test_ss_dgc_identity_probes_select_filtered_eigenvalues_of_degree_M_series():
    # W = I: Z(t) = p_M(A~) with p_M the degree-M series of g_sigma(t - .), so
    # K_W = p_M, K_Z = p_M^2 and Alg. 4 returns the eigenvalues p_M(lambda_i) that
    # pass the truncation and the range filter.  RESS-DGC at the same M uses the
    # degree-M/2 series instead; both are checked against dense eigenvalues.
    A, lam, Q = _dense_sym(30, 43, -1.0, 1.0)
    A = sp.csr_matrix(A)
    N, M, sigma = 30, 16, 0.08
    a, b = -1.05, 1.05
    t = np.linspace(-0.8, 0.8, 9)
    r = O.ss_dgc(A, np.eye(N), t, M, sigma, interval=(a, b))
    lt = (2 * lam - (a + b)) / (b - a)
    T = np.cos(np.outer(np.arccos(lt), np.arange(M + 1)))
    gm = O.g_max(sigma, N)
    for i, ti in enumerate(t):
        mf = O.dgc_coefficients(ti, M, sigma, N, a, b, n_theta=2 * M)
        p = T @ mf
        keep = (p >= 1e-7 * p.max()) & (p <= (1 + 1e-6) * gm) & (p >= -1e-6 * gm)
        assert abs(r["dos_ss"][i] - p[keep].sum()) < 1e-12 * gm
        assert r["rank_xi"][i] == keep.sum()


def test_ss_dgc_single_probe_is_a_rayleigh_quotient():
    # N_v = 1: K_W = w^T p(A) w and K_Z = w^T p(A)^2 w are scalars, so the
    # estimate is their ratio when it lies in [0, g_max] (and K_W is kept).
    A, lam, Q = _dense_sym(25, 44, -1.0, 1.0)
    N, M, sigma = 25, 40, 0.1
    a, b = -1.02, 1.02
    w = wl.random_block(N, 1, 45)
    t = np.linspace(-0.9, 0.9, 13)
    r = O.ss_dgc(sp.csr_matrix(A), w, t, M, sigma, interval=(a, b))
    c2 = (Q.T @ w[:, 0]) ** 2
    lt = (2 * lam - (a + b)) / (b - a)
    T = np.cos(np.outer(np.arccos(lt), np.arange(M + 1)))
    gm = O.g_max(sigma, N)
    for i, ti in enumerate(t):
        p = T @ O.dgc_coefficients(ti, M, sigma, N, a, b, n_theta=2 * M)
        kw, kz = float(c2 @ p), float(c2 @ p ** 2)
        want = kz / kw if kw > 0 and -1e-6 * gm <= kz / kw <= (1 + 1e-6) * gm else 0.0
        assert abs(r["dos_ss"][i] - want) <= 1e-12 * gm


def test_ss_dgc_recovers_low_rank_trace_and_equals_ress_at_twice_the_degree():
    # Theorem 3 regime (r eigenvalues near t, N_v = r + 10): the estimate is the
    # exact trace; and since Z^T Z and W^T Z are the degree-2M and degree-M
    # series of the same moments, SS-DGC at degree M is RESS-DGC at degree 2M.
    rng = np.random.default_rng(13)
    N, r, sigma = 120, 6, 0.05
    lam = np.concatenate([rng.uniform(-0.1, 0.1, r), rng.uniform(0.7, 0.95, N - r)])
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    A = sp.csr_matrix(Q @ np.diag(lam) @ Q.T)
    W = wl.random_block(N, r + 10, 14)
    t = np.array([-0.05, 0.0, 0.04])
    ss = O.ss_dgc(A, W, t, 600, sigma, interval=(-1.0, 1.0))
    ex = O.exact_dos(lam, t, sigma)
    assert np.max(np.abs(ss["dos_ss"] - ex)) < 1e-8 * np.max(ex)
    ress = O.ress_dgc(A, W, r + 10, t, 1200, sigma, interval=(-1.0, 1.0))
    assert np.max(np.abs(ss["dos_ss"] - ress["dos_ss"])) < 1e-9 * np.max(ex)
    assert np.array_equal(ss["rank_s"], ress["rank_s"])
