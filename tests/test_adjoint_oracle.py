"""Pins of the adjoint oracle (oracle/adjoint_oracle.py) against what the
mathematics fixes, independent of the oracle's own reverse loop:

* complex-step derivatives of the forward moment loop (exact to rounding for
  a polynomial in A, no cancellation): every diagonal entry, stored
  off-diagonal entries, and a stencil's per-axis couplings;
* the dense-eigh closed form for W = sqrt(N) I and G_l = g_l I, where
  L = N sum_j p(lambda~_j) with p = sum_l g_l T_l and so
  dL/dA~ = N Q p'(Lambda) Q^T, p' from numpy's Chebyshev derivative;
* the KPM loss weights against a perturbation of the moments themselves.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adjoint_oracle as AO
from oracle import ssm_oracle as O
import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _small(nx=6, ny=5, seed=7):
    st = wl.Stencil(dims=(1, ny, nx), periodic=(False, False, False),
                    diag=4.0 + np.random.default_rng(seed).uniform(-1, 1, nx * ny), offdiag=(0.0, -1.0, -1.0))
    csr = wl.stencil_to_csr(st)
    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    a, b = O.spectral_interval(A)
    return st, A, a, b


def _complex_step(At, W, M, G, E, h=1e-30):
    Ac = sp.csr_matrix(At, dtype=np.complex128) + 1j * h * sp.csr_matrix(E, dtype=np.complex128)
    return float(np.imag(AO.moments_linear_loss(Ac, W.astype(np.complex128), M, G))) / h


def test_adjoint_matches_complex_step_entries():
    st, A, a, b = _small()
    At = O.transform(A, a, b)
    n = A.shape[0]
    rng = np.random.default_rng(3)
    W = rng.standard_normal((n, 4))
    M = 14
    G = rng.standard_normal((M + 1, 4, 4))  # not symmetric: only sym(G) may matter
    diag, pat = AO.moments_adjoint_direct(At, W, M, G)
    scale = np.max(np.abs(diag))
    for i in (0, 7, n - 1):
        E = sp.csr_matrix(([1.0], ([i], [i])), shape=(n, n))
        ref = _complex_step(At, W, M, G, E)
        assert abs(diag[i] - ref) <= 1e-12 * scale, (i, diag[i], ref)
        assert abs(pat[i, i] - ref) <= 1e-12 * scale
    P = sp.coo_matrix(At)
    off = [(r, c) for r, c in zip(P.row, P.col) if r != c][:6]
    for (i, j) in off:
        E = sp.csr_matrix(([1.0], ([i], [j])), shape=(n, n))
        ref = _complex_step(At, W, M, G, E)
        assert abs(pat[i, j] - ref) <= 1e-12 * scale, (i, j, pat[i, j], ref)


def test_adjoint_dense_eigh_closed_form():
    st, A, a, b = _small(5, 4, seed=11)
    At = O.transform(A, a, b)
    n = A.shape[0]
    W = np.sqrt(n) * np.eye(n)
    M = 20
    g = np.random.default_rng(5).standard_normal(M + 1)
    G = g[:, None, None] * np.eye(n)[None]
    diag, pat = AO.moments_adjoint_direct(At, W, M, G)
    lam, Q = np.linalg.eigh(At.toarray())
    dp = np.polynomial.chebyshev.chebval(lam, np.polynomial.chebyshev.chebder(g))
    ref = n * (Q * dp[None, :]) @ Q.T
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(diag - np.diag(ref))) <= 1e-11 * scale
    P = sp.coo_matrix(pat)
    assert np.max(np.abs(P.data - ref[P.row, P.col])) <= 1e-11 * scale


def test_stencil_parameter_grad_complex_step():
    st = wl.Stencil(dims=(3, 4, 5), periodic=(True, False, True),
                    diag=6.0 + np.random.default_rng(2).uniform(-1, 1, 60), offdiag=(-1.0, -0.7, -1.2))
    csr = wl.stencil_to_csr(st)
    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    a, b = O.spectral_interval(A)
    At = O.transform(A, a, b)
    n = A.shape[0]
    rng = np.random.default_rng(9)
    W = rng.standard_normal((n, 3))
    M = 10
    G = rng.standard_normal((M + 1, 3, 3))
    diag_t, pat_t = AO.moments_adjoint_direct(At, W, M, G)
    dA_diag = AO.grad_wrt_a(diag_t, a, b)
    dA_pat = AO.grad_wrt_a(pat_t, a, b)
    g_diag, g_off = AO.stencil_parameter_grad(dA_pat, dA_diag, st, wl.stencil_to_csr)
    for d in range(3):
        off = [0.0, 0.0, 0.0]
        off[d] = 1.0
        Ed = wl.stencil_to_csr(dataclasses.replace(st, diag=np.zeros(n), offdiag=tuple(off)))
        E = O.csr_matrix(n, Ed.rowptr, Ed.colind, Ed.val) * (2.0 / (b - a))
        ref = _complex_step(At, W, M, G, E)
        assert abs(g_off[d] - ref) <= 1e-11 * max(1.0, abs(ref)), (d, g_off[d], ref)
    i = 17
    E = sp.csr_matrix(([2.0 / (b - a)], ([i], [i])), shape=(n, n))
    assert abs(g_diag[i] - _complex_step(At, W, M, G, E)) <= 1e-11 * np.max(np.abs(g_diag))


def test_kpm_loss_weights_linear_in_moments():
    rng = np.random.default_rng(4)
    M, k, nt = 8, 5, 7
    X = rng.standard_normal((M + 1, k, k))
    mu = rng.standard_normal((nt, M + 1))
    w = rng.standard_normal(nt)
    g = AO.kpm_loss_weights(mu, w, k)

    def loss(Xv):
        return float(w @ O.kpm_dos(mu, Xv))

    for l in (0, 3, M):
        Xp = X.copy()
        Xp[l] += np.eye(k)
        # <g_l I, I> = k g_l; the loss is linear so the difference is exact up to rounding
        assert abs((loss(Xp) - loss(X)) - k * g[l]) <= 1e-12 * max(1.0, abs(k * g[l]))


def test_symmetric_part_matches_symmetric_perturbation():
    c = wl.er_normalized_laplacian(60, 5.0, 3)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    a, b = O.spectral_interval(A)
    At = O.transform(A, a, b)
    rng = np.random.default_rng(1)
    W = rng.standard_normal((60, 3))
    M = 9
    G = rng.standard_normal((M + 1, 3, 3))
    _, pat = AO.moments_adjoint_direct(At, W, M, G)
    Ps = AO.symmetric_part(pat)
    P = sp.coo_matrix(At)
    pairs = [(r, q) for r, q in zip(P.row, P.col) if r < q][:5]
    for (i, j) in pairs:
        E = sp.csr_matrix(([1.0, 1.0], ([i, j], [j, i])), shape=At.shape)
        ref = _complex_step(At, W, M, G, E)
        assert abs(Ps[i, j] + Ps[j, i] - ref) <= 1e-12 * max(1.0, abs(ref))
        assert abs(Ps[i, j] - Ps[j, i]) <= 1e-14 * max(1.0, abs(ref))
