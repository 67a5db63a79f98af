"""Plain FP64 CPU oracle for the spectrum sweeping DOS estimator (RESS-DGC).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
restatement of L. Lin, "Randomized estimation of spectral densities of large
matrices made accurate" (arXiv 1504.07690) that the CUDA path is checked
against.  Only the test suite, the package's smoke check and the benchmark's
CPU-baseline leg may import it; the product path never does.  It shares no
code with the CUDA library: it takes the operator and the probe block W as
plain arrays and recomputes everything from the paper's definitions, in
float64, with numpy / scipy primitives (sparse matvec, FFT, dense eigh).

Every function names the passage it follows.  Where the paper is silent or
ambiguous the reading taken is stated in the docstring:

* sigma and the sweep points t are in the original units of A (Section 3.2,
  the worked example 1/(N sqrt(2 pi sigma^2)) = 0.008 for N=1000, sigma=0.05).
* The spectral interval [a, b] is the Gershgorin interval padded by 1e-3 of
  its width on each side (Section 2 only requires the spectrum inside (a,b)).
* N_theta = 2M in Algorithm 1 (the paper asks for N_theta > M).
* nu_l (Proposition 1) is computed by Algorithm 1's quadrature applied to
  the square of the degree-M/2 series, which Theorem 4 requires.
* Moments are symmetrised, X_l <- (X_l + X_l^T)/2 (exact in exact arithmetic).
* Algorithm 4's truncation keeps s_j >= tau * max s (tau default 1e-7, the
  value the paper uses for its pseudo-inverse variant) and s_j above the
  rounding floor of K_W(t) (see rounding_floor); nothing is kept when
  max s <= 0.  The range filter keeps xi in [-kappa g_max, (1+kappa) g_max],
  a rounding slack around the paper's closed interval [0, g_max].
* Algorithm 8 uses the unit-mass Gaussian N g_sigma for the deconvolution
  (the factor N of the trace formula then matches) and a periodic grid;
  the spectral bounds are mapped onto [-a, a], a = 0.93, and frequencies at
  which the Gaussian's DFT is below 1e-14 of its peak are dropped.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, Optional, Tuple

import numpy as np
import scipy.sparse as sp
from scipy.special import erf

__all__ = [
    "csr_matrix", "gershgorin", "spectral_interval", "transform",
    "g_sigma", "g_max", "dgc_coefficients", "squared_coefficients",
    "jackson_factors", "lorentz_factors", "damping_factors", "coefficient_tables",
    "moments_direct", "moments_doubling",
    "kpm_dos", "assemble", "rounding_floor", "geneig", "ress_dos_point", "pinv_trace", "ress_dgc",
    "exact_dos", "relative_l1_error", "trace_grid", "deconvolve_h",
    "trace_f", "logdet_shifted",
]


# --------------------------------------------------------------------------
# Operator and spectral map (Section 2)
# --------------------------------------------------------------------------

def csr_matrix(n: int, rowptr, colind, val) -> sp.csr_matrix:
    """Wrap CSR arrays as a scipy matrix (float64)."""
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(colind),
                          np.asarray(rowptr)), shape=(n, n))


def gershgorin(A: sp.spmatrix) -> Tuple[float, float]:
    """Gershgorin interval [min_i(A_ii - R_i), max_i(A_ii + R_i)], R_i = sum_{j!=i}|A_ij|."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    r = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def spectral_interval(A: sp.spmatrix, pad: float = 1e-3) -> Tuple[float, float]:
    """(a, b) containing the spectrum strictly: Gershgorin padded by pad*width."""
    lo, hi = gershgorin(A)
    w = hi - lo
    if w <= 0.0:
        w = max(abs(lo), 1.0)
    return lo - pad * w, hi + pad * w


def transform(A: sp.spmatrix, a: float, b: float) -> sp.csr_matrix:
    """A~ = (2A - (a+b)I)/(b-a), spectrum of A~ inside (-1, 1) (Section 2)."""
    n = A.shape[0]
    return sp.csr_matrix((2.0 * A - (a + b) * sp.identity(n)) / (b - a))


# --------------------------------------------------------------------------
# Gaussian regularisation and Chebyshev coefficients (Eq. gaussian, Alg. 1)
# --------------------------------------------------------------------------

def g_sigma(s, sigma: float, N: int):
    """g_sigma(s) = exp(-s^2 / (2 sigma^2)) / (N sqrt(2 pi sigma^2)) (Eq. gaussian)."""
    s = np.asarray(s, dtype=np.float64)
    return np.exp(-s * s / (2.0 * sigma * sigma)) / (N * math.sqrt(2.0 * math.pi * sigma * sigma))


def g_max(sigma: float, N: int) -> float:
    """Upper end of the range filter, 1/(N sqrt(2 pi sigma^2)) (Section 3.2)."""
    return 1.0 / (N * math.sqrt(2.0 * math.pi * sigma * sigma))


def dgc_coefficients(t: float, M: int, sigma: float, N: int, a: float, b: float,
                     n_theta: Optional[int] = None) -> np.ndarray:
    """mu_l(t), l = 0..M, of g_sigma(t - x) in Chebyshev polynomials of A~ (Alg. 1).

    theta_j = j pi / N_theta (j < 2 N_theta); g_j = g_sigma(t - x(cos theta_j))
    with x(s) = (a+b)/2 + (b-a)/2 s the map back to A's units; g^ = DFT(g);
    mu_l = (2 - delta_l0) / (2 N_theta) Re g^_l.
    """
    if n_theta is None:
        n_theta = 2 * M
    if n_theta <= M:
        raise ValueError("Algorithm 1 needs N_theta > M")
    j = np.arange(2 * n_theta)
    theta = j * math.pi / n_theta
    x = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(theta)
    g = g_sigma(t - x, sigma, N)
    ghat = np.fft.fft(g)
    mu = ghat[: M + 1].real / (2.0 * n_theta)
    mu[1:] *= 2.0
    return mu


def squared_coefficients(mu_half: np.ndarray, M: int,
                         n_theta: Optional[int] = None) -> np.ndarray:
    """nu_l, l = 0..M, with (sum_{k<=M/2} mu_k T_k)^2 = sum_{l<=M} nu_l T_l (Prop. 1).

    Algorithm 1's quadrature applied to q(theta) = (sum_k mu_k cos k theta)^2,
    a trigonometric polynomial of degree <= M, which 2 N_theta > 2M points
    integrate exactly.
    """
    if n_theta is None:
        n_theta = 2 * M
    if n_theta <= M:
        raise ValueError("Proposition 1 quadrature needs N_theta > M")
    K = len(mu_half) - 1
    if 2 * K > M:
        raise ValueError("mu_half must have degree <= M/2")
    theta = np.arange(2 * n_theta) * math.pi / n_theta
    series = np.cos(np.outer(theta, np.arange(K + 1))) @ mu_half
    q = series * series
    qhat = np.fft.fft(q)
    nu = qhat[: M + 1].real / (2.0 * n_theta)
    nu[1:] *= 2.0
    return nu


# --------------------------------------------------------------------------
# Optional damping of the truncated series (the KPM literature the paper's
# KPM remark cites: Weisse, Wellein, Alvermann and Fehske, Rev. Mod. Phys. 78,
# 275 (2006), Section II.C).  The paper itself uses no damping; these factors
# multiply mu_l before anything else is formed from them.
# --------------------------------------------------------------------------

def jackson_factors(n_mom: int) -> np.ndarray:
    """Jackson factors g_n, n = 0..n_mom-1, for a series of n_mom terms.

    g_n = [(n_mom - n + 1) cos(pi n / (n_mom + 1))
           + sin(pi n / (n_mom + 1)) cot(pi / (n_mom + 1))] / (n_mom + 1),
    the closed form of the kernel that is the squared modulus of a
    sine-weighted trigonometric polynomial (so it is nonnegative and g_0 = 1).
    """
    n = np.arange(n_mom, dtype=np.float64)
    q = math.pi / (n_mom + 1)
    return ((n_mom - n + 1) * np.cos(q * n) + np.sin(q * n) / math.tan(q)) / (n_mom + 1)


def lorentz_factors(n_mom: int, lam: float = 4.0) -> np.ndarray:
    """Lorentz factors g_n = sinh(lam (1 - n / n_mom)) / sinh(lam), n < n_mom."""
    n = np.arange(n_mom, dtype=np.float64)
    return np.sinh(lam * (1.0 - n / n_mom)) / math.sinh(lam)


def damping_factors(kind: int, n_mom: int, lam: float = 4.0) -> np.ndarray:
    """0: none (the paper), 1: Jackson, 2: Lorentz with parameter lam."""
    if kind == 0:
        return np.ones(n_mom)
    if kind == 1:
        return jackson_factors(n_mom)
    if kind == 2:
        return lorentz_factors(n_mom, lam)
    raise ValueError(f"unknown damping kind {kind}")


def coefficient_tables(t: np.ndarray, M: int, sigma: float, N: int, a: float, b: float,
                       n_theta: Optional[int] = None, damping: int = 0,
                       lam: float = 4.0) -> Dict[str, np.ndarray]:
    """Per-sweep-point tables used by Algorithms 2 and 7.

    mu_full[i, l], l <= M (the DGC/KPM line, Alg. 2);
    mu_half[i, l], l <= M/2 and zero above (Alg. 7, step 1);
    nu[i, l], l <= M (Alg. 7, step 2, via Prop. 1).
    All three use the same 2 N_theta-point grid, N_theta = 2M by default.
    With damping (see damping_factors) the degree-M series is multiplied by the
    factors of M+1 terms and the degree-M/2 series by those of M/2+1 terms
    before nu is formed, so nu stays the exact square of the series K_W uses.
    """
    if M % 2:
        raise ValueError("RESS-DGC needs an even degree M")
    if n_theta is None:
        n_theta = 2 * M  # one quadrature grid for every table
    t = np.asarray(t, dtype=np.float64)
    nt = t.size
    mu_full = np.zeros((nt, M + 1))
    mu_half = np.zeros((nt, M + 1))
    nu = np.zeros((nt, M + 1))
    gf = damping_factors(damping, M + 1, lam)
    gh = damping_factors(damping, M // 2 + 1, lam)
    for i in range(nt):
        mu_full[i] = gf * dgc_coefficients(t[i], M, sigma, N, a, b, n_theta)
        mh = gh * dgc_coefficients(t[i], M // 2, sigma, N, a, b, n_theta)
        mu_half[i, : M // 2 + 1] = mh
        nu[i] = squared_coefficients(mh, M, n_theta)
    return dict(mu_full=mu_full, mu_half=mu_half, nu=nu)


# --------------------------------------------------------------------------
# Moments (Alg. 2 / Alg. 7 recurrence)
# --------------------------------------------------------------------------

def moments_direct(At: sp.spmatrix, W: np.ndarray, M: int) -> np.ndarray:
    """X_l = W^T T_l(A~) W for l = 0..M by the paper's three-term loop (Alg. 7).

    V_c <- W, V_m <- 0; for l = 0..M: X_l = W^T V_c;
    V_p <- (2 - delta_l0) A~ V_c - V_m; V_m <- V_c; V_c <- V_p.
    W holds both blocks [W, W~] side by side; the moments of every pair of
    columns come out of one loop.  X_l is symmetrised.
    """
    W = np.asarray(W, dtype=np.float64)
    n, k = W.shape
    X = np.empty((M + 1, k, k))
    Vm = np.zeros_like(W)
    Vc = W.copy()
    for l in range(M + 1):
        X[l] = W.T @ Vc
        Vp = (1.0 if l == 0 else 2.0) * (At @ Vc) - Vm
        Vm, Vc = Vc, Vp
    return 0.5 * (X + np.transpose(X, (0, 2, 1)))


def moments_doubling(At: sp.spmatrix, W: np.ndarray, M: int) -> np.ndarray:
    """Same moments from M/2 products, by T_{j+k} = 2 T_j T_k - T_{|j-k|}.

    X_{2k} = 2 V_k^T V_k - X_0 and X_{2k+1} = 2 V_{k+1}^T V_k - X_1 with
    V_k = T_k(A~) W.  Used as a self-check of moments_direct.
    """
    W = np.asarray(W, dtype=np.float64)
    n, k = W.shape
    X = np.empty((M + 1, k, k))
    Vm, Vc = W, At @ W          # V_{j-1}, V_j with j = 1; only three blocks live
    X[0] = W.T @ W
    X[1] = W.T @ Vc
    for j in range(1, M // 2 + 1):
        X[2 * j] = 2.0 * Vc.T @ Vc - X[0]
        if 2 * j + 1 <= M:
            Vn = 2.0 * (At @ Vc) - Vm
            X[2 * j + 1] = 2.0 * Vn.T @ Vc - X[1]
            Vm, Vc = Vc, Vn
    return 0.5 * (X + np.transpose(X, (0, 2, 1)))


# --------------------------------------------------------------------------
# KPM / DGC line (Alg. 2) and the RESS-DGC per-point estimate (Alg. 4, 6, 7)
# --------------------------------------------------------------------------

def kpm_dos(mu_full: np.ndarray, X: np.ndarray) -> np.ndarray:
    """phi_KPM(t_i) = sum_l mu_l(t_i) zeta_l, zeta_l = Tr[X_l] / n_cols (Alg. 2)."""
    zeta = np.trace(X, axis1=1, axis2=2) / X.shape[1]
    return mu_full @ zeta


def assemble(mu_row: np.ndarray, nu_row: np.ndarray, X: np.ndarray, n_v: int):
    """K_W, K_Z, K_C, K_W~ at one sweep point (Alg. 7, accumulation steps).

    K_W = sum_l mu_l X_l[W,W],  K_Z = sum_l nu_l X_l[W,W],
    K_C = sum_l mu_l X_l[W~,W], K_W~ = sum_l mu_l X_l[W~,W~]
    (mu is zero above M/2, so these are the degree-M/2 sums).
    """
    K = np.tensordot(mu_row, X, axes=(0, 0))
    KZ = np.tensordot(nu_row, X[:, :n_v, :n_v], axes=(0, 0))
    return K[:n_v, :n_v], KZ, K[n_v:, :n_v], K[n_v:, n_v:]


def rounding_floor(mu_half_row: np.ndarray, X: np.ndarray, n_v: int, eps: float) -> float:
    """Size below which an eigenvalue of K_W(t) is rounding noise.

    K_W(t) = sum_l mu_l X_l[W,W] with |X_l[i][j]| <= max_i X_0[i][i] (Cauchy-
    Schwarz, |T_l| <= 1); the three-term recurrence lets the rounding error
    of X_l grow at most linearly in l, so the error of K_W is of order
    eps * max_i X_0[i][i] * sum_l (l+1) |mu_l|; times n_v for the 2-norm of an
    n_v x n_v perturbation and a safety factor.
    """
    x0 = float(np.max(np.diag(X[0])[:n_v]))
    l = np.arange(mu_half_row.size)
    return FLOOR_SAFETY * n_v * eps * x0 * float(np.sum((l + 1.0) * np.abs(mu_half_row)))


FLOOR_SAFETY = 8.0
EPS_FP64 = 2.0 ** -52


def geneig(K_W: np.ndarray, K_Z: np.ndarray, gmax: float, tau: float = 1e-7,
           kappa: float = 1e-6, flag_eps: float = 0.0, floor: float = 0.0):
    """Generalised eigenproblem K_Z C = K_W C Xi restricted as in Alg. 4.

    1. K_W = U S U^T;  2. keep s_j >= max(tau max s, floor);  3. eigh of
    S~^-1/2 U~^T K_Z U~ S~^-1/2 = X Xi X^T;  4. keep xi in the range of
    g_sigma, [-kappa gmax, (1+kappa) gmax];  5. C~ = U~ S~^-1/2 X~.

    `floor` is the rounding floor of K_W (see rounding_floor): where K_W(t)
    is numerically zero (t outside the spectrum) the paper's relative rule
    alone would keep pure rounding noise, whose ratios xi land anywhere in
    the filter range.

    Returns (xi_kept, C_kept, info) where info has the kept ranks and a
    flag that is set when some s_j or xi lies within flag_eps (relative to
    max s, resp. gmax) of a threshold, i.e. where the result is
    discontinuous in its input.
    """
    s, U = np.linalg.eigh(0.5 * (K_W + K_W.T))
    smax = float(np.max(s)) if s.size else 0.0
    flagged = False
    if smax <= 0.0:
        n = K_W.shape[0]
        return np.zeros(0), np.zeros((n, 0)), dict(rank_s=0, rank_xi=0, flagged=False)
    thr = max(tau * smax, floor)
    keep = s >= thr
    if flag_eps > 0.0 and np.any(np.abs(s - thr) <= flag_eps * smax):
        flagged = True
    Ut = U[:, keep]
    isq = 1.0 / np.sqrt(s[keep])
    Bm = (Ut.T @ K_Z @ Ut) * isq[:, None] * isq[None, :]
    xi, Xv = np.linalg.eigh(0.5 * (Bm + Bm.T))
    lo, hi = -kappa * gmax, (1.0 + kappa) * gmax
    sel = (xi >= lo) & (xi <= hi)
    if flag_eps > 0.0 and (np.any(np.abs(xi - lo) <= flag_eps * gmax)
                           or np.any(np.abs(xi - hi) <= flag_eps * gmax)):
        flagged = True
    C = (Ut * isq[None, :]) @ Xv[:, sel]
    return xi[sel], C, dict(rank_s=int(keep.sum()), rank_xi=int(sel.sum()), flagged=flagged)


def ress_dos_point(K_W, K_Z, K_C, K_Wt, gmax: float, tau: float = 1e-7,
                   kappa: float = 1e-6, flag_eps: float = 0.0, floor: float = 0.0):
    """One sweep point of Alg. 7 (Alg. 6's estimate applied to g^{M/2}(tI - A)).

    phi = Tr Xi~ + (1/N~_v) (Tr K_W~ - Tr K_C C~ C~^T K_C^T); the hybrid
    correction is absent when N~_v = 0.
    """
    xi, C, info = geneig(K_W, K_Z, gmax, tau, kappa, flag_eps, floor)
    phi = float(np.sum(xi))
    nvh = K_Wt.shape[0]
    if nvh > 0:
        KC = K_C @ C
        phi += (float(np.trace(K_Wt)) - float(np.sum(KC * KC))) / nvh
    return phi, info


def pinv_trace(K_W: np.ndarray, K_Z: np.ndarray, tau: float = 1e-7, flag_eps: float = 0.0, floor: float = 0.0):
    """Tr[K_W^+ K_Z], the pseudo-inverse form of the estimate (Section 3.2).

    K_W = U S U^T; the pseudo-inverse keeps s_j >= max(tau max s, floor) (the
    paper drops negative eigenvalues and those below a 1e-7 fraction of the
    largest; the floor is Alg. 4's, see rounding_floor) and
    Tr[K_W^+ K_Z] = sum_kept (u_j^T K_Z u_j) / s_j.  Unlike Alg. 4 no range
    filter follows: every direction kept contributes.  Returns (value, info)
    with the kept rank and the threshold flag as in geneig.
    """
    s, U = np.linalg.eigh(0.5 * (K_W + K_W.T))
    smax = float(np.max(s)) if s.size else 0.0
    if smax <= 0.0:
        return 0.0, dict(rank_s=0, rank_xi=0, flagged=False)
    thr = max(tau * smax, floor)
    keep = s >= thr
    flagged = bool(flag_eps > 0.0 and np.any(np.abs(s - thr) <= flag_eps * smax))
    Ut = U[:, keep]
    val = float(np.sum(np.einsum("ij,ik,kj->j", Ut, 0.5 * (K_Z + K_Z.T), Ut) / s[keep]))
    r = int(keep.sum())
    return val, dict(rank_s=r, rank_xi=r, flagged=flagged)


def ress_dgc(A: sp.spmatrix, W_all: np.ndarray, n_v: int, t: np.ndarray, M: int,
             sigma: float, tau: float = 1e-7, kappa: float = 1e-6,
             interval: Optional[Tuple[float, float]] = None,
             n_theta: Optional[int] = None, flag_eps: float = 0.0,
             moments: str = "direct", eps_floor: float = EPS_FP64, damping: int = 0,
             lam: float = 4.0, estimator: str = "alg4") -> Dict[str, np.ndarray]:
    """RESS-DGC (Alg. 7) and the DGC/KPM line (Alg. 2) on the same probes.

    W_all = [W, W~] (N x (n_v + n_vh)).  eps_floor sets the rounding floor
    of Alg. 4's truncation (0 disables it).  damping / lam select optional
    damping factors of the series (coefficient_tables).  estimator "pinv"
    replaces Alg. 4 + Alg. 6 by Tr[K_W^+ K_Z] (pinv_trace; no hybrid block).
    Returns dos_ss, dos_kpm, the kept ranks, the flags, the interval and the
    moments.
    """
    if estimator not in ("alg4", "pinv"):
        raise ValueError(estimator)
    if estimator == "pinv" and W_all.shape[1] != n_v:
        raise ValueError("the pseudo-inverse form takes no hybrid block")
    A = sp.csr_matrix(A)
    N = A.shape[0]
    a, b = interval if interval is not None else spectral_interval(A)
    At = transform(A, a, b)
    tab = coefficient_tables(t, M, sigma, N, a, b, n_theta, damping, lam)
    X = (moments_direct if moments == "direct" else moments_doubling)(At, W_all, M)
    out = ress_from_moments(X, tab, n_v, g_max(sigma, N), tau, kappa, flag_eps, eps_floor, estimator)
    out["dos_kpm"] = kpm_dos(tab["mu_full"], X)
    return dict(out, a=a, b=b, X=X, **tab)


def ress_from_moments(X: np.ndarray, tab: Dict[str, np.ndarray], n_v: int, gm: float, tau: float = 1e-7,
                      kappa: float = 1e-6, flag_eps: float = 0.0, eps_floor: float = EPS_FP64,
                      estimator: str = "alg4") -> Dict[str, np.ndarray]:
    """Alg. 7's per-point loop on given moments: the first n_v columns of X are W, the
    rest W~ (so one set of moments serves every split N_v + N~_v of the same probes).
    tab holds the coefficient tables of coefficient_tables."""
    nt = tab["mu_half"].shape[0]
    dos_ss = np.zeros(nt)
    rank_s = np.zeros(nt, dtype=np.int64)
    rank_xi = np.zeros(nt, dtype=np.int64)
    flags = np.zeros(nt, dtype=bool)
    for i in range(nt):
        K_W, K_Z, K_C, K_Wt = assemble(tab["mu_half"][i], tab["nu"][i], X, n_v)
        fl = rounding_floor(tab["mu_half"][i], X, n_v, eps_floor) if eps_floor > 0 else 0.0
        if estimator == "pinv":
            dos_ss[i], info = pinv_trace(K_W, K_Z, tau, flag_eps, fl)
        else:
            dos_ss[i], info = ress_dos_point(K_W, K_Z, K_C, K_Wt, gm, tau, kappa, flag_eps, fl)
        rank_s[i], rank_xi[i], flags[i] = info["rank_s"], info["rank_xi"], info["flagged"]
    return dict(dos_ss=dos_ss, rank_s=rank_s, rank_xi=rank_xi, flagged=flags)


def ss_dgc(A: sp.spmatrix, W: np.ndarray, t: np.ndarray, M: int, sigma: float, tau: float = 1e-7,
           kappa: float = 1e-6, interval: Optional[Tuple[float, float]] = None,
           n_theta: Optional[int] = None, flag_eps: float = 0.0, eps_floor: float = EPS_FP64,
           damping: int = 0, lam: float = 4.0, estimator: str = "alg4") -> Dict[str, np.ndarray]:
    """SS-DGC (Alg. 5): the filtered blocks Z(t_i) are formed explicitly.

    mu_l(t_i), l <= M, by Alg. 1 (the degree-M table, with the damping factors
    of M+1 terms when damping is set); V_c <- W, V_m <- 0; for l = 0..M:
    Z(t_i) += mu_l(t_i) V_c for every point, then V_p <- (2 - delta_l0) A~ V_c - V_m.
    Per point the generalised problem Z^T Z C = W^T Z C Xi is solved by Alg. 4
    (geneig) and the estimate is Tr Xi.  Readings: W^T Z, symmetric in exact
    arithmetic, is symmetrised (geneig does so); Alg. 4's rounding floor is
    rounding_floor over the degree-M table (K_W = sum_{l<=M} mu_l W^T V_l).
    estimator "pinv" replaces Alg. 4 by Tr[K_W^+ K_Z] as in ress_dgc.
    Memory: n_t blocks of N x n_v.
    """
    if estimator not in ("alg4", "pinv"):
        raise ValueError(estimator)
    A = sp.csr_matrix(A)
    N = A.shape[0]
    W = np.asarray(W, dtype=np.float64)
    n_v = W.shape[1]
    a, b = interval if interval is not None else spectral_interval(A)
    At = transform(A, a, b)
    tab = coefficient_tables(t, M, sigma, N, a, b, n_theta, damping, lam)
    mu = tab["mu_full"]
    nt = len(t)
    Z = np.zeros((nt, N, n_v))
    Vm = np.zeros_like(W)
    Vc = W.copy()
    for l in range(M + 1):
        Z += mu[:, l][:, None, None] * Vc[None, :, :]
        if l < M:
            Vp = (1.0 if l == 0 else 2.0) * (At @ Vc) - Vm
            Vm, Vc = Vc, Vp
    X0 = (W.T @ W)[None]
    gm = g_max(sigma, N)
    dos = np.zeros(nt)
    rank_s = np.zeros(nt, dtype=np.int64)
    rank_xi = np.zeros(nt, dtype=np.int64)
    flags = np.zeros(nt, dtype=bool)
    for i in range(nt):
        K_W = W.T @ Z[i]
        K_Z = Z[i].T @ Z[i]
        fl = rounding_floor(mu[i], X0, n_v, eps_floor) if eps_floor > 0 else 0.0
        if estimator == "pinv":
            dos[i], info = pinv_trace(K_W, K_Z, tau, flag_eps, fl)
        else:
            xi, _, info = geneig(K_W, K_Z, gm, tau, kappa, flag_eps, fl)
            dos[i] = float(np.sum(xi))
        rank_s[i], rank_xi[i], flags[i] = info["rank_s"], info["rank_xi"], info["flagged"]
    return dict(dos_ss=dos, rank_s=rank_s, rank_xi=rank_xi, flagged=flags, a=a, b=b, mu_full=mu)


# --------------------------------------------------------------------------
# Reference quantities (Eq. DOS0, Eq. error)
# --------------------------------------------------------------------------

def exact_dos(eigs: np.ndarray, t: np.ndarray, sigma: float) -> np.ndarray:
    """phi_sigma(t) = sum_i g_sigma(t - lambda_i) from a full eigenvalue list."""
    eigs = np.asarray(eigs, dtype=np.float64)
    N = eigs.size
    return g_sigma(np.asarray(t)[:, None] - eigs[None, :], sigma, N).sum(axis=1)


def relative_l1_error(approx: np.ndarray, exact: np.ndarray) -> float:
    """sum_i |phi~_i - phi_i| / sum_i |phi_i| (Eq. error)."""
    return float(np.sum(np.abs(approx - exact)) / np.sum(np.abs(exact)))


# --------------------------------------------------------------------------
# Trace of a matrix function (Section 5, Eq. hform, pifunc, Alg. 8)
# --------------------------------------------------------------------------

DECONV_CUTOFF = 1e-14


def trace_grid(lo: float, hi: float, n_t: int, a: float = 0.93):
    """Uniform periodic grid for Alg. 8.

    The spectral bounds [lo, hi] are mapped onto [-a, a] of the unit
    variable t~ (centre c, half-width hw = (hi-lo)/(2a)); t~_i = -1 + 2i/n_t;
    x_i = c + hw t~_i.  Returns (t~, x, dx, c, hw).
    """
    c = 0.5 * (lo + hi)
    hw = 0.5 * (hi - lo) / a
    tt = -1.0 + 2.0 * np.arange(n_t) / n_t
    x = c + hw * tt
    return tt, x, hw * 2.0 / n_t, c, hw


def pi_window(tt: np.ndarray, a: float, sigma_tilde: float) -> np.ndarray:
    """pi(t) = 1/2 [erf((1+a-2t)/s~) - erf((-1-a-2t)/s~)] (Eq. pifunc)."""
    return 0.5 * (erf((1.0 + a - 2.0 * tt) / sigma_tilde) - erf((-1.0 - a - 2.0 * tt) / sigma_tilde))


def deconvolve_h(f: Callable, n_t: int, lo: float, hi: float, sigma: float,
                 sigma_tilde: float = 0.016, a: float = 0.93):
    """f~ on the periodic grid with (f~ * G_sigma) = h (Eq. deconvolv, hform).

    h(t~) = f(x(t~)) pi(t~) + (f(x(-1)) + f(x(1)))/2 (1 - pi(t~)); G_sigma is
    the unit-mass Gaussian N g_sigma; the convolution is the exact circular
    one on the grid, dx sum_j f~_j G(x_i - x_j), solved by the DFT.  f must
    be defined on the whole grid [c - hw, c + hw].  Frequencies at which the
    kernel's DFT is below DECONV_CUTOFF of its peak are set to zero: the
    method assumes h's spectrum decays faster than the Gaussian's, so only
    rounding is left there, and dividing it by an underflowed kernel would
    not be defined.
    Returns (x, dx, ftilde, h).
    """
    tt, x, dx, c, hw = trace_grid(lo, hi, n_t, a)
    fend = 0.5 * (f(c - hw) + f(c + hw))
    pw = pi_window(tt, a, sigma_tilde)
    h = f(x) * pw + fend * (1.0 - pw)
    L = n_t * dx
    off = dx * (((np.arange(n_t) + n_t // 2) % n_t) - n_t // 2)
    kern = np.zeros(n_t)
    for m in range(-3, 4):
        kern += np.exp(-((off + m * L) ** 2) / (2.0 * sigma * sigma))
    kern /= math.sqrt(2.0 * math.pi * sigma * sigma)
    khat = dx * np.fft.fft(kern)
    keep = np.abs(khat) >= DECONV_CUTOFF * np.max(np.abs(khat))
    fhat = np.zeros(n_t, dtype=np.complex128)
    fhat[keep] = np.fft.fft(h)[keep] / khat[keep]
    ft = np.fft.ifft(fhat).real
    return x, dx, ft, h


def trace_f(f: Callable, N: int, dos_at: Callable, n_t: int, lo: float, hi: float,
            sigma: float, sigma_tilde: float = 0.016, a: float = 0.93) -> float:
    """Tr f(A) ~ N dx sum_i f~(x_i) phi~_sigma(x_i) (Alg. 8).

    dos_at(x) returns the regularised DOS estimate at the grid points.
    """
    x, dx, ft, _ = deconvolve_h(f, n_t, lo, hi, sigma, sigma_tilde, a)
    return float(N * dx * np.sum(ft * dos_at(x)))


def logdet_shifted(A: sp.spmatrix, shift: float) -> float:
    """log det(A + shift I) = Tr log(A + shift I) for A + shift I positive definite,
    from a sparse LU factorisation (sum of log |U_ii|; minimum-degree ordering of
    A + A^T).  The exact reference for Tr f(A) with f(t) = log(t + shift)
    (Section 5's log-determinant application), exact up to the factorisation's
    rounding."""
    import scipy.sparse.linalg as spla

    B = sp.csc_matrix(sp.csr_matrix(A) + shift * sp.identity(A.shape[0]))
    lu = spla.splu(B, permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
    return float(np.sum(np.log(np.abs(lu.U.diagonal()))))
