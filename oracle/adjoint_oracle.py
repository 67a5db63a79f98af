"""Plain FP64 CPU oracle for the adjoint of the Chebyshev moment recurrence.

TEST INFRASTRUCTURE ONLY.  Like ssm_oracle, this module is the slow,
obviously-correct reference that the CUDA path is checked against; only the
test suite, the package's smoke check and the benchmark's CPU-baseline leg
may import it, and it shares no code with the CUDA library.

The paper has no gradients.  What is differentiated here is the moment loop
exactly as Alg. 7 runs it (Section 2's map A~ = (2A - (a+b)I)/(b-a), then
V_0 = W, V_1 = A~ W, V_{l+1} = 2 A~ V_l - V_{l-1}, X_l = W^T V_l,
symmetrised), for a loss that depends on A only through the moments,

    L = sum_{l=0..M} <G_l, X_l>,     G_l = dL/dX_l  (any n_tot x n_tot matrices).

Readings taken (none is in the paper):
* [a, b] is held fixed: the spectral interval is a constant of the plan, not
  a function of A, so dL/dA = (2/(b-a)) dL/dA~.
* Only sym(G_l) matters, because X_l is symmetrised.
* dL/dA_ij is the derivative for a perturbation of the single stored entry
  (i, j) of this loop; only its symmetric part (symmetric_part) is a property
  of the loss, and a symmetric pair (i, j), (j, i) tied to one weight
  receives the sum of both entries of it.  A stencil's per-axis coupling offdiag[d] and its diagonal
  receive the directional derivative along d A / d offdiag[d], d A / d A_ii.

The adjoint is written out in the loop's own notation: with
Gbar_l = W sym(G_l) the direct gradient of L with respect to V_l, the
adjoint blocks U_l = dL/dV_l obey, from l = M down to 1,
    U_M = Gbar_M,  U_{M-1} = Gbar_{M-1} + 2 A~ U_M,
    U_l = Gbar_l + 2 A~ U_{l+1} - U_{l+2},
and since A~ enters V_1 = A~ V_0 once and every V_{l+1} (l >= 1) as 2 A~ V_l,
    dL/dA~ = U_1 V_0^T + sum_{l=1..M-1} 2 U_{l+1} V_l^T,
read on the sparsity pattern of A (plus its diagonal).
"""
from __future__ import annotations

from typing import Tuple

import numpy as np
import scipy.sparse as sp

__all__ = ["moments_forward_blocks", "moments_adjoint_direct", "grad_wrt_a", "symmetric_part",
           "stencil_parameter_grad", "kpm_loss_weights", "moments_linear_loss"]


def moments_forward_blocks(At: sp.spmatrix, W: np.ndarray, M: int):
    """V_0..V_M of Alg. 7's loop (V_{l+1} = (2 - delta_l0) A~ V_l - V_{l-1}), dtype-generic."""
    W = np.asarray(W)
    V = [W, At @ W]
    for l in range(1, M):
        V.append(2.0 * (At @ V[l]) - V[l - 1])
    return V[: M + 1]


def moments_linear_loss(At: sp.spmatrix, W: np.ndarray, M: int, G: np.ndarray):
    """L = sum_l <G_l, sym(W^T V_l)> evaluated in the dtype of At (complex allowed)."""
    V = moments_forward_blocks(At, W, M)
    L = 0.0
    for l in range(M + 1):
        X = np.asarray(W).T @ V[l]
        L = L + np.sum(G[l] * 0.5 * (X + X.T))
    return L


def moments_adjoint_direct(At: sp.spmatrix, W: np.ndarray, M: int, G: np.ndarray,
                           pattern: sp.spmatrix = None) -> Tuple[np.ndarray, sp.csr_matrix]:
    """dL/dA~ for L = sum_l <G_l, X_l>, by the reverse of the M-step loop.

    Returns (d_diag, d_pat): d_diag[i] = dL/dA~_ii and d_pat a CSR matrix with
    the sparsity pattern of `pattern` (default: A~'s) holding dL/dA~_ij for
    every stored entry.
    """
    At = sp.csr_matrix(At)
    W = np.asarray(W, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    if G.shape[0] != M + 1:
        raise ValueError("need M+1 matrices G_l")
    Gs = 0.5 * (G + np.transpose(G, (0, 2, 1)))
    V = moments_forward_blocks(At, W, M)
    Gbar = [W @ Gs[l] for l in range(M + 1)]
    U = [None] * (M + 3)
    zero = np.zeros_like(W)
    U[M + 1] = zero
    U[M + 2] = zero
    for l in range(M, 0, -1):
        U[l] = Gbar[l] + 2.0 * (At @ U[l + 1]) - U[l + 2]
    # dL/dA~_ij = sum_l c_l <U_{l+1}[i,:], V_l[j,:]>, c_0 = 1, c_l = 2 (l >= 1)
    n = W.shape[0]
    P = sp.csr_matrix(At if pattern is None else pattern)
    P.sort_indices()
    rows = np.repeat(np.arange(n), np.diff(P.indptr))
    cols = P.indices
    vals = np.zeros(cols.size)
    diag = np.zeros(n)
    for l in range(M):
        c = 1.0 if l == 0 else 2.0
        vals += c * np.einsum("ek,ek->e", U[l + 1][rows], V[l][cols])
        diag += c * np.einsum("ik,ik->i", U[l + 1], V[l])
    d_pat = sp.csr_matrix((vals, P.indices.copy(), P.indptr.copy()), shape=P.shape)
    return diag, d_pat


def symmetric_part(d_pat: sp.csr_matrix) -> sp.csr_matrix:
    """(G + G^T)/2 on a symmetric pattern: the gradient with respect to a symmetric A.

    For a symmetric A~ the moments do not change under a perturbation E - E^T,
    so only the symmetric part of dL/dA~ is a property of the loss; the reverse
    of a different but equivalent loop (e.g. by the doubling identities, which
    hold for symmetric A~ only) may differ in the antisymmetric part.
    """
    P = sp.csr_matrix(d_pat)
    S = 0.5 * (P + P.T)
    # read back on P's own pattern and order
    rows = np.repeat(np.arange(P.shape[0]), np.diff(P.indptr))
    vals = np.asarray(S[rows, P.indices]).ravel()
    return sp.csr_matrix((vals, P.indices.copy(), P.indptr.copy()), shape=P.shape)


def grad_wrt_a(d_tilde, a: float, b: float):
    """Chain rule through A~ = (2A - (a+b)I)/(b-a) with [a, b] fixed: dA~/dA_ij = 2/(b-a)."""
    return d_tilde * (2.0 / (b - a))


def stencil_parameter_grad(dA_pat: sp.csr_matrix, dA_diag: np.ndarray, st, csr_of) -> Tuple[np.ndarray, np.ndarray]:
    """Gradient with respect to a stencil's diagonal and per-axis couplings.

    A = diag(st.diag) + sum_d offdiag[d] E_d, with E_d the (0/1, duplicates
    summed) adjacency of axis d as csr_of builds it.  dL/d diag_i = dL/dA_ii and
    dL/d offdiag[d] = sum_ij (E_d)_ij dL/dA_ij, the pattern and the diagonal
    read from (dA_pat, dA_diag).
    """
    import dataclasses
    n = dA_diag.size
    g_off = np.zeros(3)
    dense_lookup = sp.csr_matrix(dA_pat)
    for d in range(3):
        off = [0.0, 0.0, 0.0]
        off[d] = 1.0
        unit = dataclasses.replace(st, diag=np.zeros(n), offdiag=tuple(off))
        E = csr_of(unit)
        Ed = sp.csr_matrix((np.asarray(E.val, np.float64), np.asarray(E.colind), np.asarray(E.rowptr)),
                           shape=(n, n))
        # diagonal entries of E_d (self-loops of periodic extent-1 axes) pair with dA_diag
        ed = Ed.diagonal()
        Eoff = Ed - sp.diags(ed)
        g_off[d] = float(Eoff.multiply(dense_lookup).sum()) + float(np.dot(ed, dA_diag))
    return dA_diag.copy(), g_off


def kpm_loss_weights(mu_full: np.ndarray, dL_dphi: np.ndarray, n_cols: int) -> np.ndarray:
    """g_l with dL/dX_l = g_l I for a loss of the KPM line phi(t_i) = sum_l mu_l(t_i) tr X_l / n_cols
    (Alg. 2): g_l = sum_i dL/dphi(t_i) mu_l(t_i) / n_cols."""
    return (np.asarray(dL_dphi, np.float64) @ np.asarray(mu_full, np.float64)) / n_cols
