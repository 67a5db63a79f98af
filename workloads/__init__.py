"""Seeded synthetic inputs for the spectrum sweeping DOS estimator.

This module builds operators and random probe blocks only.  It holds none of
the estimator's arithmetic (no spectral map, no Chebyshev coefficients, no
moments, no trace estimation), so both the CPU oracle and the CUDA path can
take their inputs from here without sharing any of the method.

The paper's test matrices (Section 6: ModES3D, a 7-point periodic -Laplacian
plus a Gaussian potential; pe3k and shwater from the University of Florida
collection) are not available; the generators below stand in for them with
the same structure: 5- or 7-point stencils with a random diagonal potential,
and sparse symmetric graph Laplacians with 5-10 nonzeros per row.

Grid convention for stencils: ``dims = (d0, d1, d2)`` (unused trailing axes
have extent 1), row index ``i = (i0 * d1 + i1) * d2 + i2`` (C order, the last
axis fastest).  The operator is

    (A v)_i = diag[i] v_i + sum_axis offdiag[axis] (v_{i - s} + v_{i + s})

where the two neighbours along an axis wrap around when that axis is
periodic and are absent past a Dirichlet boundary.  Duplicate neighbours
(periodic extent 1 or 2) add up.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Stencil",
    "CSR",
    "stencil_to_csr",
    "laplacian2d_dirichlet_potential",
    "anderson2d",
    "laplacian3d_lognormal",
    "laplacian3d_normal_potential",
    "er_normalized_laplacian",
    "random_block",
    "CONFIGS",
    "make_operator",
    "sweep_points",
    "er_batch",
]


@dataclasses.dataclass
class Stencil:
    """A (2*ndim+1)-point constant-coefficient stencil plus a diagonal."""

    dims: Tuple[int, int, int]
    periodic: Tuple[bool, bool, bool]
    diag: np.ndarray  # float64, length prod(dims)
    offdiag: Tuple[float, float, float]

    @property
    def n(self) -> int:
        return int(self.dims[0] * self.dims[1] * self.dims[2])

    @property
    def ndim(self) -> int:
        return sum(1 for d in self.dims if d > 1) or 1


@dataclasses.dataclass
class CSR:
    """Symmetric sparse matrix, full storage, sorted column indices."""

    n: int
    rowptr: np.ndarray  # int64, n+1
    colind: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def stencil_to_csr(st: Stencil) -> CSR:
    """Expand a stencil descriptor into explicit CSR (duplicates summed)."""
    d0, d1, d2 = st.dims
    n = st.n
    idx = np.arange(n, dtype=np.int64).reshape(d0, d1, d2)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.asarray(st.diag, dtype=np.float64).ravel()]
    for axis in range(3):
        ext = st.dims[axis]
        c = float(st.offdiag[axis])
        if c == 0.0 or (ext == 1 and not st.periodic[axis]):
            continue
        for shift in (-1, +1):
            src = idx
            dst = np.roll(idx, -shift, axis=axis)  # neighbour i + shift along axis
            if not st.periodic[axis]:
                pos = np.arange(ext)
                keep = (pos + shift >= 0) & (pos + shift < ext)
                shape = [1, 1, 1]
                shape[axis] = ext
                mask = np.broadcast_to(keep.reshape(shape), idx.shape)
                r = src[mask]
                q = dst[mask]
            else:
                r = src.ravel()
                q = dst.ravel()
            rows.append(r.ravel())
            cols.append(q.ravel())
            vals.append(np.full(r.size, c))
    r = np.concatenate(rows)
    q = np.concatenate(cols)
    v = np.concatenate(vals)
    return _coo_to_csr(n, r, q, v)


def _coo_to_csr(n: int, r: np.ndarray, q: np.ndarray, v: np.ndarray) -> CSR:
    key = r.astype(np.int64) * n + q.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key = key[order]
    v = v[order]
    uniq, start = np.unique(key, return_index=True)
    vsum = np.add.reduceat(v, start) if v.size else v
    rr = (uniq // n).astype(np.int64)
    cc = (uniq % n).astype(np.int32)
    counts = np.bincount(rr, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n=n, rowptr=rowptr, colind=cc, val=vsum.astype(np.float64))


def laplacian2d_dirichlet_potential(nx: int, seed: int, amp: float = 1.0) -> Stencil:
    """2D 5-point -Laplacian (diag 4, off -1), Dirichlet, plus v ~ U[-amp, amp]."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-amp, amp, size=nx * nx)
    return Stencil(dims=(nx, nx, 1), periodic=(False, False, False),
                   diag=4.0 + v, offdiag=(-1.0, -1.0, 0.0))


def anderson2d(nx: int, seed: int, w: float = 2.0, hop: float = -1.0) -> Stencil:
    """2D Anderson tight-binding: periodic, hopping ``hop``, on-site U[-w, w]."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(-w, w, size=nx * nx)
    return Stencil(dims=(nx, nx, 1), periodic=(True, True, False),
                   diag=eps, offdiag=(hop, hop, 0.0))


def laplacian3d_lognormal(nx: int, seed: int, s: float = 0.5) -> Stencil:
    """3D 7-point -Laplacian (diag 6, off -1), periodic, plus LogNormal(0, s)."""
    rng = np.random.default_rng(seed)
    v = rng.lognormal(0.0, s, size=nx ** 3)
    return Stencil(dims=(nx, nx, nx), periodic=(True, True, True),
                   diag=6.0 + v, offdiag=(-1.0, -1.0, -1.0))


def laplacian3d_normal_potential(nx: int, seed: int, s: float = 0.3) -> Stencil:
    """3D 7-point -Laplacian, periodic, plus a N(0, s^2) diagonal potential."""
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, s, size=nx ** 3)
    return Stencil(dims=(nx, nx, nx), periodic=(True, True, True),
                   diag=6.0 + v, offdiag=(-1.0, -1.0, -1.0))


def er_normalized_laplacian(n: int, mean_degree: float, seed: int,
                            wlo: float = 0.5, whi: float = 1.5) -> CSR:
    """Symmetric normalized Laplacian I - D^-1/2 W D^-1/2 of a weighted G(n, p).

    p = mean_degree / (n - 1); no self loops; weights U[wlo, whi]; an
    isolated vertex gets L_ii = 0.
    """
    rng = np.random.default_rng(seed)
    p = mean_degree / max(n - 1, 1)
    m = rng.binomial(n * (n - 1) // 2, p)
    i = rng.integers(0, n, size=2 * m + 16)
    j = rng.integers(0, n, size=2 * m + 16)
    keep = i != j
    a = np.minimum(i[keep], j[keep])
    b = np.maximum(i[keep], j[keep])
    key = np.unique(a.astype(np.int64) * n + b)[:m]
    a = (key // n).astype(np.int64)
    b = (key % n).astype(np.int64)
    wgt = rng.uniform(wlo, whi, size=a.size)
    deg = np.bincount(a, weights=wgt, minlength=n) + np.bincount(b, weights=wgt, minlength=n)
    dinv = np.where(deg > 0, 1.0 / np.sqrt(np.where(deg > 0, deg, 1.0)), 0.0)
    off = -wgt * dinv[a] * dinv[b]
    diag = np.where(deg > 0, 1.0, 0.0)
    r = np.concatenate([a, b, np.arange(n)])
    q = np.concatenate([b, a, np.arange(n)])
    v = np.concatenate([off, off, diag])
    return _coo_to_csr(n, r, q, v)


def random_block(n: int, ncols: int, seed: int, kind: str = "gaussian") -> np.ndarray:
    """N x ncols probe block (row-major float64): Gaussian N(0,1) or Rademacher."""
    rng = np.random.default_rng(seed)
    if kind == "gaussian":
        return rng.standard_normal((n, ncols))
    if kind == "rademacher":
        return rng.integers(0, 2, size=(n, ncols)).astype(np.float64) * 2.0 - 1.0
    raise ValueError(f"unknown probe kind {kind!r}")


def sweep_points(lo: float, hi: float, n_t: int) -> np.ndarray:
    """n_t points uniform on the closed interval [lo, hi]."""
    return np.linspace(lo, hi, n_t)


def explicit_points(lo: float, hi: float, n_t: int = 16) -> np.ndarray:
    """The few sweep points of the explicit-block (SS-DGC) runs: n_t points uniform
    strictly inside [lo, hi] (the ends of a Gershgorin interval carry no spectrum)."""
    return np.linspace(lo, hi, n_t + 2)[1:-1]


# Workload recipes (operator seed 1000+k, probe seed 2000+k).
CONFIGS = {
    "lap2d_dirichlet_32": dict(
        op="lap2d_dirichlet", nx=32, op_seed=1001, n_v=40, n_vh=0, probe="gaussian",
        probe_seed=2001, M=200, n_t=101, sigma=0.05),
    "anderson2d_256": dict(
        op="anderson2d", nx=256, op_seed=1002, n_v=200, n_vh=0, probe="rademacher",
        probe_seed=2002, M=1000, n_t=400, sigma=0.02),
    "lap3d_lognormal_64": dict(
        op="lap3d_lognormal", nx=64, op_seed=1003, n_v=256, n_vh=0, probe="gaussian",
        probe_seed=2003, M=2000, n_t=800, sigma=0.06),
    # B normalized Laplacians of G(N_b, 8/(N_b-1)), N_b ~ U{2000..60000}
    "er_batch_128": dict(
        op="er_batch", B=128, n_lo=2000, n_hi=60000, mean_degree=8.0, op_seed=1004, n_v=64, n_vh=0,
        probe="gaussian", probe_seed=2004, M=500, n_t=200, sigma=0.05),
    # trainable N(0, 0.3^2) potential on a 100^3 periodic 7-point Laplacian
    "lap3d_normal_100": dict(
        op="lap3d_normal", nx=100, op_seed=1005, n_v=128, n_vh=0, probe="gaussian",
        probe_seed=2005, M=800, n_t=400, sigma=0.05, target_seed=3005),
}


def er_batch(B: int, n_lo: int, n_hi: int, mean_degree: float, seed: int):
    """B weighted ER normalized Laplacians with sizes uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, size=B)
    return [er_normalized_laplacian(int(n), mean_degree, seed * 1000 + k) for k, n in enumerate(sizes)]


def make_operator(name: str, **over) -> Stencil:
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    op = cfg["op"]
    if op == "lap2d_dirichlet":
        return laplacian2d_dirichlet_potential(cfg["nx"], cfg["op_seed"])
    if op == "anderson2d":
        return anderson2d(cfg["nx"], cfg["op_seed"])
    if op == "lap3d_lognormal":
        return laplacian3d_lognormal(cfg["nx"], cfg["op_seed"])
    if op == "lap3d_normal":
        return laplacian3d_normal_potential(cfg["nx"], cfg["op_seed"])
    if op == "er_batch":
        return er_batch(cfg["B"], cfg["n_lo"], cfg["n_hi"], cfg["mean_degree"], cfg["op_seed"])
    raise ValueError(op)
