"""The row-partitioned form of the moment computation on CPU ranks (the multi-GPU split of a
single large operator, which this single-GPU build does not run on hardware).

Two gloo ranks on 127.0.0.1 each own a contiguous slab of rows of A~ and of the probe
block.  Per recurrence step a rank needs the rows of V_k its slab's stencil couples to, so
the slabs of V_k are exchanged (an all-gather standing in for the halo exchange), and each
rank forms its rows of V_{k+1} = 2 A~ V_k - V_{k-1}.  The Gram products of the doubling
identities (X_{2k} = 2 V_k^T V_k - X_0, X_{2k+1} = 2 V_{k+1}^T V_k - X_1) are sums over rows,
so every rank forms them over its own rows and one SUM all-reduce per step joins them.  The
joined moments must equal the oracle's unpartitioned Alg. 7 loop (moments_direct) to
rounding, whatever the split: an even split and a ragged one are checked.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import workloads as wl  # noqa: E402
from oracle import ssm_oracle as O  # noqa: E402

M = 24


def _problem():
    st = wl.anderson2d(12, 3301)
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    a, b = O.spectral_interval(A)
    At = O.transform(A, a, b)
    W = wl.random_block(c.n, 6, 3302, "rademacher")
    return At, W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, cut, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        At, W = _problem()
        n, nc = W.shape
        r0, r1 = (0, cut) if rank == 0 else (cut, n)
        rows = At[r0:r1]  # this rank's rows of A~ (all columns)
        sizes = [cut, n - cut]

        def gather(v_loc):
            # gloo gathers equal shapes: slabs padded to the larger one, then trimmed
            mx = max(sizes)
            pad = np.zeros((mx, nc))
            pad[:v_loc.shape[0]] = v_loc
            parts = [torch.zeros((mx, nc), dtype=torch.float64) for _ in sizes]
            dist.all_gather(parts, torch.from_numpy(pad))
            return np.vstack([p.numpy()[:sz] for p, sz in zip(parts, sizes)])

        def allsum(g):
            t = torch.from_numpy(np.ascontiguousarray(g))
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.numpy()

        S = M // 2
        X = np.zeros((M + 1, nc, nc))
        v_prev = None
        v_cur = W[r0:r1].copy()
        X0 = allsum(v_cur.T @ v_cur)
        X[0] = X0
        X1 = None
        for k in range(S):
            full = gather(v_cur)  # the rows of V_k the slab couples to (here: all of them)
            if k == 0:
                v_next = rows @ full
            else:
                v_next = 2.0 * (rows @ full) - v_prev
            ge = allsum(v_next.T @ v_next)  # V_{k+1}^T V_{k+1}, summed over both slabs
            go = allsum(v_next.T @ v_cur)   # V_{k+1}^T V_k
            if k == 0:
                X1 = 0.5 * (go + go.T)
                X[1] = X1
            else:
                X[2 * k + 1] = (go + go.T) - X1
            X[2 * k + 2] = 2.0 * ge - X0
            v_prev, v_cur = v_cur, v_next
        if rank == 0:
            out.put(X)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("cut", [72, 53])
def test_row_partitioned_moments_equal_the_unpartitioned_loop(cut):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, cut, out)) for r in range(2)]
    for p in procs:
        p.start()
    X = out.get(timeout=60)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    At, W = _problem()
    Xr = O.moments_direct(At, W, M)
    assert np.max(np.abs(X - Xr)) <= 1e-12 * np.max(np.abs(Xr))
