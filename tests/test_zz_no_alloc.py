"""The allocation-free Gram pair matches the allocating one.

ssm_gram_pair_noalloc serves callers that cannot call cudaMalloc (memory
owned by another pool, latency-critical paths, hosts that forbid raw CUDA
allocations): it keeps its partial sums in a fixed device array instead.
This file is collected last so that a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1504_07690_gb300 import _native as N

    return N.load()


def _call(lib, name, A, B, Gaa, Gab, stream):
    fn = getattr(lib, name)
    n_rows, n_cols = A.shape
    return fn(A.data_ptr(), None if B is None else B.data_ptr(), n_rows, n_cols, n_cols, Gaa.data_ptr(),
              None if Gab is None else Gab.data_ptr(), stream)


# (rows, columns, with B): slices clamped by the scratch (200 columns), a ragged
# small case, G_aa alone (B = NULL), and the limit of 512 columns, where one
# slice fills the whole 4 MiB array
SHAPES = [(9001, 200, True), (4097, 37, True), (3001, 150, False), (2049, 512, True)]


@pytest.mark.parametrize("n_rows,n_cols,with_b", SHAPES, ids=[f"{r}x{c}{'' if b else '-aa'}" for r, c, b in SHAPES])
def test_noalloc_gram_pair_matches_allocating_entry_point_twice(lib, n_rows, n_cols, with_b):
    rng = np.random.default_rng(23 + n_cols)
    stream = torch.cuda.current_stream().cuda_stream
    A = torch.from_numpy(rng.standard_normal((n_rows, n_cols))).cuda()
    B = torch.from_numpy(rng.standard_normal((n_rows, n_cols))).cuda() if with_b else None
    ref_aa = torch.empty((n_cols, n_cols), dtype=torch.float64, device="cuda")
    ref_ab = torch.empty_like(ref_aa) if with_b else None
    assert _call(lib, "ssm_gram_pair", A, B, ref_aa, ref_ab, stream) == 0
    torch.cuda.synchronize()
    scale_aa = ref_aa.abs().max().item()
    for _ in range(2):  # two calls in a row share the fixed scratch
        out_aa = torch.full_like(ref_aa, float("nan"))
        out_ab = torch.full_like(ref_ab, float("nan")) if with_b else None
        assert _call(lib, "ssm_gram_pair_noalloc", A, B, out_aa, out_ab, stream) == 0
        torch.cuda.synchronize()
        assert (out_aa - ref_aa).abs().max().item() <= 1e-13 * scale_aa
        if with_b:
            assert (out_ab - ref_ab).abs().max().item() <= 1e-13 * ref_ab.abs().max().item()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    A = torch.zeros((16, 513), dtype=torch.float64, device="cuda")
    G = torch.zeros((513, 513), dtype=torch.float64, device="cuda")
    st = lib.ssm_gram_pair_noalloc(A.data_ptr(), None, 16, 513, 513, G.data_ptr(), None,
                                   torch.cuda.current_stream().cuda_stream)
    assert st == 1  # SSM_EINVAL
    assert b"512" in lib.ssm_last_error(None)
