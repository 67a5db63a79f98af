"""Failure detection without faulting the GPU.

* Bounded waits: the mbarrier wait every tensor-core kernel uses gives up
  after its poll limit and reports SSM_ETIMEOUT (nothing in flight; the kernel
  returns normally), and the device stays usable: a plan runs afterwards and
  matches the oracle.
* Allocation failures: the library's allocation hook makes the k-th device
  allocation of a plan's life fail; every such call returns SSM_ENOMEM,
  releases what it had allocated (device memory back to where it was), and
  a plan created after the hook is disarmed works.
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


def _small_run(S, precision="fp64"):
    st = wl.make_operator("lap2d_dirichlet_32", nx=12)
    W = wl.random_block(st.n, 8, 41)
    plan = S.ssm_plan_create(stencil=st, n_v=6, n_vh=2, degree=40, precision=precision)
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], 9)
    X = S.ssm_moments(plan, W, return_moments=True)
    ss, kpm, rank = S.ssm_dos(plan, t, 0.3)
    c = wl.stencil_to_csr(st)
    r = O.ress_dgc(O.csr_matrix(c.n, c.rowptr, c.colind, c.val), W, 6, t, 40, 0.3, interval=(info["a"], info["b"]))
    plan.close()
    return X, kpm, r


def test_bounded_wait_reports_timeout_and_device_stays_usable(S):
    S.ssm_selftest_wait(1000, arrive=True)  # the phase completes: SSM_OK
    for polls in (1, 64, 4096):
        with pytest.raises(S.SSMError) as e:
            S.ssm_selftest_wait(polls, arrive=False)
        assert e.value.name == "SSM_ETIMEOUT"
    with pytest.raises(S.SSMError) as e:
        S.ssm_selftest_wait(0, arrive=False)
    assert e.value.name == "SSM_EINVAL"
    X, kpm, r = _small_run(S)
    assert np.max(np.abs(X - r["X"])) <= 1e-11 * np.max(np.abs(r["X"]))
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp64_tc"])
def test_every_allocation_failure_returns_enomem_and_releases(S, precision):
    st = wl.make_operator("lap2d_dirichlet_32", nx=12)
    W = wl.random_block(st.n, 8, 41)
    t = np.linspace(-1.0, 9.0, 9)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    k, failures = 0, 0
    try:
        while True:
            S.ssm_debug_fail_alloc(k)
            try:
                plan = S.ssm_plan_create(stencil=st, n_v=6, n_vh=2, degree=40, precision=precision)
                S.ssm_moments(plan, W)
                S.ssm_dos(plan, t, 0.3)
                plan.close()
                break  # every allocation of the run succeeded: all failure points visited
            except S.SSMError as e:
                assert e.name == "SSM_ENOMEM", (k, e)
                failures += 1
            k += 1
            assert k < 200
    finally:
        S.ssm_debug_fail_alloc(-1)
    assert failures >= 5
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 64 << 20  # nothing held on (allocator granularity)
    X, kpm, r = _small_run(S, precision)
    tol = 1e-4 if precision == "mixed" else 1e-10
    assert O.relative_l1_error(kpm, r["dos_kpm"]) <= tol
