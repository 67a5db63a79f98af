"""The N > 1 path of bench.py on the CPU: ranks are independent replicas (the operator
is not partitioned), the job's time per step is the slowest rank's (a MAX all-reduce
over the process group) and the job's value counts every rank's units.  Run as two
gloo ranks on 127.0.0.1; the reference arm prints from rank 0 only."""
import io
import os
import socket
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench._dist()
        t = bench.over_ranks(times[r], dist)
        out.put((r, w, t, bench.whole_job_value(1e12, w, t)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.5, 0.75), (2.0, 1.0)])
def test_two_gloo_ranks_take_the_slowest_time_and_count_both_replicas(times):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(out.get(timeout=5) for _ in range(2))
    slow = max(times)
    for r, (rank, ws, t, value) in enumerate(res):
        assert rank == r and ws == 2
        assert t == slow
        assert value == pytest.approx(2 * 1e12 / slow, rel=1e-15)


def test_single_rank_needs_no_process_group():
    assert bench.over_ranks(3.25, None) == 3.25
    assert bench.whole_job_value(10.0, 1, 2.0) == 5.0


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    # under torchrun only rank 0 times the oracle and prints; the others exit without work
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda *a, **k: called.append(1) or (1.0, ""))
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(None, {"n_v": 1, "n_vh": 0, "M": 2}, None, None, None) is None
    assert buf.getvalue() == "" and not called
