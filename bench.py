"""Benchmark of the spectrum sweeping DOS hot path on one GB300 (or N replicas).

One step = one pass of the whole hot path on the 2D Anderson workload
(256 x 256 periodic, hopping -1, on-site U[-2, 2]; N = 65536, nnz = 327680),
N_v = 200 Rademacher probes, degree M = 1000, 400 sweep points, sigma = 0.02:
  ssm_moments  - spectral map, M/2 recurrence steps with the doubling Gram
                 products, float64 moments;
  ssm_dos      - Alg. 1 / Prop. 1 coefficient tables, per-point assembly,
                 Alg. 4 + Alg. 6 solves (RESS-DGC) and the KPM line.
Metric: effective matrix-applies/s = nnz * n_tot * M / t_step.
The line also carries, per precision (mixed, fp64_tc, fp64), its ms/step and
the relative L1 error of both DOS lines against the CPU oracle run on the
same workload (Eq. error; the oracle takes about a minute on the host).

--impl reference times the CPU oracle (plain float64 numpy/scipy from the
paper's formulas) on a bounded sample of the same workload.
Multi-GPU: the operator is not partitioned; every rank runs an independent
replica on its own GPU (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

CONFIG = "anderson2d_256"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", 0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of every rank's x (its time per step): the job's time is its slowest
    replica's.  dist: torch.distributed with an initialised process group, or None."""
    if dist is None:
        return float(x)
    import torch

    tt = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


UNIT = "matrix-applies/s (nnz*n_tot*M/s)"


def bench_config(nnz: int, ws: int) -> dict:
    """The workload both arms (this GPU path and the CPU oracle) are measured on."""
    return {"workload": "anderson2d_256: 2D Anderson 256x256 periodic, N=65536, nnz=%d, N_v=200 "
                        "rademacher, M=1000, 400 sweep points, sigma=0.02" % nnz,
            "l2": "inputs larger than L2 (3 recurrence blocks of 52 MB + 320 MB of moments)",
            "parallelism": "replicas" if ws > 1 else "single"}


def whole_job_value(units_per_replica: float, ws: int, seconds_per_step: float) -> float:
    """Throughput of the whole job: every replica processes the same units (weak scaling)."""
    return units_per_replica * ws / seconds_per_step


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _workload():
    c = dict(wl.CONFIGS[CONFIG])
    st = wl.make_operator(CONFIG)
    W = wl.random_block(st.n, c["n_v"] + c["n_vh"], c["probe_seed"], c["probe"])
    csr = wl.stencil_to_csr(st)
    return c, st, W, csr


def _hash_sources(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1504_07690_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, null if the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))[kernel]
    except Exception:
        return None
    if d.get("source_hash") != _hash_sources(d["sources"]):
        return None
    return d["dram_bytes_per_launch"]


# ----------------------------------------------------------------------------- rooflines

FP64_FMA_PER_SM_CLK = 2   # float64 FMAs per SM clock on this part (1.26 TFLOP/s at 2.07 GHz)


def fp64_gemm_tflops(n: int = 4096, reps: int = 5) -> float:
    """Measured float64 throughput of this GPU: cuBLAS DGEMM (torch.matmul) on n x n operands,
    timed with CUDA events after two warm-up products.  It is the denominator of the float64
    kernels' rooflines when it exceeds the per-clock figure above."""
    import torch

    g = torch.Generator(device="cuda").manual_seed(5)
    a = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    b = torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g)
    for _ in range(2):
        c = a @ b
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        c = a @ b
    e1.record()
    torch.cuda.synchronize()
    del a, b, c
    return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12


def solve_flops(ranks, n: int) -> float:
    """Float64 flops of the per-point solver, by the route each point takes ((r, r_s) per
    point: kept rank, eigenvalues inside the filter; the paths that run when every test
    passes):
    r = n: the full-rank test (Cholesky of K_W less the threshold, n^3/3), the inertia test
    by congruence (two Choleskys, 2/3 n^3), Cholesky of K_W (n^3/3) and the trace from a
    triangular solve with a triangular right-hand side (n^3/3): 5/3 n^3 (when the inertia
    test fails: two solves (2 n^3) and the reduction of C (4/3 n^3) instead of the last);
    r = 0: counted as nothing (the Gershgorin bound or one Cholesky of floor I - K_W decides);
    0 < r < n: reduction (4/3 n^3), then with d = n - r dropped directions and 3 d < r the
    dropped eigenvectors' back-transform (2 n^2 d) and two-sided reflections of K_W and K_Z
    (8 n^2 d), else the kept basis: back-transform (2 n^2 r), K_Z Y (2 n^2 r), Y^T K_Z Y and
    Z^T T Z (2 n r^2); then the r x r pencil as in the r = n case without the full-rank
    test (4/3 r^3, or 13/3 r^3 when the inertia test fails)."""
    tot = 0.0
    for r, rs in ranks:
        if r == n:
            f = 5.0 / 3.0 * n ** 3 if rs == r else (1.0 / 3.0 + 2.0 / 3.0 + 1.0 / 3.0 + 2.0 + 4.0 / 3.0) * n ** 3
        elif r == 0:
            f = 0.0
        else:
            d = n - r
            f = 4.0 / 3.0 * n ** 3 + (4.0 / 3.0 if rs == r else 13.0 / 3.0) * r ** 3
            if 3 * d < r:
                f += 10.0 * n * n * d
            else:
                f += 4.0 * n * n * r + 2.0 * n * r * r
        tot += f
    return tot


def stencil_kernel_name(st, mixed: bool) -> str:
    """The float32 step of a grid whose axes other than the last two have extent 1 (after
    dropping trailing axes of extent 1) is the row-group kernel; every other step the
    per-item kernel."""
    d = list(st.dims)
    while len(d) > 1 and d[-1] == 1:
        d.pop()
    return "stencil_march_kernel" if mixed and all(x == 1 for x in d[:-2]) else "stencil_step_kernel"


def kernel_rooflines(st, c, stats, args, hbm, bf16, peak_kind, clocks, ranks=None):
    """Per-kernel algorithmic work / measured launch time against its bound.

    Algorithmic work per launch:
      stencil_step_kernel  bytes = (3 N n_tot + N) e   (read V_k, V_{k-1}, diag; write V_{k+1}); on 2D
                           grids in float32 the row-group stencil_march_kernel, same bytes
      gram_tc_kernel       flops = 3 x 2 N (n_tot(n_tot+1)/2 + n_tot^2)   (split-bf16 products)
      gram_kernel (fp32)   flops = 2 N (n_tot(n_tot+1)/2 + n_tot^2)
      assemble_kernel      flops = 2 n_t ((M/2+1) n_tot(n_tot+1)/2 + (M+1) n_v(n_v+1)/2)   per step (fp64)
      assemble_oz_kernel   bf16 slice products issued for the same sums (mixed: 6 slices, fp64_tc: 7;
                           asm_oz_issued_flops); its time is the assembly phase, slicing included
      solve_kernel         flops = sum over points of the route's count (solve_flops)
    """
    N = st.n
    n_tot = c["n_v"] + c["n_vh"]
    nv = c["n_v"]
    M, n_t = c["M"], c["n_t"]
    steps = args.steps
    mixed = args.precision == "mixed"
    e = 4 if mixed else 8  # float64 and float pairs: 8 bytes a value
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    fp64_clk = 152 * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    dgemm = getattr(args, "fp64_gemm_tflops", None)
    if dgemm and dgemm > fp64_clk:
        fp64_peak, fp64_src = dgemm, "cuBLAS DGEMM 4096^3 measured in this run: %.3f TFLOP/s" % dgemm
    else:
        fp64_peak = fp64_clk
        fp64_src = "fp64: 152 SMs x 2 FMA/clk x 2 x %.0f MHz (cuBLAS DGEMM measured %s TFLOP/s)" % (
            sm_mhz, "%.3f" % dgemm if dgemm else "n/a")
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    out = []
    rl = max(1, stats["recurrence_launches"])
    rec_ms = stats["ms_recurrence"] / rl
    if args.precision == "fp64_tc":
        out = _rooflines_fp64tc(N, n_tot, stats, steps, rec_ms, hbm, bf16, peak_kind)
        a_flops = asm_oz_issued_flops(n_t, M, n_tot, nv, slices=7)
        a_ms = stats["ms_assemble"] / steps
        r = dict(kernel="assemble_oz_kernel", bound="tensor", achieved=a_flops / (a_ms * 1e-3) / 1e12, peak=bf16,
                 unit="TFLOP/s", traffic=None, work_per_launch=a_flops / 2, launch_ms=a_ms / 2, ms_per_step=a_ms,
                 peak_source=f"MEASURED_PEAKS.json bf16_tflops ({peak_kind}); issued bf16 slice products (7 slices)")
        r["frac"] = r["achieved"] / r["peak"]
        return out + [r]
    rec_bytes = (3.0 * N * n_tot + N) * e
    sk = stencil_kernel_name(st, mixed)
    out.append(dict(kernel=sk, bound="hbm", achieved=rec_bytes / (rec_ms * 1e-3) / 1e9,
                    peak=hbm, unit="GB/s", traffic=_traffic(sk), work_per_launch=rec_bytes,
                    launch_ms=rec_ms, ms_per_step=stats["ms_recurrence"] / steps,
                    peak_source=f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"))
    gl = max(1, stats["gram_launches"])
    g_ms = stats["ms_gram"] / gl
    pair = n_tot * (n_tot + 1) / 2.0 + n_tot * n_tot
    if mixed and n_tot <= 256:
        g_flops = 3.0 * 2.0 * N * pair
        out.append(dict(kernel="gram_tc_kernel", bound="tensor", achieved=g_flops / (g_ms * 1e-3) / 1e12,
                        peak=bf16, unit="TFLOP/s", traffic=_traffic("gram_tc_kernel"), work_per_launch=g_flops,
                        launch_ms=g_ms, ms_per_step=stats["ms_gram"] / steps,
                        peak_source=f"MEASURED_PEAKS.json bf16_tflops ({peak_kind})"))
    else:
        g_flops = 2.0 * N * pair
        pk = fp32_peak if mixed else fp64_peak
        out.append(dict(kernel="gram_kernel", bound="alu", achieved=g_flops / (g_ms * 1e-3) / 1e12, peak=pk,
                        unit="TFLOP/s", traffic=None, work_per_launch=g_flops, launch_ms=g_ms,
                        ms_per_step=stats["ms_gram"] / steps,
                        peak_source=("fp32 CUDA-core peak: 152 SMs x 128 FMA/clk x 2 x %.0f MHz" % sm_mhz)
                        if mixed else fp64_src))
    a_terms = n_t * ((M // 2 + 1) * n_tot * (n_tot + 1) / 2.0 + (M + 1) * nv * (nv + 1) / 2.0)
    a_ms = stats["ms_assemble"] / steps
    if mixed:
        # bf16 slice products issued by the two tensor-core assembly launches (the phase
        # also holds the slicing of the moments and coefficients)
        a_flops = asm_oz_issued_flops(n_t, M, n_tot, nv)
        out.append(dict(kernel="assemble_oz_kernel", bound="tensor", achieved=a_flops / (a_ms * 1e-3) / 1e12,
                        peak=bf16, unit="TFLOP/s", traffic=_traffic("assemble_oz_kernel"), work_per_launch=a_flops / 2,
                        launch_ms=a_ms / 2, ms_per_step=a_ms,
                        peak_source=f"MEASURED_PEAKS.json bf16_tflops ({peak_kind}); issued bf16 slice products"))
    else:
        a_flops = 2.0 * a_terms
        out.append(dict(kernel="assemble_kernel", bound="alu", achieved=a_flops / (a_ms * 1e-3) / 1e12,
                        peak=fp64_peak, unit="TFLOP/s", traffic=None, work_per_launch=a_flops / 2,
                        launch_ms=a_ms / 2, ms_per_step=a_ms,
                        peak_source=fp64_src))
    s_flops = solve_flops(ranks, nv) if ranks is not None else n_t * 14.3 * nv ** 3
    s_ms = stats["ms_solve"] / steps
    out.append(dict(kernel="solve_kernel", bound="alu", achieved=s_flops / (s_ms * 1e-3) / 1e12, peak=fp64_peak,
                    unit="TFLOP/s", traffic=None, work_per_launch=s_flops, launch_ms=s_ms, ms_per_step=s_ms,
                    peak_source=fp64_src))
    for r in out:
        r["frac"] = r["achieved"] / r["peak"]
    return out


def asm_oz_issued_flops(n_t: int, M: int, n_tot: int, nv: int, slices: int = 6) -> float:
    """bf16 flops the tensor cores issue for the tensor-core assembly: K (n_tot(n_tot+1)/2
    packed entries, l <= M/2) and K_Z (n_v(n_v+1)/2 entries, l <= M), 21 slice pairs each
    (six slices, mixed plans) or 28 (seven, float64-accurate plans); points rounded to 64,
    entries to 128, l to 16."""
    def up(x, m):
        return (x + m - 1) // m * m
    tp = up(n_t, 64)
    k = up(n_tot * (n_tot + 1) // 2, 128) * up(M // 2 + 1, 16)
    kz = up(nv * (nv + 1) // 2, 128) * up(M + 1, 16)
    pairs = slices * (slices + 1) // 2
    return pairs * 2.0 * tp * (k + kz)


def oz_issued_flops(N: int, n_tot: int) -> float:
    """bf16 flops the tensor cores issue for the two Gram products of one SSM_FP64_TC step:
    tile D0 (128 x min(n, 128)) and D1 (128 x (n - 128)) with the 12 slice pairs i <= j,
    i + j <= 7, tile O (128 x (n - 128)) with all 21 pairs; n = n_tot rounded to 16."""
    ntp = (n_tot + 15) // 16 * 16
    per_row = 12 * 128 * min(ntp, 128) * 2.0
    if ntp > 128:
        per_row += (21 + 12) * 128 * (ntp - 128) * 2.0
    return 2.0 * N * per_row


def _rooflines_fp64tc(N, n_tot, stats, steps, rec_ms, hbm, bf16, peak_kind):
    """SSM_FP64_TC: the float-pair recurrence step (read V_k, V_{k-1}, write V_{k+1}, U_k: 8 bytes
    a value, plus the diagonal pair) and the slice Gram products on the tensor cores."""
    ld = (n_tot + 3) // 4 * 4
    rec_bytes = 4.0 * N * ld * 8 + 8.0 * N
    gl = max(1, stats["gram_launches"])
    g_ms = stats["ms_gram"] / gl
    g_flops = oz_issued_flops(N, n_tot)
    out = [dict(kernel="stencil_step_df_kernel", bound="hbm", achieved=rec_bytes / (rec_ms * 1e-3) / 1e9, peak=hbm,
                unit="GB/s", traffic=_traffic("stencil_step_df_kernel"), work_per_launch=rec_bytes, launch_ms=rec_ms,
                ms_per_step=stats["ms_recurrence"] / steps, peak_source=f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"),
           dict(kernel="gram_oz_kernel", bound="tensor", achieved=g_flops / (g_ms * 1e-3) / 1e12, peak=bf16,
                unit="TFLOP/s", traffic=_traffic("gram_oz_kernel"), work_per_launch=g_flops, launch_ms=g_ms,
                ms_per_step=stats["ms_gram"] / steps,
                peak_source=f"MEASURED_PEAKS.json bf16_tflops ({peak_kind}); issued bf16 slice products")]
    for r in out:
        r["frac"] = r["achieved"] / r["peak"]
    return out


# ----------------------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(c, st, W, csr, rec_steps: int = 24, points: int = 6):
    """Time the CPU oracle on a bounded sample of the workload, scaled to one full step.

    Sample: the first `rec_steps` of the paper's M+1 three-term steps (Alg. 7
    loop with X_l = W^T V_l), and assembly + Alg. 4/6 at `points` sweep points
    with full-length moment tables; both scaled linearly to M+1 steps and n_t
    points (their costs are linear in those counts).
    """
    from oracle import ssm_oracle as O

    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    a, b = O.spectral_interval(A)
    At = O.transform(A, a, b)
    M, n_t, nv, sigma = c["M"], c["n_t"], c["n_v"], c["sigma"]
    t0 = time.perf_counter()
    Xs = O.moments_direct(At, W, rec_steps - 1)
    t_rec = time.perf_counter() - t0
    X = np.zeros((M + 1,) + Xs.shape[1:])
    X[: Xs.shape[0]] = Xs
    lo, hi = O.gershgorin(A)
    tpts = np.linspace(lo, hi, n_t)[:: max(1, n_t // points)][:points]
    t1 = time.perf_counter()
    tab = O.coefficient_tables(tpts, M, sigma, A.shape[0], a, b)
    gm = O.g_max(sigma, A.shape[0])
    for i in range(tpts.size):
        K = O.assemble(tab["mu_half"][i], tab["nu"][i], X, nv)
        O.ress_dos_point(*K, gm)
    O.kpm_dos(tab["mu_full"], X)
    t_pts = time.perf_counter() - t1
    t_step = t_rec * (M + 1) / rec_steps + t_pts * n_t / tpts.size
    sample = (f"{rec_steps} of {M + 1} recurrence+moment steps and {tpts.size} of {n_t} sweep points "
              f"(coefficients, assembly, Alg. 4/6), scaled linearly to one full step")
    return t_step, sample


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info

        info = threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return os.cpu_count()


def run_reference(args, c, st, W, csr):
    ws, rank, local = _dist()
    if rank != 0:
        return
    nnz = csr.nnz
    n_tot = c["n_v"] + c["n_vh"]
    units = float(nnz) * n_tot * c["M"]
    times = []
    sample = ""
    for i in range(args.warmup + args.steps):
        t, sample = cpu_oracle_sample(c, st, W, csr, rec_steps=args.ref_rec_steps, points=args.ref_points)
        if i >= args.warmup:
            times.append(t)
    t_step = float(np.mean(times))
    value = units / t_step
    line = {
        "impl": "reference", "metric": "ssm_dos_effective_matrix_applies_per_s", "value": value,
        "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "precision": "float64 CPU oracle",
        "config": bench_config(nnz, ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- accuracy

def oracle_reference(c, st, W, csr, t, info):
    """The oracle's DOS lines on the whole workload (doubling moments, flags at 1e-8)."""
    from oracle import ssm_oracle as O

    A = O.csr_matrix(csr.n, csr.rowptr, csr.colind, csr.val)
    t0 = time.perf_counter()
    r = O.ress_dgc(A, W, c["n_v"], t, c["M"], c["sigma"], interval=(info["a"], info["b"]), flag_eps=1e-8,
                   moments="doubling")
    return r, time.perf_counter() - t0


def l1_errors(ss, kpm, ref):
    """Relative L1 errors (Eq. error) of both DOS lines against the oracle; RESS-DGC on the
    points the oracle does not flag as within 1e-8 of an Alg. 4 threshold."""
    from oracle import ssm_oracle as O

    ok = ~ref["flagged"]
    return {"ss_l1": O.relative_l1_error(ss[ok], ref["dos_ss"][ok]),
            "kpm_l1": O.relative_l1_error(kpm, ref["dos_kpm"]), "points": int(ok.size),
            "flagged": int((~ok).sum())}


def time_precision(S, st, c, Wd, td, precision, units, warmup, steps, n_v=None, n_vh=None):
    """ms/step of one precision's plan (same step as the timed region), and its DOS lines;
    n_v / n_vh split the same probe columns between W and the hybrid block W~."""
    import torch

    n_v = c["n_v"] if n_v is None else n_v
    n_vh = c["n_vh"] if n_vh is None else n_vh
    plan = S.ssm_plan_create(stencil=st, n_v=n_v, n_vh=n_vh, degree=c["M"], precision=precision)

    def step():
        S.ssm_moments(plan, Wd)
        return S.ssm_dos(plan, td, c["sigma"], want_rank=False)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ss, kpm, _ = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"ms_per_step": ms, "value": units / (ms * 1e-3), "steps": steps, "warmup": warmup}
    plan.close()
    return out, ss.cpu().numpy(), kpm.cpu().numpy()


# ----------------------------------------------------------------------------- GPU arm

def run_gpu(args, c, st, W, csr):
    import torch

    import paper_1504_07690_gb300 as S

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.backend == "nccl" else "gloo")
    dev = torch.device("cuda", local)
    n_tot = c["n_v"] + c["n_vh"]
    M, n_t, sigma = c["M"], c["n_t"], c["sigma"]
    plan = S.ssm_plan_create(stencil=st, n_v=c["n_v"], n_vh=c["n_vh"], degree=M, precision=args.precision)
    info = S.ssm_plan_info(plan)
    t = np.linspace(info["lo"], info["hi"], n_t)
    Wd = torch.from_numpy(W).to(dev)
    td = torch.from_numpy(t).to(dev)
    nnz = info["nnz"]
    units = float(nnz) * n_tot * M

    def step():
        S.ssm_moments(plan, Wd)
        return S.ssm_dos(plan, td, sigma, want_rank=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    S.ssm_stats_reset(plan)
    S.ssm_timing_enable(plan, True)
    clocks = Clocks(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("ssm_timed")  # ncu --nvtx --nvtx-include ssm_timed/ profiles this region
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ck = clocks.stop()
    ms = over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    S.ssm_timing_enable(plan, False)
    stats = S.ssm_stats_get(plan)
    value = whole_job_value(units, ws, ms * 1e-3)

    # rooflines of the main kernels; "roofline" is the dominant one of the timed region
    hbm, bf16, bf16s, peak_kind = _peaks()
    phases = {k: stats[k] / args.steps for k in ("ms_coeffs", "ms_recurrence", "ms_gram", "ms_reduce",
                                                  "ms_assemble", "ms_solve", "ms_kpm")}
    args.fp64_gemm_tflops = fp64_gemm_tflops() if rank == 0 else None
    # kept ranks of the sweep points (untimed) decide each point's solver route
    _, _, rk = S.ssm_dos(plan, td, sigma, want_kpm=False)
    ranks = [(int(a), int(b)) for a, b in rk.cpu().numpy()]
    roofs = kernel_rooflines(st, c, stats, args, hbm, bf16, peak_kind, ck, ranks)
    dominant = max(roofs, key=lambda r: r["ms_per_step"])
    roofline = dict(dominant)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Wh = torch.from_numpy(W).pin_memory()
        th = torch.from_numpy(t).pin_memory()
        outs = torch.empty((2, n_t), dtype=torch.float64).pin_memory()

        def step_host():
            S.ssm_moments(plan, Wh)
            ss, kp, _ = S.ssm_dos(plan, th, sigma, want_rank=False)
            return ss, kp

        step_host()
        torch.cuda.synchronize()
        # the same per-phase CUDA events as in the device-timed region, so that the two
        # numbers differ by the copies and the host clock only
        S.ssm_timing_enable(plan, True)
        if dist is not None:
            dist.barrier()
        h0 = time.perf_counter()
        for _ in range(args.steps):
            step_host()
        torch.cuda.synchronize()
        hs = (time.perf_counter() - h0) / args.steps
        S.ssm_timing_enable(plan, False)
        hs = over_ranks(hs, dist, dev)
        e2e = {"value": whole_job_value(units, ws, hs), "unit": UNIT,
               "h2d_bytes_per_step": int(W.nbytes + t.nbytes), "d2h_bytes_per_step": int(2 * t.nbytes)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t_cpu, sample = cpu_oracle_sample(c, st, W, csr, rec_steps=args.ref_rec_steps, points=args.ref_points)
        cpu = {"value": units / t_cpu, "unit": "matrix-applies/s", "cores": _blas_threads(), "kind": "oracle",
               "sample": sample}

    # accuracy of every precision against the oracle on this workload, next to its speed:
    # the metric's "vs the float64 GPU path at L1 error"
    precisions = None
    if rank == 0 and ws == 1 and not args.no_accuracy:
        ref, t_oracle = oracle_reference(c, st, W, csr, t, info)
        ss_m, kp_m, _ = S.ssm_dos(plan, td, sigma, want_rank=False)
        precisions = {"oracle_s": t_oracle, "mixed": dict({"ms_per_step": ms, "value": value},
                                                       **l1_errors(ss_m.cpu().numpy(), kp_m.cpu().numpy(), ref))}
        tc, ss_t, kp_t = time_precision(S, st, c, Wd, td, "fp64_tc", units, args.warmup, args.steps)
        precisions["fp64_tc"] = dict(tc, **l1_errors(ss_t, kp_t, ref))
        if not args.no_fp64:
            f64, ss_f, kp_f = time_precision(S, st, c, Wd, td, "fp64", units, 1, 1)
            precisions["fp64"] = dict(f64, **l1_errors(ss_f, kp_f, ref))
        ok = [k for k in ("mixed", "fp64_tc", "fp64") if k in precisions and precisions[k]["ss_l1"] <= 1e-4]
        precisions["fastest_within_1e-4_ss"] = min(ok, key=lambda k: precisions[k]["ms_per_step"]) if ok else None
        # the same 200 probe columns split N_v = N~_v = 100 (Alg. 7's hybrid), against the
        # oracle's Alg. 7 loop on its own moments with the same split
        from oracle import ssm_oracle as O
        half = c["n_v"] // 2
        ref_h = O.ress_from_moments(ref["X"], ref, half, O.g_max(sigma, st.n), flag_eps=1e-8)
        ref_h["dos_kpm"] = ref["dos_kpm"]
        ok_b = ~(ref["flagged"] | ref_h["flagged"])
        precisions["oracle_hybrid_vs_single_l1"] = O.relative_l1_error(ref_h["dos_ss"][ok_b], ref["dos_ss"][ok_b])
        # the oracle's estimates for three splits of the same probes: DOS mass over t and the
        # distance to the (unbiased) KPM line
        dt = float(t[1] - t[0])
        study = {}
        for nv_s in (c["n_v"], (3 * c["n_v"]) // 4, half):
            d_s = ref["dos_ss"] if nv_s == c["n_v"] else (
                ref_h["dos_ss"] if nv_s == half else
                O.ress_from_moments(ref["X"], ref, nv_s, O.g_max(sigma, st.n))["dos_ss"])
            study[f"{nv_s}+{c['n_v'] - nv_s}"] = {"integral": float(np.sum(d_s) * dt),
                                                 "l1_vs_kpm": O.relative_l1_error(d_s, ref["dos_kpm"])}
        study["kpm"] = {"integral": float(np.sum(ref["dos_kpm"]) * dt)}
        precisions["oracle_split_study"] = study
        for prec in ("mixed", "fp64_tc"):
            hy, ss_h, kp_h = time_precision(S, st, c, Wd, td, prec, units, 1, 1, n_v=half, n_vh=c["n_v"] - half)
            precisions[f"{prec}_hybrid_{half}_{c['n_v'] - half}"] = dict(hy, **l1_errors(ss_h, kp_h, ref_h))

    batched = adjoint = lap3d = None
    if rank == 0 and not args.no_lap3d:
        lap3d = bench_lap3d(S, hbm)
    if rank == 0 and not args.no_batched:
        batched = bench_batched(S, hbm)
    if rank == 0 and not args.no_adjoint:
        adjoint = bench_adjoint(S, hbm)
    ssdgc = None
    if rank == 0 and not args.no_ssdgc:
        fp64_peak = max(args.fp64_gemm_tflops or 0.0, 152 * FP64_FMA_PER_SM_CLK * 2 * ((ck or {}).get("sm_mhz") or 2070.0)
                        * 1e6 / 1e12)
        ssdgc = bench_ssdgc(S, fp64_peak)

    if rank == 0:
        line = {
            "metric": "ssm_dos_effective_matrix_applies_per_s", "value": value,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32", "fp64": "f64", "fp64_tc": "f32x2"}[args.precision], "data": "synthetic",
            "precision": args.precision,
            "config": bench_config(nnz, ws),
            "roofline": roofline, "rooflines": roofs, "phases_ms_per_step": phases,
            "gpu_launches": int(stats["launches"]),
            "e2e": e2e, "cpu_baseline": cpu, "clocks": ck,
            "precisions": precisions,
            "lap3d": lap3d, "batched": batched, "adjoint": adjoint, "ssdgc": ssdgc,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


def bench_batched(S, hbm, warmup: int = 1, steps: int = 2):
    """Row a9: the 128-graph batched workload, recurrence as one captured CUDA graph."""
    import torch
    c = dict(wl.CONFIGS["er_batch_128"])
    graphs = wl.make_operator("er_batch_128")
    N = sum(g.n for g in graphs)
    nnz = sum(g.nnz for g in graphs)
    # a normalised Laplacian's spectrum lies in [0, 2]: that interval, padded by 1e-3 of its
    # width on each side, for every graph (so all graphs share one coefficient table)
    plan = S.ssm_plan_create_batched(graphs, n_v=c["n_v"], degree=c["M"], precision="mixed", lo=-2e-3,
                                     hi=2.0 + 2e-3)
    W = torch.from_numpy(wl.random_block(N, c["n_v"], c["probe_seed"], c["probe"])).cuda()
    t = torch.from_numpy(np.concatenate([np.linspace(0.0, 2.0, c["n_t"]) for _ in graphs])).cuda()

    def step():
        S.ssm_moments(plan, W)
        return S.ssm_dos(plan, t, c["sigma"], want_rank=False)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    S.ssm_stats_reset(plan)
    S.ssm_timing_enable(plan, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = S.ssm_stats_get(plan)
    S.ssm_timing_enable(plan, False)
    M, nv = c["M"], c["n_v"]
    rec_ms = st["ms_recurrence"] / steps
    # per recurrence step: read V_k, V_{k-1}, write V_{k+1} (float32), CSR values and columns
    step_bytes = 3.0 * N * nv * 4 + nnz * 8.0 + 8.0 * N
    achieved = step_bytes * (M // 2) / (rec_ms * 1e-3) / 1e9
    out = {"workload": "er_batch_128: 128 weighted ER normalized Laplacians, N_b ~ U{2000..60000} "
                       "(sum N = %d, nnz = %d), N_v=64 gaussian, M=500, 200 points each on [0, 2], interval [0, 2] "
                       "padded by 2e-3, sigma=0.05, mixed" % (N, nnz),
           "metric": "batched matrix-applies/s (sum_b nnz_b*N_v*M/s)", "value": nnz * nv * M / (ms * 1e-3),
           "ms_per_step": ms, "phases_ms_per_step": {k: v / steps for k, v in st.items() if k.startswith("ms_")},
           "csr_threads_autotuned": S.ssm_batch_tuning(plan)["csr_threads"],
           "gram_slabs_autotuned": S.ssm_batch_tuning(plan)["gram_slabs"], "graph_launches_per_step": 1,
           "roofline": {"kernel": "recurrence graph (CSR step + tensor-core Gram + reduction), per step",
                        "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": None, "bytes_per_step": step_bytes}}
    plan.close()
    return out


def bench_lap3d(S, hbm, runs=(("mixed", 256, 0), ("fp64_tc", 256, 0), ("mixed", 128, 128), ("fp64_tc", 128, 128)),
                n_trace: int = 1024):
    """The 3D log-normal workload (64^3 periodic 7-point -Laplacian + LogNormal(0, 0.5) potential,
    N = 262144, N_v = 256 Gaussian probes, M = 2000, 800 sweep points, sigma = 0.06) and its
    Tr log(A + I) by Alg. 8 on an n_trace-point grid, per precision: one warm-up and one timed
    step (moments + DOS), the trace timed on its own, both trace estimates against the exact
    log det(A + I) of tests/golden/lap3d_lognormal_64_logdet.json when that file exists.
    Each precision runs with the 256 probe columns all in W (N~_v = 0) and split evenly
    between W and the hybrid block W~ (Alg. 6 / Alg. 7's N_v = N~_v split): under each
    Gaussian of this workload lie thousands of eigenvalues, far more than 256, where the
    low-rank estimate alone cannot hold them and the hybrid term carries the rest."""
    import torch
    name = "lap3d_lognormal_64"
    c = dict(wl.CONFIGS[name])
    st = wl.make_operator(name)
    W = torch.from_numpy(wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])).cuda()
    exact = None
    gpath = os.path.join(ROOT, "tests", "golden", "lap3d_lognormal_64_logdet.json")
    if os.path.exists(gpath):
        exact = json.load(open(gpath))["logdet"]
    out = {"workload": "lap3d_lognormal_64: 3D 7-point periodic 64^3 (N=262144) + LogNormal(0,0.5), N_v=256 "
                       "gaussian, M=2000, 800 points, sigma=0.06; Tr log(A+I) on a %d-point grid" % n_trace,
           "exact_logdet": exact}
    for prec, nv, nvh in runs:
        plan = S.ssm_plan_create(stencil=st, n_v=nv, n_vh=nvh, degree=c["M"], precision=prec)
        info = S.ssm_plan_info(plan)
        td = torch.from_numpy(np.linspace(info["lo"], info["hi"], c["n_t"])).cuda()
        units = float(info["nnz"]) * (nv + nvh) * c["M"]

        def step():
            S.ssm_moments(plan, W)
            return S.ssm_dos(plan, td, c["sigma"], want_rank=False)

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t0 = time.perf_counter()
        tr_ss, tr_kpm = S.ssm_trace_f(plan, lambda v: math.log(v + 1.0), n_trace, c["sigma"], 0.016, 0.93)
        t_tr = time.perf_counter() - t0
        r = {"ms_per_step": ms, "value": units / (ms * 1e-3), "trace_ms": t_tr * 1e3, "tr_log_ss": tr_ss,
             "tr_log_kpm": tr_kpm}
        if exact is not None:
            r["tr_log_ss_rel_err"] = (tr_ss - exact) / exact
            r["tr_log_kpm_rel_err"] = (tr_kpm - exact) / exact
        out[f"{prec}_nv{nv}_nvh{nvh}"] = r
        plan.close()
    return out


def bench_ssdgc(S, fp64_peak, warmup: int = 1, steps: int = 2, n_t: int = 16):
    """SS-DGC with explicit filtered blocks (Alg. 5, ssm_dos_explicit) on the benchmark operator
    (Anderson 256^2, N_v = 200 Rademacher probes, M = 1000) at n_t sweep points inside the
    spectrum: CUDA events over `steps` calls after `warmup`.  Alg. 5 adds every recurrence
    block into all n_t blocks Z(t_i): 2 N N_v n_t (M+1) float64 flops in zacc_kernel, its
    roofline against the float64 peak.  Beside it, RESS-DGC at degree 2M on the
    float64-accurate tensor-core plan, which forms the same pencil from moments (K_W of
    degree M, K_Z its square), and the relative L1 difference of the two estimates."""
    import torch
    c = dict(wl.CONFIGS["anderson2d_256"])
    st = wl.make_operator("anderson2d_256")
    nv, M = c["n_v"], c["M"]
    W = torch.from_numpy(wl.random_block(st.n, nv, c["probe_seed"], c["probe"])).cuda()
    plan = S.ssm_plan_create(stencil=st, n_v=nv, degree=M, precision="fp64")
    info = S.ssm_plan_info(plan)
    t = torch.from_numpy(wl.explicit_points(info["lo"], info["hi"], n_t)).cuda()
    for _ in range(warmup):
        S.ssm_dos_explicit(plan, W, t, c["sigma"], want_rank=False)
    torch.cuda.synchronize()
    S.ssm_stats_reset(plan)
    S.ssm_timing_enable(plan, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        dos, _ = S.ssm_dos_explicit(plan, W, t, c["sigma"], want_rank=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    S.ssm_timing_enable(plan, False)
    stt = S.ssm_stats_get(plan)
    plan.close()
    phases = {k: stt[k] / steps for k in ("ms_coeffs", "ms_recurrence", "ms_gram", "ms_assemble", "ms_solve")}
    z_flops = 2.0 * st.n * nv * n_t * (M + 1)
    z_ms = phases["ms_assemble"]
    out = {"workload": "anderson2d_256 (N=65536, N_v=200 rademacher, M=1000, sigma=0.02) at %d points "
                       "inside the spectrum; SS-DGC (Alg. 5), float64" % n_t,
           "metric": "matrix-applies/s (nnz*N_v*M/s)", "ms_per_call": ms,
           "value": float(info["nnz"]) * nv * M / (ms * 1e-3), "phases_ms_per_call": phases,
           "roofline": {"kernel": "zacc_kernel", "bound": "alu", "achieved": z_flops / (z_ms * 1e-3) / 1e12,
                        "peak": fp64_peak, "unit": "TFLOP/s", "frac": z_flops / (z_ms * 1e-3) / 1e12 / fp64_peak,
                        "work_per_call": z_flops}}
    # the same pencil from moments: RESS-DGC at degree 2M on the float64 tensor-core plan
    p2 = S.ssm_plan_create(stencil=st, n_v=nv, degree=2 * M, precision="fp64_tc")
    S.ssm_moments(p2, W)
    ss2, _, _ = S.ssm_dos(p2, t, c["sigma"], want_kpm=False, want_rank=False)
    torch.cuda.synchronize()
    e0.record()
    S.ssm_moments(p2, W)
    ss2, _, _ = S.ssm_dos(p2, t, c["sigma"], want_kpm=False, want_rank=False)
    e1.record()
    torch.cuda.synchronize()
    p2.close()
    a, b = dos.cpu().numpy(), ss2.cpu().numpy()
    out["ress_2M_fp64_tc_ms"] = e0.elapsed_time(e1)
    out["l1_vs_ress_2M"] = float(np.abs(a - b).sum() / np.abs(b).sum())
    return out


def bench_adjoint(S, hbm, warmup: int = 1, steps: int = 2):
    """Row a10: KPM-DOS + Tr exp(-A) loss on the 100^3 potential workload, gradient by the adjoint."""
    import torch
    c = dict(wl.CONFIGS["lap3d_normal_100"])
    st = wl.make_operator("lap3d_normal_100")
    plan = S.ssm_plan_create(stencil=st, n_v=c["n_v"], degree=c["M"], precision="mixed", options=2)
    info = S.ssm_plan_info(plan)
    W = torch.from_numpy(wl.random_block(st.n, c["n_v"], c["probe_seed"], c["probe"])).cuda()
    t = torch.linspace(info["lo"], info["hi"], c["n_t"], dtype=torch.float64, device="cuda")
    dt = float(t[1] - t[0])
    xw, ww = S.ssm_trace_weights(plan, lambda x: math.exp(-x), 512, 0.05, 0.016, 0.93, device="cuda")
    tt = torch.cat([t, xw])
    # target: the KPM DOS of the same stencil with another potential (seed 3005)
    v_t = np.random.default_rng(c["target_seed"]).normal(0.0, 0.3, st.n) + (st.diag - np.mean(st.diag))
    v_t = np.clip(v_t, np.min(st.diag), np.max(st.diag))
    with torch.no_grad():
        target = S.KPMDensity.apply(torch.from_numpy(v_t).cuda(), plan, W, t, c["sigma"]).clone()
    v = torch.from_numpy(st.diag.copy()).cuda().requires_grad_(True)

    def step():
        v.grad = None
        phi = S.KPMDensity.apply(v, plan, W, tt, c["sigma"])
        loss = ((phi[: c["n_t"]] - target) ** 2).sum() * dt + (ww * phi[c["n_t"]:]).sum()
        loss.backward()
        return loss

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    S.ssm_stats_reset(plan)
    S.ssm_timing_enable(plan, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stt = S.ssm_stats_get(plan)
    S.ssm_timing_enable(plan, False)
    N, nv, M = st.n, c["n_v"], c["M"]
    S_ = M // 2
    adj_ms = stt["ms_adjoint"] / steps
    # per backward step: U_{k+1} (+ neighbours from L2), U_{k+2}, V_{k-1}, V_k, V_{k+1} read, U_k written,
    # one recomputed V (3 blocks), per-row float64 accumulators (4 read + 4 written)
    step_bytes = 9.0 * N * nv * 4 + 64.0 * N
    achieved = step_bytes * S_ / (adj_ms * 1e-3) / 1e9
    gnorm = float(v.grad.norm()) if v.grad is not None else None
    out = {"workload": "lap3d_normal_100: 3D 7-point periodic 100^3 (N=1e6) + N(0,0.3^2) potential, N_v=128, "
                       "M=800, loss = KPM DOS L2 to a target on 400 points + Tr exp(-A) (Alg. 8 weights, 512 points)",
           "metric": "forward+backward matrix-applies/s (nnz*N_v*M/s, forward counted once)",
           "value": info["nnz"] * nv * M / (ms * 1e-3), "ms_per_step": ms,
           "phases_ms_per_step": {k: v_ / steps for k, v_ in stt.items() if k.startswith("ms_")},
           "grad_norm": gnorm,
           "roofline": {"kernel": "adjoint steps (adj_stencil_kernel + recomputed stencil steps)", "bound": "hbm",
                        "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                        "bytes_per_step": step_bytes}}
    plan.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp64_tc"])
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the oracle run and the per-precision accuracy and speed table")
    ap.add_argument("--no-fp64", action="store_true", help="skip the CUDA-core float64 plan in that table")
    ap.add_argument("--backend", default="nccl", choices=["nccl", "gloo"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-plan row (128 graphs)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint row (100^3 potential)")
    ap.add_argument("--no-lap3d", action="store_true", help="skip the 64^3 log-normal row (Tr log(A+I))")
    ap.add_argument("--no-ssdgc", action="store_true", help="skip the explicit-block SS-DGC row (Alg. 5)")
    ap.add_argument("--ref-rec-steps", type=int, default=100)
    ap.add_argument("--ref-points", type=int, default=20)
    args = ap.parse_args()
    c, st, W, csr = _workload()
    if args.impl == "reference":
        run_reference(args, c, st, W, csr)
    else:
        run_gpu(args, c, st, W, csr)


if __name__ == "__main__":
    main()
