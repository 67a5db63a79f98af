"""Write the exact Tr log(A + I) = log det(A + I) of the 3D log-normal workload
(64^3 periodic 7-point -Laplacian plus a LogNormal(0, 0.5) potential, operator
seed 1003) to lap3d_lognormal_64_logdet.json, with oracle.logdet_shifted (sparse
LU).  Run once on a CPU (about 15 minutes and several GB at 64^3); the benchmark
reads the file to state the error of its Tr log(A + I) estimates.

    python tests/golden/make_logdet_lap3d.py [nx]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import ssm_oracle as O  # noqa: E402


def main():
    nx = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    st = wl.make_operator("lap3d_lognormal_64", nx=nx)
    c = wl.stencil_to_csr(st)
    A = O.csr_matrix(c.n, c.rowptr, c.colind, c.val)
    t0 = time.time()
    ld = O.logdet_shifted(A, 1.0)
    out = {"workload": "lap3d_lognormal_64", "nx": nx, "n": c.n, "shift": 1.0, "logdet": ld,
           "method": "oracle.logdet_shifted (scipy splu, MMD on A + A^T)", "seconds": round(time.time() - t0, 1)}
    name = "lap3d_lognormal_64_logdet.json" if nx == 64 else f"lap3d_lognormal_{nx}_logdet.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
