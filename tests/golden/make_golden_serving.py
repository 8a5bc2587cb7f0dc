"""Write oracle summaries of the small requests of the seeded serving stream.

Calls only the FP64 CPU oracle (oracle/) on the requests of
workloads.serving.request_stream(n, seed, darcy_frac, darcy_grid) whose
unknown count is at most `max_dofs` (the oracle solves those in seconds to a
minute); output: tests/golden/serving_oracle.json with, per request index,
the PCG iteration count, the displacement (or pressure) at every stride-th
unknown and its 2-norm.  Usage:
  python tests/golden/make_golden_serving.py [n] [seed] [max_dofs]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solver  # noqa: E402
from workloads.serving import dofs_of, request_stream  # noqa: E402


def main(n=200, seed=6, max_dofs=60000, nsamples=400):
    out = dict(n=n, seed=seed, darcy_frac=0.3, darcy_grid="spe10", tol=1e-8, requests={})
    t0 = time.time()
    for i, (key, p, _) in enumerate(request_stream(n, seed=seed, darcy_frac=0.3,
                                                   darcy_grid="spe10")):
        if dofs_of(p) > max_dofs:
            continue
        r = solver.solve(p, precond="geneo", tol=1e-8)
        u = r["u"]
        stride = max(1, u.size // nsamples)
        out["requests"][str(i)] = dict(key=key, dofs=int(u.size), iterations=int(r["iterations"]),
                                       sample_stride=int(stride),
                                       u_samples=[float(v) for v in u[::stride]],
                                       u_norm=float(np.linalg.norm(u)))
        print(i, key, u.size, r["iterations"], f"{time.time() - t0:.0f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serving_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, len(out["requests"]))


if __name__ == "__main__":
    a = sys.argv[1:]
    main(int(a[0]) if a else 200, int(a[1]) if len(a) > 1 else 6,
         int(a[2]) if len(a) > 2 else 60000)
