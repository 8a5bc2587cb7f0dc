"""Write oracle summaries of the full-size workloads for the GPU parity tests.

Calls only the FP64 CPU oracle (oracle/) on the seeded inputs of `workloads`.
Output: tests/golden/<name>_oracle.json with the PCG iteration count, the
Lanczos condition estimate, the coarse dimension, per-subdomain mode counts
and eigenvalues, the displacement at a fixed sample of dofs (every
stride-th dof), its 2-norm, and the 2-norm of every consecutive chunk of
CHUNK dofs (so a comparison touches every dof, not only the samples).
Names starting with "d-" are the Darcy workloads (workloads.darcy).
Usage: python tests/golden/make_golden.py c2 [nsamples]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import solver  # noqa: E402
from workloads.darcy import darcy_config  # noqa: E402


CHUNK = 1024


def main(name, nsamples=600):
    p = darcy_config(name) if name.startswith("d-") else workloads.config(name)
    t = time.time()
    r = solver.solve(p, precond="geneo", tol=1e-8)
    u = r["u"]
    stride = max(1, u.size // nsamples)
    idx = np.arange(0, u.size, stride)
    out = dict(config=name, tol=1e-8, iterations=int(r["iterations"]),
               kappa=float(r["kappa"]), n_coarse=int(r["n_coarse"]),
               modes=[int(m) for m in r["modes"]],
               lambdas=[[float(v) for v in lam[:21]] for lam in r["lambdas"]],
               u_norm=float(np.linalg.norm(u)), u_min_z=float(u[2::3].min()),
               sample_stride=int(stride), u_samples=[float(v) for v in u[idx]],
               chunk=CHUNK,
               u_chunk_norms=[float(np.linalg.norm(u[i:i + CHUNK]))
                              for i in range(0, u.size, CHUNK)],
               rel_res_true=float(r["true_rel_res"]),
               oracle_seconds=dict(assemble=r["t_assemble"], setup=r["t_setup"],
                                   solve=r["t_solve"], total=time.time() - t))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["iterations"], out["n_coarse"], out["oracle_seconds"])


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "c2",
         int(sys.argv[2]) if len(sys.argv) > 2 else 600)
