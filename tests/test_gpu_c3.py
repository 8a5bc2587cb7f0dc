"""Full-size 128x64x48 laminate with a fibre wrinkle (1,232,595 dofs, 8x4x4
subdomains), in the launch configuration bench.py times.

Against the oracle's stored summary of this workload
(tests/golden/c3_oracle.json, written by make_golden.py from oracle/ only; the
oracle takes about 25 minutes on 8 cores): the mixed-precision path (FP32
factors, FP64 flexible CG) and the all-FP64 path each match the oracle's
displacement within 1e-6 relative L2 at 4,002 stored samples and in the norm
of every chunk of 1,024 dofs, its iteration count within 2, and (FP64 and
mixed alike, the GenEO set-up being FP64 in both) its 2,560-dimensional coarse
space: per-subdomain mode counts and eigenvalues (1e-7 relative).

Independently of the stored summary, the residual is also checked through
quantities the oracle computes entry by entry: at 3,000 sampled dofs
the residual entry b_i - (A u)_i, with row i of A built from the oracle's own
element stiffness matrices of the (up to 8) elements around the node, must be
below 2 x 1e-8 x ||b||_2 (implied by ||b - A u||_2 <= 1e-8 ||b||_2), and the
GPU-reported true relative residual must be <= 2e-8.
"""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import fem, material

from gpu_common import check_against_golden, require_gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c3_oracle.json")

pytestmark = pytest.mark.gpu


def sampled_residual(p, u, dofs):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    nnx, nny = nx + 1, ny + 1
    x, y, z = p["x"], p["y"], p["z"]
    b = fem.top_pressure_load(p)
    dmask = np.zeros(u.size, bool)
    dmask[p["dirichlet_dofs"]] = True
    b[p["dirichlet_dofs"]] = p["dirichlet_values"]   # symmetric elimination, g = 0 here
    out = np.zeros(len(dofs))
    cache = {}
    for t, d in enumerate(dofs):
        n, r = divmod(int(d), 3)
        i, rem = n % nnx, n // nnx
        j, k = rem % nny, rem // nny
        if dmask[d]:
            out[t] = b[d] - u[d]
            continue
        acc = 0.0
        for ez in (k - 1, k):
            for ey in (j - 1, j):
                for ex in (i - 1, i):
                    if not (0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz):
                        continue
                    e = ex + nx * (ey + ny * ez)
                    key = (int(p["elem_mat"][e]), float(p["elem_theta"][e]),
                           float(p["elem_phi"][e]), x[ex + 1] - x[ex], y[ey + 1] - y[ey],
                           z[ez + 1] - z[ez])
                    if key not in cache:
                        Cv = material.element_stiffness_voigt(p["materials"][key[0]], key[1], key[2])
                        cache[key] = fem.element_stiffness(Cv, *key[3:])
                    Ke = cache[key]
                    a = (i - ex) + 2 * (j - ey) + 4 * (k - ez)
                    ed = fem.element_dofs(nx, ny, ex, ey, ez)
                    ue = np.where(dmask[ed], 0.0, u[ed])
                    acc += Ke[3 * a + r] @ ue
        out[t] = b[d] - acc
    return out, np.linalg.norm(b)


def test_c3_mixed_precision_residual_sampled_by_oracle():
    pkg = require_gpu()
    p = workloads.config("c3")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_MIXED_FP32)
    u, st = s.solve(tol=1e-8, max_it=3000)
    s.close()
    assert st["rel_res_true"] <= 2e-8
    assert st["flexible"] == 1
    assert st["n_coarse"] > 0
    rng = np.random.default_rng(11)
    dofs = np.sort(rng.choice(u.size, 3000, replace=False))
    res, bn = sampled_residual(p, u, dofs)
    assert np.abs(res).max() <= 2e-8 * bn


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_c3_matches_oracle(prec):
    pkg = require_gpu()
    gold = json.load(open(GOLD))
    p = workloads.config("c3")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_MIXED_FP32 if prec == "mixed" else pkg.GENEO_FP64)
    u, st = s.solve(tol=1e-8, max_it=3000)
    coarse = s.coarse_info()
    s.close()
    check_against_golden(u, st, gold, coarse)
    assert st["rel_res_true"] <= 2e-8
    assert st["flexible"] == (1 if prec == "mixed" else 0)
