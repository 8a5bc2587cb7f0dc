"""GPU path vs the oracle on the paper's Example 1 plate (Sec. 5; Table 1).

The 100 x 20 mm plate of twelve plies [-45/45/0/90/45/-45/-45/45/90/0/45/-45]
and eleven resin interlayers on its base mesh (20 x 5 x 35 elements, element
aspect ratios up to 435), clamped at x = 0 under top pressure, split 2 x 2 in
plane with overlap 1 and the threshold rule capped at 20 modes: the wanted
GenEO eigenvalues crowd towards the overlap-localised modes, the case the
oracle's sparse eigensolver pin covers.  Same tolerances as the other parity
tests: eigenvalues 1e-7 relative, coarse span angles within the Ritz acceptance's bound, solution 1e-6
relative L2 with iterations within +-2 (FP64), and 1e-6 for the mixed
precision solve at a tolerance of 1e-10; the true residual within twice the
oracle's, which sits at the FP64 floor of b - A u for this system.  With the
zero-energy-mode coarse space the GPU reaches Table 1's printed coarse
dimensions for 4, 8, 16 and 32 subdomains (in-plane grids 2x2, 8x1, 8x2, 8x4),
and its 32-subdomain ZEM solve matches the oracle's.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import decomp, fem, geneo, solver as osolver
from workloads.laminate import make_block

from gpu_common import rel, require_gpu, span_tolerance

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "example1_plate.json")))


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def plate(grid=(2, 2)):
    m = GOLD["base_mesh"]
    nply = len(GOLD["stacking_deg"])
    nz = m["elements_per_ply"] * nply + m["elements_per_resin"] * GOLD["resin_layers"]
    p = make_block(m["nx"], m["ny"], nz, GOLD["stacking_deg"], resin_between=True,
                   partition=(grid[0], grid[1], 1, 1),
                   modes=dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01))
    lx, ly = GOLD["plate_mm"]
    p["x"] = np.linspace(0.0, lx, m["nx"] + 1)
    p["y"] = np.linspace(0.0, ly, m["ny"] + 1)
    return p


def test_plate_eigenvalues_and_span(pkg):
    p = plate()
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64)
    modes, lam, nh = s.coarse_info()
    A, _ = fem.assemble_system(p)
    subs = decomp.partition(p)
    Zo, info = geneo.coarse_space(p, subs, A)
    assert list(modes) == [d["m"] for d in info]
    for j, d in enumerate(info):
        kk = int(modes[j])
        ref = d["lam"][:kk]
        assert np.all(np.abs(lam[j, :kk] - ref) <= 1e-7 * np.maximum(np.abs(ref), 1e-2)), j
    Phi, AH = s.coarse()
    assert Phi.shape[1] == nh == Zo.shape[1]
    assert sla.subspace_angles(Phi, Zo.toarray()).max() <= span_tolerance(
        [d["m"] for d in info], [d["lam"] for d in info], p["modes"]["shift"])
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plate_solve_matches_oracle(pkg, prec):
    p = plate()
    s = pkg.GeneoSolver()
    s.assemble(p)
    tol = 1e-8 if prec == "fp64" else 1e-10
    s.setup(p, pkg.GENEO_FP64 if prec == "fp64" else pkg.GENEO_MIXED_FP32)
    u, st = s.solve(tol=tol, max_it=2000)
    ref = osolver.solve(p, precond="geneo", tol=tol)
    assert rel(u, ref["u"]) <= 1e-6
    # b - A u cannot be computed in FP64 on this system to better than about 6e-8
    # of ||b|| (the oracle's own true residual at 1e-8 and at 1e-10 alike), so
    # the true residual is held to the oracle's rather than to 2 tol
    assert st["rel_res_true"] <= max(2 * tol, 2 * ref["true_rel_res"]), \
        (st["rel_res_true"], ref["true_rel_res"])
    if prec == "fp64":
        assert abs(st["iterations"] - ref["iterations"]) <= 2, (st["iterations"], ref["iterations"])
    s.close()


GRIDS = {4: (2, 2), 8: (8, 1), 16: (8, 2), 32: (8, 4)}


@pytest.mark.parametrize("n", sorted(GRIDS))
def test_plate_table1_zem_dimension(pkg, n):
    p = plate(GRIDS[n])
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, pkg.GENEO_COARSE_ZEM)
    modes, _, nh = s.coarse_info()
    assert len(modes) == n
    assert nh == GOLD["table1_zem_dim"][str(n)]
    if n == 32:
        tol = GOLD["table1_residual_reduction"]
        u, st = s.solve(tol=tol, max_it=2000)
        ref = osolver.solve(p, precond="zem", tol=tol)
        assert st["n_coarse"] == ref["n_coarse"] == nh
        assert rel(u, ref["u"]) <= 1e-4
        assert abs(st["iterations"] - ref["iterations"]) <= 2, (st["iterations"], ref["iterations"])
    s.close()
