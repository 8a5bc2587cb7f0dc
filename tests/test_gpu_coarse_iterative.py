"""Inexact (iterative) coarse solve on the GPU against the oracle's (Sec. 3.3.3).

For very large coarse spaces the paper solves A_H y = w by preconditioned CG
and makes the outer Krylov method flexible.  The GPU runs block-Jacobi PCG on
A_H (blocks = each subdomain's modes) in one cooperative launch; the oracle
runs the same algorithm with dense Cholesky solves of the blocks.  Because
the GPU's and the oracle's coarse bases differ only by a change of basis
inside each subdomain's span (eigenvectors of a cluster are not unique), and
block-Jacobi PCG iterates transform with such a change, the inexact coarse
correction Z y_k is the same for both:
  - at inner tolerance 1e-14 the application equals the direct one (1e-9 to
    the oracle's direct two-level operator),
  - with the inner step count fixed (tolerance 1e-14, at most 5 steps) it
    matches the oracle's inexact algorithm run on the GPU's own coarse basis
    and A_H (1e-9: the same iteration on the same data),
  - at tolerance 1e-2 (about 35 inner steps) it matches the oracle's inexact
    application on the oracle's basis within 1e-3: whether the inner
    residual crosses the tolerance at one step or the next depends on
    rounding, and one inner step moves z by up to about 1e-4 on these blocks,
  - flexible CG with the inexact coarse solve matches the oracle's solution
    (1e-6, iterations +-2) and reports the inner steps it took.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import decomp, fem, geneo, krylov, solver

from gpu_common import rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def _oracle(p, **kw):
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Z, info = geneo.coarse_space(p, subs, A, "dense")
    return A, krylov.TwoLevelAS(A, subs, Z, block_sizes=[d["m"] for d in info], **kw)


@pytest.mark.parametrize("name", ["small", "c1"])
@pytest.mark.parametrize("tol,maxit", [(1e-14, 500), (1e-14, 5), (1e-2, 500)])
def test_inexact_coarse_application(pkg, name, tol, maxit):
    p = dict(workloads.config(name), coarse_solver="cg", coarse_tol=tol, coarse_maxit=maxit)
    A, Md = _oracle(p)
    _, Mi = _oracle(p, coarse="cg", coarse_tol=tol, coarse_maxit=maxit)
    r = np.random.default_rng(3).normal(size=A.shape[0])
    r[p["dirichlet_dofs"]] = 0.0
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64)
    z = s.apply_preconditioner(r)
    assert np.array_equal(z, s.apply_preconditioner(r))
    modes, _, _ = s.coarse_info()
    Phi, _ = s.coarse()
    s.close()
    if maxit == 500 and tol < 1e-10:
        assert rel(z, Md(r)) <= 1e-9
        return
    zi = Mi(r)
    assert rel(zi, Md(r)) > 1e-6               # the inexact solve is not the direct one here
    if maxit == 5:
        Mg = krylov.TwoLevelAS(A, decomp.partition(p), sp.csc_matrix(Phi), coarse="cg",
                               coarse_tol=tol, coarse_maxit=maxit, block_sizes=list(modes))
        assert rel(z, Mg(r)) <= 1e-9
    else:
        assert rel(z, zi) <= 1e-3


@pytest.mark.parametrize("name", ["small", "c1"])
def test_flexible_cg_with_inexact_coarse_solve(pkg, name):
    p = dict(workloads.config(name), coarse_solver="cg", coarse_tol=1e-2)
    ref = solver.solve(p, precond="geneo", tol=1e-8, eig_method="dense", coarse="cg",
                       coarse_tol=1e-2)
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64)
    u, st = s.solve(tol=1e-8, max_it=2000)
    s.close()
    assert st["flexible"] == 1
    assert st["coarse_inner_iterations"] > 0
    assert rel(u, ref["u"]) <= 1e-6
    assert abs(st["iterations"] - ref["iterations"]) <= 2
    assert st["rel_res_true"] <= 2e-8
