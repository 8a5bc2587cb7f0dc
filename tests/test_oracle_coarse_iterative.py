"""Pins for the oracle's inexact (iterative) coarse solve (Sec. 3.3.3).

When the coarse space is too large for a direct solve, the paper solves the
coarse problem by preconditioned CG; the coarse solve is then inexact and the
outer Krylov method must be flexible.  Here: block-Jacobi PCG on A_H over the
subdomain blocks.  Pins: at a tight inner tolerance the coarse solve meets its
residual bound before the iteration cap and the whole preconditioner equals
the direct one; with a single block covering A_H (an exact preconditioner) it
takes one step; a loose inner tolerance leaves a preconditioner that is not
linear in its argument, yet flexible CG still converges to the same solution
in not many more iterations than with the direct coarse solve.
"""
import numpy as np

import workloads
from oracle import decomp, fem, geneo, krylov, solver


def _two_level(name, **kw):
    p = workloads.config(name)
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Z, info = geneo.coarse_space(p, subs, A, "dense")
    sizes = [d["m"] for d in info]
    return p, A, b, subs, Z, sizes


def test_tight_inner_tolerance_equals_direct():
    p, A, b, subs, Z, sizes = _two_level("c1")
    Md = krylov.TwoLevelAS(A, subs, Z)
    Mi = krylov.TwoLevelAS(A, subs, Z, coarse="cg", coarse_tol=1e-14, block_sizes=sizes)
    r = np.random.default_rng(0).normal(size=A.shape[0])
    r[p["dirichlet_dofs"]] = 0.0
    zd, zi = Md(r), Mi(r)
    assert np.linalg.norm(zi - zd) <= 1e-10 * np.linalg.norm(zd)
    w = Z.T @ r
    yd = Md.coarse_solve(w)
    yi = Mi.coarse_solve(w)
    assert np.linalg.norm(Md.AH @ yi - w) <= 1e-13 * np.linalg.norm(w)
    assert np.linalg.norm(yi - yd) <= 1e-9 * np.linalg.norm(yd)
    assert Mi.inner_iterations[-1] < Mi.coarse_maxit


def test_single_block_is_one_step():
    p, A, b, subs, Z, sizes = _two_level("c1")
    Mi = krylov.TwoLevelAS(A, subs, Z, coarse="cg", coarse_tol=1e-12, block_sizes=[Z.shape[1]])
    w = np.random.default_rng(1).normal(size=Z.shape[1])
    y = Mi.coarse_solve(w)
    assert Mi.inner_iterations[-1] == 1
    assert np.linalg.norm(Mi.AH @ y - w) <= 1e-10 * np.linalg.norm(w)


def test_loose_tolerance_is_nonlinear_but_flexible_cg_converges():
    p, A, b, subs, Z, sizes = _two_level("small")
    Mi = krylov.TwoLevelAS(A, subs, Z, coarse="cg", coarse_tol=1e-1, block_sizes=sizes)
    rng = np.random.default_rng(2)
    r1, r2 = rng.normal(size=A.shape[0]), rng.normal(size=A.shape[0])
    for r in (r1, r2):
        r[p["dirichlet_dofs"]] = 0.0
    lin = Mi(r1 + r2) - Mi(r1) - Mi(r2)
    assert np.linalg.norm(lin) > 1e-8 * np.linalg.norm(Mi(r1 + r2))   # not a fixed linear map
    ref = solver.solve(p, precond="geneo", tol=1e-8)
    it = solver.solve(p, precond="geneo", tol=1e-8, coarse="cg", coarse_tol=1e-1)
    assert it["true_rel_res"] <= 2e-8
    assert np.linalg.norm(it["u"] - ref["u"]) <= 1e-6 * np.linalg.norm(ref["u"])
    assert ref["iterations"] <= it["iterations"] <= 1.5 * ref["iterations"] + 2


def test_block_jacobi_inverts_the_subdomain_blocks():
    # guards the block layout: the preconditioner is the inverse of A_H's
    # block diagonal over the subdomains' coarse columns
    p, A, b, subs, Z, sizes = _two_level("c1")
    Mi = krylov.TwoLevelAS(A, subs, Z, coarse="cg", block_sizes=sizes)
    D = np.zeros_like(Mi.AH)
    o = 0
    for m in sizes:
        D[o:o + m, o:o + m] = Mi.AH[o:o + m, o:o + m]
        o += m
    x = np.random.default_rng(3).normal(size=Z.shape[1])
    assert np.linalg.norm(Mi._block_jacobi(D @ x) - x) <= 1e-10 * np.linalg.norm(x)
    assert sum(1 for m in sizes if m) > 1
