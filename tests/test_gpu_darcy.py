"""The scalar Darcy problem (eqn:Darcy, eq-fe-darcy) on the GPU vs the oracle.

Same tolerances as the elasticity parity tests: matrix entries 1e-12 of the
largest, load 1e-13, SpMV 1e-13, one FP64 one-level application 1e-9, GenEO
eigenvalues 1e-7 (floor 1e-2), solutions 1e-6 relative with iteration counts
within 2 (FP64 and mixed precision), on layered log-normal permeability with
a contrast of 1e6-1e7.
"""
import numpy as np
import pytest

from oracle import darcy, decomp, fem, geneo, krylov, solver as osolver
from workloads.darcy import darcy_config

from gpu_common import bsr_to_csr, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def _solver(pkg, p):
    s = pkg.GeneoSolver()
    s.assemble(p)
    return s


@pytest.mark.parametrize("name", ["d-tiny", "d-small"])
def test_darcy_assembly_and_spmv(pkg, name):
    p = darcy_config(name)
    s = _solver(pkg, p)
    assert s.ndof == s.nnode
    rp, col, val, b = s.system()
    A = bsr_to_csr(rp, col, val, s.nnode, nc=1)
    Ao, bo = darcy.assemble_system(p)
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()
    x = np.random.default_rng(0).normal(size=s.ndof)
    assert rel(s.spmv(x), Ao @ x) <= 1e-13
    s.close()


def test_darcy_one_level_apply(pkg):
    p = darcy_config("d-small")
    s = _solver(pkg, p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, pkg.GENEO_COARSE_NONE)
    A, _ = fem.assemble_system(p)
    M = krylov.OneLevelAS(A, decomp.partition(p))
    r = np.random.default_rng(1).normal(size=s.ndof)
    r[p["dirichlet_dofs"]] = 0.0
    assert rel(s.apply_preconditioner(r), M(r)) <= 1e-9
    s.close()


def test_darcy_geneo_eigenvalues(pkg):
    p = darcy_config("d-small")
    s = _solver(pkg, p)
    s.setup(p)
    modes, lam, nh = s.coarse_info()
    A, _ = fem.assemble_system(p)
    Z, info = geneo.coarse_space(p, decomp.partition(p), A)
    assert list(modes) == [d["m"] for d in info]
    for j, d in enumerate(info):
        for i in range(d["m"]):
            ref = d["lam"][i]
            assert abs(lam[j, i] - ref) <= 1e-7 * max(abs(ref), 1e-2)
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,coarse", [("d-small", "geneo"), ("d-tiny", "geneo")])
def test_darcy_solve_matches_oracle(pkg, prec, name, coarse):
    p = darcy_config(name)
    ref = osolver.solve(p, precond=coarse, tol=1e-8)
    s = _solver(pkg, p)
    s.setup(p, prec)
    u, st = s.solve(tol=1e-8, max_it=3000)
    assert rel(u, ref["u"]) <= 1e-6
    assert abs(st["iterations"] - ref["iterations"]) <= 2
    assert st["n_coarse"] == ref["n_coarse"]
    s.close()


def test_darcy_zem_on_a_floating_partition(pkg):
    p = darcy_config("d-small", partition=(2, 1, 3, 1))     # the upper layers float
    ref = osolver.solve(p, precond="zem", tol=1e-8)
    s = _solver(pkg, p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, pkg.GENEO_COARSE_ZEM)
    u, st = s.solve(tol=1e-8, max_it=3000)
    assert st["n_coarse"] == ref["n_coarse"] > 0
    assert rel(u, ref["u"]) <= 1e-6
    assert abs(st["iterations"] - ref["iterations"]) <= 2
    s.close()


def test_darcy_new_source_on_resident_system(pkg):
    p = darcy_config("d-small")
    s = _solver(pkg, p)
    s.setup(p)
    nodal = np.random.default_rng(3).normal(size=s.ndof)
    s.set_load(nodal, 2.5)
    _, _, _, b = s.system()
    q = dict(p)
    q["source"], q["nodal_load"] = 2.5, nodal
    _, bo = darcy.assemble_system(q)
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()
    u, st = s.solve(tol=1e-8)
    ref = osolver.solve(q, precond="geneo", tol=1e-8)
    assert rel(u, ref["u"]) <= 1e-6
    s.close()


def test_darcy_has_no_stresses(pkg):
    p = darcy_config("d-tiny")
    s = _solver(pkg, p)
    with pytest.raises(Exception):
        s.element_stress(np.zeros(s.ndof))
    s.close()
