"""New load cases on a resident system (geneo_set_load) against the oracle.

The right-hand side after geneo_set_load must be the oracle's load for the new
traction and nodal forces with the same (non-homogeneous) Dirichlet lifting,
and bit-identical to a fresh assembly with that load; a solve on the resident
preconditioner must reproduce a fresh assemble + set-up + solve bit for bit
and the direct solution of the oracle's system.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads
from oracle import fem

from gpu_common import rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def _problem(seed):
    p = workloads.config("small")
    rng = np.random.default_rng(seed)
    # clamped face with prescribed, non-zero displacements
    p["dirichlet_values"] = 1e-3 * rng.normal(size=p["dirichlet_dofs"].size)
    return p


def _with_load(p, nodal, pressure):
    q = dict(p)
    q["nodal_load"] = nodal
    q["top_pressure"] = pressure
    return q


def test_set_load_rhs_matches_oracle_and_fresh_assembly(pkg):
    p = _problem(11)
    s = pkg.GeneoSolver()
    s.assemble(p)
    nodal = np.random.default_rng(12).normal(size=s.ndof)
    s.set_load(nodal, 3.5)
    _, _, _, b = s.system()
    p2 = _with_load(p, nodal, 3.5)
    _, bo = fem.assemble_system(p2)
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()
    f = pkg.GeneoSolver()
    f.assemble(p2)
    _, _, _, bf = f.system()
    assert np.array_equal(b, bf)
    # pressure only, no nodal forces: back to the original problem's load
    s.set_load(None, p["top_pressure"])
    _, _, _, b1 = s.system()
    _, bo1 = fem.assemble_system(p)
    assert np.abs(b1 - bo1).max() <= 1e-13 * np.abs(bo1).max()
    s.close()
    f.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_resident_solve_with_new_load(pkg, prec):
    p = _problem(21)
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, prec)
    u1, st1 = s.solve(tol=1e-10, max_it=3000)
    nodal = 0.05 * np.random.default_rng(22).normal(size=s.ndof)
    s.set_load(nodal, 0.7)
    u2, st2 = s.solve(tol=1e-10, max_it=3000)
    p2 = _with_load(p, nodal, 0.7)
    f = pkg.GeneoSolver()
    f.assemble(p2)
    f.setup(p2, prec)
    uf, stf = f.solve(tol=1e-10, max_it=3000)
    assert st2["iterations"] == stf["iterations"]
    assert np.array_equal(u2, uf)
    A, bo = fem.assemble_system(p2)
    ud = spla.spsolve(A.tocsc(), bo)
    assert rel(u2, ud) <= 1e-7
    assert rel(u1, u2) > 1e-3          # the load did change
    s.close()
    f.close()


def test_set_load_before_assemble_is_an_error(pkg):
    s = pkg.GeneoSolver()
    with pytest.raises(Exception):
        s.set_load(None, 1.0)
    s.close()
