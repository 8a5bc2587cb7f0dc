"""Batched solves of uneven instances in one launch per step (the
many-instance form of the solve; Sec. 3.1 per instance).

A batch of set-up contexts of different sizes and kinds (laminated blocks of
2 to 8 subdomains with fixed and threshold-rule mode counts, a clamped
plate-like block, a scalar Darcy block) is solved together: one launch per
Krylov step over all instances, the one-level local solves of every
(instance, subdomain) item in one persistent work-queue launch, the
iterations in a CUDA graph.  Each instance keeps its own scalars, so each
result must be the instance's own solution:
  - against the FP64 oracle: u within 1e-6 (FP64 at tol 1e-8, iterations +-2;
    mixed precision at tol 1e-10),
  - against the same instance solved alone through geneo_solve: iterations
    within 1 (FP64: the same operator, sums in another order) and u within
    1e-9 (FP64),
  - a second batched solve is bit-identical to the first,
  - every batched launch shape (look-ahead or one row per step, tiles from
    global memory or staged) gives the same FP64 result within 1e-12.
"""
import numpy as np
import pytest

import workloads
from oracle import solver
from workloads.darcy import darcy_config
from workloads.laminate import make_block

from gpu_common import rel, require_gpu

pytestmark = pytest.mark.gpu

_ORACLE = {}


def instances():
    thr = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)
    return [workloads.config("tiny"), workloads.config("small"), workloads.config("c1"),
            make_block(10, 6, 4, [0.0, 90.0, 90.0, 0.0], partition=(3, 2, 1, 1), modes=thr,
                       name="block-10x6x4"),
            make_block(14, 4, 3, [45.0, -45.0, -45.0], partition=(4, 1, 1, 1), modes=thr,
                       name="strip-14x4x3"),
            darcy_config("d-tiny")]


def oracle(k, p, tol):
    key = (k, tol)
    if key not in _ORACLE:
        _ORACLE[key] = solver.solve(p, precond="geneo", tol=tol, eig_method="dense")
    return _ORACLE[key]


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def _setup(pkg, ps, prec):
    out = []
    for p in ps:
        s = pkg.GeneoSolver()
        s.assemble(p)
        s.setup(p, prec)
        out.append(s)
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle_and_single_solves(pkg, prec):
    ps = instances()
    tol = 1e-8 if prec == 0 else 1e-10
    solvers = _setup(pkg, ps, prec)
    singles = [s.solve(tol=tol, max_it=3000) for s in solvers]
    batch = pkg.GeneoBatch(solvers)
    us, stats = batch.solve(tol=tol, max_it=3000)
    us2, stats2 = batch.solve(tol=tol, max_it=3000)
    batch.close()
    for s in solvers:
        s.close()
    for k, (p, u, st) in enumerate(zip(ps, us, stats)):
        ref = oracle(k, p, tol)
        assert rel(u, ref["u"]) <= 1e-6, (p.get("name"), rel(u, ref["u"]))
        assert st["rel_res_true"] <= 2 * tol * (50 if p.get("kind") == "darcy" else 1), p.get("name")
        u1, st1 = singles[k]
        if prec == 0:
            assert abs(st["iterations"] - ref["iterations"]) <= 2, p.get("name")
            assert abs(st["iterations"] - st1["iterations"]) <= 1, p.get("name")
            assert rel(u, u1) <= 1e-9, p.get("name")
            assert abs(st["kappa_est"] - st1["kappa_est"]) <= 0.05 * st1["kappa_est"]
        else:
            assert st["flexible"] == 1
            assert abs(st["iterations"] - st1["iterations"]) <= 2, p.get("name")
        assert np.array_equal(u, us2[k]) and st["iterations"] == stats2[k]["iterations"]


@pytest.mark.parametrize("rows,staged", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_batch_launch_shapes_agree(pkg, monkeypatch, rows, staged):
    ps = instances()[:5]
    monkeypatch.setenv("GENEO_SCHWARZ_ROWS", str(rows))
    monkeypatch.setenv("GENEO_SCHWARZ_STAGED", str(staged))
    solvers = _setup(pkg, ps, 0)
    batch = pkg.GeneoBatch(solvers)
    us, stats = batch.solve(tol=1e-8, max_it=3000)
    batch.close()
    for s in solvers:
        s.close()
    for k, (p, u, st) in enumerate(zip(ps, us, stats)):
        assert (st["schwarz_rows"], st["schwarz_staged"]) == (rows, staged)
        ref = oracle(k, p, 1e-8)
        assert rel(u, ref["u"]) <= 1e-6, p.get("name")
        assert abs(st["iterations"] - ref["iterations"]) <= 2


def test_batch_refuses_mixed_precisions_and_unsolved_contexts(pkg):
    ps = instances()[:2]
    a, b = _setup(pkg, ps[:1], 0)[0], _setup(pkg, ps[1:2], 1)[0]
    with pytest.raises(pkg.GeneoError) as e:
        pkg.GeneoBatch([a, b])
    assert e.value.status == 1
    c = pkg.GeneoSolver()
    c.assemble(ps[1])                               # assembled, not set up
    with pytest.raises(pkg.GeneoError) as e:
        pkg.GeneoBatch([a, c])
    assert "set up" in str(e.value)
    with pytest.raises(pkg.GeneoError):
        pkg.GeneoBatch([a, a])
    d = pkg.GeneoSolver()
    q = dict(ps[1], coarse_solver="cg")
    d.assemble(q)
    d.setup(q, 0)
    with pytest.raises(pkg.GeneoError) as e:
        pkg.GeneoBatch([a, d])
    assert "direct coarse" in str(e.value)
    for s in (a, b, c, d):
        s.close()
