"""Subdomains whose local vector does not fit in shared memory.

The local solves and the GenEO eigensolver's band solves normally keep a
subdomain's whole local vector in shared memory, which holds about 27,900
FP64 (57,000 FP32) unknowns.  Beyond that the same look-ahead sweep streams
the vector through a ring of max(w + 2, 3) tile rows in every CTA: the
forward sweep writes y to a scratch vector as it goes and the backward sweep
reads it back (Sec. 3.1, eqn:onelevelAS; the shift-invert solves of
Sec. 3.3.2).

1. The ring form does the arithmetic of the look-ahead launch with the same
   cluster size in the same order, so with both pinned (GENEO_SCHWARZ_STAGED=2
   against ROWS=0, STAGED=0, and GENEO_SCHWARZ_CLUSTER = 1, 2, 4 or 8) the
   preconditioner application and the whole solve are bit-identical, FP64
   and FP32, on narrow and wide bands.
2. The eigensolver's ring (GENEO_BAND_SOLVE_RING=1) gives bit-identical
   eigenvalues, coarse spaces and solutions.
3. The d-large Darcy block (36x64x24 cells, two subdomains of 30,525 interior
   and 31,450 Neumann unknowns) can only run in the ring forms; its FP64 and
   mixed solves are compared with the oracle's stored summary
   (tests/golden/d-large_oracle.json, written by make_golden.py from oracle/
   alone) at the parity tolerances of the other full-size tests: u 1e-6
   relative at the samples and by chunk norms, iterations within 2, the same
   mode counts and eigenvalues within 1e-7.
"""
import json
import os

import numpy as np
import pytest

import workloads
from workloads.darcy import darcy_config
from workloads.laminate import make_block

from gpu_common import check_against_golden, require_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FP64_WHOLE_VECTOR = (227 * 1024 // 8) - 34 * 32     # unknowns a one-CTA FP64 launch can hold


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def _problem(name):
    if name == "wide":
        return make_block(14, 14, 28, [0.0, 90.0, 90.0, 0.0], partition=(1, 1, 2, 1))
    return workloads.config(name)


def _run_as(pkg, monkeypatch, p, prec, pins, r):
    with monkeypatch.context() as m:
        for k, v in pins.items():
            m.setenv(k, v)
        s = pkg.GeneoSolver()
        s.assemble(p)
        s.setup(p, prec, pkg.GENEO_AS, pkg.GENEO_COARSE_NONE)
        z = s.apply_preconditioner(r)
        u, st = s.solve(tol=1e-8, max_it=3000)
        s.close()
    return z, u, st


@pytest.mark.parametrize("name", ["small", "c1", "wide"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_ring_local_solves_bit_identical_to_lookahead(pkg, monkeypatch, name, prec, cluster):
    p = _problem(name)
    n = 3 * (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)
    r = np.random.default_rng(9).normal(size=n)
    r[p["dirichlet_dofs"]] = 0.0
    C = str(cluster)
    la = {"GENEO_SCHWARZ_CLUSTER": C, "GENEO_SCHWARZ_ROWS": "0", "GENEO_SCHWARZ_STAGED": "0"}
    ring = {"GENEO_SCHWARZ_CLUSTER": C, "GENEO_SCHWARZ_STAGED": "2"}
    z0, u0, st0 = _run_as(pkg, monkeypatch, p, prec, la, r)
    z1, u1, st1 = _run_as(pkg, monkeypatch, p, prec, ring, r)
    assert (st0["schwarz_cluster"], st0["schwarz_rows"], st0["schwarz_staged"]) == (cluster, 0, 0)
    assert (st1["schwarz_cluster"], st1["schwarz_rows"], st1["schwarz_staged"]) == (cluster, 0, 2)
    assert np.array_equal(z0, z1)
    assert np.array_equal(u0, u1)
    assert st0["iterations"] == st1["iterations"]
    assert st1["rel_res_true"] <= 2e-8


@pytest.mark.parametrize("name", ["c1", "wide"])
def test_ring_eigensolver_bit_identical(pkg, monkeypatch, name):
    p = _problem(name)
    out = []
    for ring in ("0", "1"):
        with monkeypatch.context() as m:
            m.setenv("GENEO_BAND_SOLVE_RING", ring)
            m.setenv("GENEO_SCHWARZ_CLUSTER", "1")
            m.setenv("GENEO_SCHWARZ_ROWS", "1")
            m.setenv("GENEO_SCHWARZ_STAGED", "0")
            s = pkg.GeneoSolver()
            s.assemble(p)
            s.setup(p, pkg.GENEO_FP64)
            modes, lam, nh = s.coarse_info()
            u, st = s.solve(tol=1e-8, max_it=3000)
            out.append((modes, lam, nh, u, st["iterations"]))
            s.close()
    (m0, l0, n0, u0, i0), (m1, l1, n1, u1, i1) = out
    assert list(m0) == list(m1) and n0 == n1 > 0
    assert np.array_equal(l0, l1)
    assert np.array_equal(u0, u1) and i0 == i1


def test_large_subdomains_need_the_ring(pkg):
    p = darcy_config("d-large")
    keep = []
    plan = pkg.geneo_plan_subdomains(pkg.GeneoSolver.mesh_of(p, keep),
                                     pkg.GeneoSolver.partition_of(p), unknowns_per_node=1)
    assert plan[:, 12].min() > FP64_WHOLE_VECTOR      # interior unknowns (local solves)
    assert plan[:, 14].min() > FP64_WHOLE_VECTOR      # Neumann unknowns (eigensolver)


@pytest.mark.parametrize("prec,pins", [
    (0, {}),                                                          # the tuner's ring shape
    (0, {"GENEO_SCHWARZ_CLUSTER": "1"}),                              # one CTA per subdomain
    (1, {}),                                                          # FP32 vectors fit whole
    (1, {"GENEO_SCHWARZ_STAGED": "2", "GENEO_SCHWARZ_CLUSTER": "8"}),
])
def test_large_subdomains_against_oracle(pkg, monkeypatch, prec, pins):
    with open(os.path.join(GOLDEN, "d-large_oracle.json")) as f:
        gold = json.load(f)
    p = darcy_config("d-large")
    for k, v in pins.items():
        monkeypatch.setenv(k, v)
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, prec)
    coarse = s.coarse_info()
    u, st = s.solve(tol=1e-8, max_it=3000)
    if prec == 0 or pins:
        assert st["schwarz_staged"] == 2
    if "GENEO_SCHWARZ_CLUSTER" in pins:
        assert st["schwarz_cluster"] == int(pins["GENEO_SCHWARZ_CLUSTER"])
    assert st["rel_res_true"] <= 2e-8
    check_against_golden(u, st, gold, coarse=coarse)
    s.close()


def test_batch_refuses_subdomains_larger_than_shared_memory(pkg):
    """The batched persistent launch holds every item's whole local vector, so
    a batch with a d-large context is refused; the context itself stays usable."""
    p = darcy_config("d-large")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, pkg.GENEO_COARSE_NONE)
    with pytest.raises(pkg.GeneoError) as e:
        pkg.GeneoBatch([s])
    assert e.value.status == 1
    assert "no batched local-solve shape fits" in str(e.value)
    u, st = s.solve(tol=1e-8, max_it=3000)
    assert st["schwarz_staged"] == 2 and st["rel_res_true"] <= 2e-8
    s.close()
