"""Gather over nodes shared by more than eight subdomain interiors.

The gather of the local solutions (Sec. 3.1, eqn:onelevelAS) goes through a
per-node map of at most eight interior subdomains, built at set-up; nodes
with more are gathered by visiting the subdomain candidates directly.  An
8x8x4 block cut into 4x4x1 subdomains with overlap 2 has such nodes (up to
nine interiors per node); the one-level application, plain and with the
partition-of-unity weights, must match the oracle there as everywhere.
"""
import numpy as np
import pytest

from oracle import decomp, fem, krylov
from workloads.laminate import make_block

from gpu_common import rel, require_gpu


def dense_overlap_block():
    modes = dict(fixed_modes=0, threshold=0.0, max_modes=6, shift=-0.01)
    return make_block(8, 8, 4, [0.0, 90.0], partition=(4, 4, 1, 2), modes=modes,
                      name="dense-overlap")


def interior_multiplicity(p, subs):
    cnt = np.zeros((p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1), int)
    for s in subs:
        cnt[np.asarray(s.int_nodes)] += 1
    return cnt


def test_partition_has_nodes_in_more_than_eight_interiors():
    p = dense_overlap_block()
    cnt = interior_multiplicity(p, decomp.partition(p))
    assert cnt.max() == 9 and (cnt > 8).sum() == 20


@pytest.mark.gpu
@pytest.mark.parametrize("weight", ["none", "pou"])
def test_one_level_apply_with_dense_overlap(weight):
    pkg = require_gpu()
    p = dense_overlap_block()
    s = pkg.GeneoSolver()
    s.assemble(p)
    sch = pkg.GENEO_AS_POU if weight == "pou" else pkg.GENEO_AS
    s.setup(p, pkg.GENEO_FP64, sch, pkg.GENEO_COARSE_NONE)
    A, _ = fem.assemble_system(p)
    M = krylov.OneLevelAS(A, decomp.partition(p), weight=weight)
    r = np.random.default_rng(7).normal(size=s.ndof)
    r[p["dirichlet_dofs"]] = 0.0
    z = s.apply_preconditioner(r)
    assert np.array_equal(z, s.apply_preconditioner(r))
    assert rel(z, M(r)) <= 1e-9
    s.close()
