"""Sarkis's partition of unity on the GPU against the oracle's (Sec. 3.2,
Sec. 3.3.1).

X_j(n) = d_j(n) / sum_k d_k(n), d the distance of node n to each interior
subdomain's artificial boundary in element layers.  It enters B_j (the GenEO
overlap matrix), the coarse basis R_j^T X_j p and the one-level weight
D_j = X_j.  With overlap 2 it differs from the multiplicity PoU (the weight
ramps across the overlap), so the checks run there: B_j and S_j entry by
entry (1e-12), the PoU-weighted one-level application (1e-9, also on a block
whose nodes sit in up to nine subdomain interiors, gathered through the
candidate lists), and GenEO-PCG (eigenvalues 1e-7, span angles within the Ritz
acceptance's bound, u 1e-6,
iterations +-2).  With overlap 1 the two PoUs are the same numbers, so the
preconditioner applications are bit-identical.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import workloads
from oracle import decomp, fem, geneo, krylov, solver
from workloads.laminate import make_block

from gpu_common import rel, require_gpu, span_tolerance

pytestmark = pytest.mark.gpu


def overlap2(name):
    if name == "dense-overlap":
        modes = dict(fixed_modes=0, threshold=0.0, max_modes=6, shift=-0.01)
        p = make_block(8, 8, 4, [0.0, 90.0], partition=(4, 4, 1, 2), modes=modes,
                       name="dense-overlap")
    else:
        p = workloads.config(name)
        p["partition"] = tuple(p["partition"][:3]) + (2,)
    p["pou"] = "sarkis"
    return p


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.mark.parametrize("name", ["small", "c1"])
def test_sarkis_local_matrices(pkg, name):
    p = overlap2(name)
    subs = decomp.partition(p)
    q = dict(p, pou="standard")
    std = decomp.partition(q)
    assert any(np.abs(a.X - b.X).max() > 0.1 for a, b in zip(subs, std))   # they differ here
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64)
    sigma = p["modes"]["shift"]
    for j, sd in enumerate(subs):
        An, Ao = geneo.local_matrices(p, sd)
        Xd = sp.diags(sd.X)
        B = (Xd @ Ao @ Xd).toarray()
        Sg, gdn = s.local_matrix(j, 1)
        pos = np.searchsorted(sd.neu_dofs, gdn)
        assert np.array_equal(sd.neu_dofs[pos], gdn)
        Sr = (An.toarray() - sigma * B)[np.ix_(pos, pos)]
        assert np.abs(Sg - Sr).max() <= 1e-12 * np.abs(Sr).max(), ("S_j", j)
        Bg, _ = s.local_matrix(j, 2)
        Br = B[np.ix_(pos, pos)]
        assert np.abs(Bg - Br).max() <= 1e-12 * np.abs(Br).max(), ("B_j", j)
    s.close()


@pytest.mark.parametrize("name", ["small", "dense-overlap"])
@pytest.mark.parametrize("prec", [0, 1])
def test_sarkis_weighted_one_level_apply(pkg, name, prec):
    p = overlap2(name)
    A, _ = fem.assemble_system(p)
    M = krylov.OneLevelAS(A, decomp.partition(p), weight="pou")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, prec, pkg.GENEO_AS_POU, pkg.GENEO_COARSE_NONE)
    r = np.random.default_rng(9).normal(size=s.ndof)
    r[p["dirichlet_dofs"]] = 0.0
    z = s.apply_preconditioner(r)
    assert np.array_equal(z, s.apply_preconditioner(r))
    assert rel(z, M(r)) <= (1e-9 if prec == 0 else 5e-3)
    s.close()


@pytest.mark.parametrize("name", ["small", "c1"])
def test_sarkis_geneo_pcg_matches_oracle(pkg, name):
    p = overlap2(name)
    ref = solver.solve(p, precond="geneo", tol=1e-8, eig_method="dense")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64)
    modes, lam, nh = s.coarse_info()
    assert list(modes) == ref["modes"] and nh == ref["n_coarse"]
    for j, lo in enumerate(ref["lambdas"]):
        kk = min(int(modes[j]) + 1, int(np.isfinite(lo).sum()), lam.shape[1])
        assert np.all(np.abs(lam[j, :kk] - lo[:kk]) <= 1e-7 * np.maximum(np.abs(lo[:kk]), 1e-2)), j
    Phi, _ = s.coarse()
    Zo, _ = geneo.coarse_space(p, decomp.partition(p), ref["A"], "dense")
    assert sla.subspace_angles(Phi, Zo.toarray()).max() <= span_tolerance(
        ref["modes"], ref["lambdas"], p["modes"]["shift"])
    u, st = s.solve(tol=1e-8, max_it=2000)
    s.close()
    assert rel(u, ref["u"]) <= 1e-6
    assert abs(st["iterations"] - ref["iterations"]) <= 2
    assert st["rel_res_true"] <= 2e-8


def test_sarkis_equals_multiplicity_at_overlap_one(pkg):
    p = workloads.config("c1")
    r = np.random.default_rng(4).normal(size=3 * 9 * 9 * 9)
    r[p["dirichlet_dofs"]] = 0.0
    out = []
    for pou, sch in (("standard", pkg.GENEO_AS_POU), ("sarkis", pkg.GENEO_AS_POU),
                     ("standard", pkg.GENEO_AS), ("sarkis", pkg.GENEO_AS)):
        s = pkg.GeneoSolver()
        s.assemble(p)
        s.setup(dict(p, pou=pou), pkg.GENEO_FP64, sch)
        out.append(s.apply_preconditioner(r))
        s.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[2], out[3])
