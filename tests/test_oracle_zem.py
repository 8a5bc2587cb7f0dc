"""Pins for the oracle's zero-energy-mode (ZEM) coarse space (Sec. 5, Table 1).

The rigid modes must be annihilated by the Neumann matrix of a floating
subdomain (zero strain energy), span the same space as GenEO's lambda = 0
eigenvectors there, and a clamped subdomain must contribute none.  With the
ZEM coarse space PCG must need fewer iterations than one-level AS and more
than GenEO, the ordering of Table 1.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import decomp, geneo, solver
import workloads


def _floating(p):
    subs = decomp.partition(p)
    return subs, [s for s in subs if s.ebox[0][0] > 0], [s for s in subs if s.ebox[0][0] == 0]


def test_rigid_modes_have_zero_energy_on_floating_subdomain():
    p = workloads.config("c1")
    subs, fl, _ = _floating(p)
    s = fl[0]
    A, _ = geneo.local_matrices(p, s)
    R = geneo.rigid_body_modes(p, s.neu_nodes)
    assert np.allclose(np.linalg.norm(R, axis=0), 1.0)
    assert np.abs(A @ R).max() <= 1e-12 * abs(A).max()
    # six independent columns
    assert np.linalg.matrix_rank(R, tol=1e-10) == 6


def test_a_wrong_rotation_is_not_a_zero_mode():
    # guards the pin above: a rotation with a flipped sign strains the body
    p = workloads.config("c1")
    _, fl, _ = _floating(p)
    s = fl[0]
    A, _ = geneo.local_matrices(p, s)
    R = geneo.rigid_body_modes(p, s.neu_nodes)
    bad = R[:, 5].copy()
    bad[1::3] *= -1.0            # (-dy, -dx, 0): a shear, not a rotation
    assert np.abs(A @ bad).max() > 1e-6 * abs(A).max()


def test_zem_span_equals_geneo_zero_eigenspace():
    p = workloads.config("c1")
    _, fl, _ = _floating(p)
    s = fl[0]
    A, Ao = geneo.local_matrices(p, s)
    Xd = sp.diags(s.X)
    lam, P = geneo.eigenpairs(A, (Xd @ Ao @ Xd).tocsr(), 8, -0.01, "dense")
    R = geneo.rigid_body_modes(p, s.neu_nodes)
    assert np.all(np.abs(lam[:6]) < 1e-9)
    assert sla.subspace_angles(P[:, :6], R).max() < 1e-8


def test_zem_modes_per_subdomain():
    p = workloads.config("c1")
    A, _ = solver.fem.assemble_system(p)
    subs = decomp.partition(p)
    Z, info = geneo.zem_space(p, subs, A)
    for s, d in zip(subs, info):
        assert d["m"] == (6 if s.ebox[0][0] > 0 else 0)
    assert Z.shape == (A.shape[0], 6 * sum(1 for s in subs if s.ebox[0][0] > 0))
    # columns are PoU-weighted modes: zero on the clamped dofs
    assert abs(Z[np.asarray(p["dirichlet_dofs"]), :]).max() == 0.0


def test_iterations_as_greater_than_zem_greater_than_geneo():
    p = workloads.config("small")
    it = {k: solver.solve(p, precond=k, tol=1e-8)["iterations"] for k in ("as", "zem", "geneo")}
    assert it["as"] > it["zem"] > it["geneo"], it


def test_rotation_columns_are_centred():
    # rotations are taken about the centre of the node set's bounding box, so
    # on a box node set they are orthogonal to the three translations
    p = workloads.config("c1")
    subs = decomp.partition(p)
    R = geneo.rigid_body_modes(p, subs[0].neu_nodes)
    assert np.abs(R[:, :3].T @ R[:, 3:]).max() <= 1e-13


@pytest.mark.parametrize("pou", ["standard", "sarkis"])
@pytest.mark.parametrize("coarse", ["zem", "geneo"])
def test_global_rigid_modes_lie_in_the_coarse_space(coarse, pou):
    # Unclamped block: every subdomain floats and keeps its six rigid modes,
    # weighted by its PoU; summed over the subdomains the PoU rebuilds each
    # global rigid displacement (sum_j R_j^T X_j R_j = I), so the coarse space
    # must contain all six.
    from oracle import fem
    p = workloads.config("small", clamp="none")
    p["modes"] = dict(fixed_modes=6, threshold=0.0, max_modes=20, shift=-0.01)
    p["pou"] = pou
    p["partition"] = tuple(p["partition"][:3]) + (2,)       # Sarkis differs from 1/multiplicity
    subs = decomp.partition(p)
    A = fem.assemble_stiffness(p)
    if coarse == "zem":
        Z, _ = geneo.zem_space(p, subs, A)
    else:
        Z, _ = geneo.coarse_space(p, subs, A)
    allnodes = np.arange(A.shape[0] // 3)
    Rg = geneo.rigid_body_modes(p, allnodes)
    assert sla.subspace_angles(Z.toarray(), Rg).max() < 1e-8
