"""Pins for the oracle's zero-energy-mode (ZEM) coarse space (Sec. 5, Table 1).

The rigid modes must be annihilated by the Neumann matrix of a floating
subdomain (zero strain energy), span the same space as GenEO's lambda = 0
eigenvectors there, and a clamped subdomain must contribute none.  With the
ZEM coarse space PCG must need fewer iterations than one-level AS and more
than GenEO, the ordering of Table 1.
"""
import numpy as np
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
