"""Pins for the oracle's decomposition and GenEO stages on the 20-node
serendipity mesh (the paper's element, Sec. 5, with Sec. 3.1-3.3).

Subdomain node sets against brute force on the element-node incidence:
Omega_j's closure holds exactly the nodes of its elements, and V_{h,0}(Omega_j)
exactly the nodes whose every element lies in Omega_j (the basis function is
supported in Omega_j), on both the serendipity and the trilinear mesh.  PoU:
sum_j R_j^T X_j R_j 1 = 1 on free dofs.  GenEO: on a floating subdomain the
generalised eigenproblem has exactly six zero eigenvalues and their
eigenspace is the rigid displacements of the subdomain's nodes.  Solver: PCG
with the GenEO preconditioner equals a dense direct solve, and the clamp
makes the serendipity system SPD; on an unclamped block both the ZEM and the
GenEO coarse spaces contain the six global rigid displacements.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import decomp, fem, geneo, serendipity as sd, solver
from workloads.laminate import make_block


def _problem(partition=(2, 1, 2, 1)):
    return sd.problem(make_block(4, 2, 4, [0.0, 90.0], partition=partition))


def _incidence(q):
    """(nodes of each element, elements of each node) by brute force."""
    nx, ny, nz = q["nx"], q["ny"], q["nz"]
    if decomp.serendipity(q):
        ids, nn = sd.node_map(nx, ny, nz)
        en = [sd.element_nodes(ids, e % nx, (e // nx) % ny, e // (nx * ny))
              for e in range(nx * ny * nz)]
    else:
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        en = [fem.element_dofs(nx, ny, e % nx, (e // nx) % ny, e // (nx * ny))[0::3] // 3
              for e in range(nx * ny * nz)]
    adj = [set() for _ in range(nn)]
    for e, ns in enumerate(en):
        for n in ns:
            adj[int(n)].add(e)
    return en, adj


@pytest.mark.parametrize("element", ["serendipity", "trilinear"])
def test_subdomain_nodes_against_incidence(element):
    p = make_block(5, 3, 4, [0.0, 90.0], partition=(2, 2, 2, 1))
    q = sd.problem(p) if element == "serendipity" else p
    en, adj = _incidence(q)
    for s in decomp.partition(q):
        el = set(s.elems.tolist())
        closure = sorted({int(n) for e in el for n in en[e]})
        supported = sorted(n for n in range(len(adj)) if adj[n] <= el)
        assert s.neu_nodes.tolist() == closure
        assert s.int_nodes.tolist() == supported


def test_pou_identity():
    q = _problem((2, 2, 2, 1))
    subs = decomp.partition(q)
    v = decomp.pou_sum(q, subs)
    assert v.size == 3 * sd.nnodes(q)
    free = np.ones(v.size, bool)
    free[q["dirichlet_dofs"]] = False
    assert np.array_equal(v[free], np.ones(free.sum()))
    assert np.all(v[~free] == 0.0)


def test_floating_subdomain_has_the_rigid_modes():
    q = _problem((2, 1, 1, 1))                   # clamp at x = 0: the x-upper half floats
    subs = decomp.partition(q)
    top = [s for s in subs if s.ebox[0][0] > 0][0]
    A, Ao = geneo.local_matrices(q, top)
    Xd = sp.diags(top.X)
    lam, P = geneo.eigenpairs(A, (Xd @ Ao @ Xd).tocsr(), 8, -0.01, "dense")
    assert np.all(np.abs(lam[:6]) < 1e-8) and lam[6] > 1e-4
    R = geneo.rigid_body_modes(q, top.neu_nodes)
    assert sla.subspace_angles(P[:, :6], R).max() < 1e-6
    Az, _ = fem.assemble_system(q)
    _, info = geneo.zem_space(q, subs, Az)
    assert sorted(d["m"] for d in info) == [0, 6]


def test_system_spd_and_pcg_matches_direct_solve():
    q = _problem()
    A, b = fem.assemble_system(q)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T, atol=1e-12 * abs(Ad).max())
    np.linalg.cholesky(Ad)
    u_d = np.linalg.solve(Ad, b)
    r = solver.solve(q, precond="geneo", tol=1e-12)
    assert np.linalg.norm(r["u"] - u_d) <= 1e-9 * np.linalg.norm(u_d)


@pytest.mark.parametrize("coarse", ["zem", "geneo"])
def test_global_rigid_modes_lie_in_the_coarse_space(coarse):
    # unclamped 20-node block: every subdomain floats, its six rigid modes
    # weighted by the PoU rebuild the six global ones
    p = make_block(4, 2, 4, [0.0, 90.0], partition=(2, 1, 2, 1), clamp="none",
                   modes=dict(fixed_modes=6, threshold=0.0, max_modes=20, shift=-0.01))
    q = dict(p, element="serendipity", dirichlet_dofs=np.zeros(0, np.int32),
             dirichlet_values=np.zeros(0))
    subs = decomp.partition(q)
    A = sd.assemble_stiffness(q)
    Z, _ = (geneo.zem_space(q, subs, A) if coarse == "zem" else geneo.coarse_space(q, subs, A))
    Rg = geneo.rigid_body_modes(q, np.arange(sd.nnodes(q)))
    assert sla.subspace_angles(Z.toarray(), Rg).max() < 1e-8
