"""GenEO coarse space (Sec. 3.2 and Sec. 3.3.2-3.3.3).

Per subdomain j (Sec. 3.3.2, eqm:matrixForm):
    A_{Omega_j} p = lambda (X_j A_{Omega_j^o} X_j) p,  ||p||_2 = 1,
with A_{Omega_j} the Neumann stiffness matrix assembled from the elements of
Omega_j (no artificial Dirichlet conditions) and A_{Omega_j^o} the one
assembled from the overlap elements only.  Global Dirichlet dofs keep an
identity row in A_{Omega_j}; X_j is zero there so they carry infinite
eigenvalues.

The eigenpairs come from the shift-and-invert transformation with a small
negative shift sigma (Sec. 3.3.2): with S = A - sigma B (SPD for sigma < 0),
    B p = mu S p,  lambda = sigma + 1 / mu,
so the smallest lambda are the largest mu.  Small problems use a dense
symmetric-definite solver on (B, S); large ones use ARPACK (the paper's
eigensolver) on the same pencil, with S as the inner-product matrix and a
sparse LU of S for its inverse.  B is only semi-definite, so handing it to
ARPACK as the inner-product matrix (its shift-invert mode on (A, B, sigma))
would make the returned vectors orthogonal only modulo ker B: with clustered
eigenvalues two of them can coincide on the support of X_j.

Coarse basis (Sec. 3.3.2): Phi_{i(j,k)} = R_j^T X_j p_k^j; coarse matrix
(Sec. 3.3.3) A_H = Phi^T A Phi with the fully assembled global A.

The zero-energy-mode coarse space (ZEM, the comparison of Sec. 5, Example 1
and Table 1) keeps instead the kernel of every local Neumann problem: the six
rigid displacements of a floating subdomain, none for a subdomain that
touches the clamped boundary (its Neumann matrix is non-singular), stitched
with the same partition of unity.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import decomp, fem

DENSE_LIMIT = 3000
INF_MU_RTOL = 1e-12    # mu below this times 1/|sigma| means lambda = infinity


def local_node_map(p, nodes):
    m = -np.ones(decomp.nnodes(p), np.int64)
    m[nodes] = np.arange(nodes.size)
    return m


def local_matrices(p, s):
    """(A_{Omega_j}, A_{Omega_j^o}) on the dofs of all nodes of Omega_j.

    Global Dirichlet dofs: A gets an identity row/column, A^o a zero one.
    """
    nm = local_node_map(p, s.neu_nodes)
    nloc = s.neu_nodes.size
    nc = decomp.ncomp(p)
    if nc == 1:
        from . import darcy
        assemble = darcy.assemble_matrix
    elif decomp.serendipity(p):
        from . import serendipity
        assemble = serendipity.assemble_stiffness_on
    else:
        assemble = fem.assemble_stiffness
    A = assemble(p, s.elems, nm, nloc)
    if s.ovl_elems.size:
        Ao = assemble(p, s.ovl_elems, nm, nloc)
    else:
        Ao = sp.csr_matrix((nc * nloc, nc * nloc))
    dmask = np.zeros(nc * decomp.nnodes(p), bool)
    dmask[np.asarray(p["dirichlet_dofs"], np.int64)] = True
    ld = np.nonzero(dmask[s.neu_dofs])[0]
    zeros = np.zeros(ld.size)
    A, _ = fem.apply_dirichlet(A, np.zeros(A.shape[0]), ld, zeros, diag=1.0)
    Ao, _ = fem.apply_dirichlet(Ao, np.zeros(Ao.shape[0]), ld, zeros, diag=0.0)
    return A, Ao


def eigenpairs(A, B, nev, sigma, method="auto"):
    """Smallest nev eigenpairs of A p = lambda B p (eqm:matrixForm), ||p|| = 1.

    Returns (lam ascending, P with unit-2-norm columns).
    """
    n = A.shape[0]
    nev = min(nev, n - 1)
    if method == "auto":
        method = "dense" if n <= DENSE_LIMIT else "arpack"
    if method == "dense":
        Ad = A.toarray()
        Bd = B.toarray()
        S = Ad - sigma * Bd
        mu, V = sla.eigh(Bd, S)                     # ascending mu
        mu = mu[::-1][:nev]
        V = V[:, ::-1][:, :nev]
        # mu -> 0 marks the infinite eigenvalues (null space of B)
        finite = mu > INF_MU_RTOL / abs(sigma)
        lam = np.full(mu.shape, np.inf)
        lam[finite] = sigma + 1.0 / mu[finite]
    elif method == "arpack":
        # the same shift-invert pencil as the dense branch, B v = mu S v with
        # S = A - sigma B SPD as the inner-product matrix (B is only
        # semi-definite, so it cannot serve as one: vectors would be
        # orthogonal only modulo ker B)
        S = (A - sigma * B).tocsc()
        lu = spla.splu(S)
        Sinv = spla.LinearOperator(S.shape, matvec=lu.solve, dtype=np.float64)
        mu, V = spla.eigsh(B.tocsc(), k=nev, M=S, Minv=Sinv, which="LA",
                           tol=1e-12, maxiter=20000)
        order = np.argsort(mu)[::-1]
        mu, V = mu[order], V[:, order]
        finite = mu > INF_MU_RTOL / abs(sigma)
        lam = np.full(mu.shape, np.inf)
        lam[finite] = sigma + 1.0 / mu[finite]
    else:
        raise ValueError(method)
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    return lam, V


def threshold(p, s):
    """Default eigenvalue threshold diam(Omega_j) / width(Omega_j^o) (Sec. 3.2).

    Reading of the footnote for a 3D box: diam = circumradius of Omega_j's box
    (half its diagonal); width = inradius of the overlap shell = O times the
    smallest element edge in Omega_j (half the shell thickness 2 O h).
    """
    x, y, z = p["x"], p["y"], p["z"]
    (x0, x1), (y0, y1), (z0, z1) = s.ebox
    diam = 0.5 * np.sqrt((x[x1] - x[x0]) ** 2 + (y[y1] - y[y0]) ** 2
                         + (z[z1] - z[z0]) ** 2)
    hmin = min(np.min(np.diff(x[x0:x1 + 1])), np.min(np.diff(y[y0:y1 + 1])),
               np.min(np.diff(z[z0:z1 + 1])))
    O = p["partition"][3]
    return diam / (O * hmin)


CLUSTER_RTOL = 1e-6
CLUSTER_ATOL = 1e-9


def select_modes(lam, fixed_modes, tau, max_modes):
    """Number of modes m_j kept (Sec. 3.2: all lambda below the threshold).

    fixed_modes > 0 keeps exactly that many; otherwise lambda <= tau, capped at
    max_modes.  Infinite eigenvalues (null space of B) are never kept.  If the cut falls inside a cluster of (numerically) equal
    eigenvalues, the whole cluster is dropped so the selected span is unique.
    """
    nfin = int(np.sum(np.isfinite(lam)))
    if fixed_modes > 0:
        m = min(fixed_modes, nfin)
    else:
        m = int(np.sum(lam <= tau))
        m = min(m, max_modes, nfin)
    while 0 < m < nfin:
        a, b = lam[m - 1], lam[m]
        if abs(b - a) <= CLUSTER_RTOL * max(abs(a), abs(b)) + CLUSTER_ATOL:
            m -= 1
        else:
            break
    return m


def coarse_space(p, subs, A, eig_method="auto"):
    """GenEO coarse basis Z (ndof x N_H, sparse) and per-subdomain data.

    Returns (Z, info) with info[j] = dict(lam, m, tau).
    """
    md = p["modes"]
    sigma = md["shift"]
    fixed, cap = md["fixed_modes"], md["max_modes"]
    cols, info = [], []
    ndof = A.shape[0]
    for s in subs:
        Aj, Aoj = local_matrices(p, s)
        Xd = sp.diags(s.X)
        Bj = (Xd @ Aoj @ Xd).tocsr()
        nev = (fixed if fixed > 0 else cap) + 1
        lam, P = eigenpairs(Aj, Bj, nev, sigma, eig_method)
        tau = md["threshold"] if md["threshold"] > 0 else threshold(p, s)
        m = select_modes(lam, fixed, tau, cap)
        for k in range(m):
            phi = np.zeros(ndof)
            phi[s.neu_dofs] = s.X * P[:, k]
            cols.append(phi)
        info.append(dict(lam=lam, m=m, tau=tau, P=P[:, :m]))
    if cols:
        Z = sp.csc_matrix(np.array(cols).T)
    else:
        Z = sp.csc_matrix((ndof, 0))
    return Z, info


def coarse_matrix(A, Z):
    """A_H = R_H A R_H^T with R_H^T = Z (Sec. 3.3.3); dense."""
    return (Z.T @ (A @ Z)).toarray()


def rigid_body_modes(p, nodes):
    """The six rigid displacements of `nodes` (3 dofs each), ||column||_2 = 1.

    Columns: translations along x, y, z; rotations about the x, y and z axes
    through the centre of the nodes' bounding box (u = omega x (X - c)).
    """
    if decomp.serendipity(p):
        from . import serendipity
        X = serendipity.node_coordinates(p)[nodes]
    else:
        nnx, nny = p["nx"] + 1, p["ny"] + 1
        i = nodes % nnx
        j = (nodes // nnx) % nny
        k = nodes // (nnx * nny)
        X = np.stack([np.asarray(p["x"])[i], np.asarray(p["y"])[j], np.asarray(p["z"])[k]], axis=1)
    c = 0.5 * (X.min(axis=0) + X.max(axis=0))
    d = X - c
    n = nodes.size
    R = np.zeros((3 * n, 6))
    for a in range(3):
        R[a::3, a] = 1.0
    # omega = e_x: (0, -dz, dy); e_y: (dz, 0, -dx); e_z: (-dy, dx, 0)
    R[1::3, 3], R[2::3, 3] = -d[:, 2], d[:, 1]
    R[0::3, 4], R[2::3, 4] = d[:, 2], -d[:, 0]
    R[0::3, 5], R[1::3, 5] = -d[:, 1], d[:, 0]
    return R / np.linalg.norm(R, axis=0)


def zem_space(p, subs, A):
    """ZEM coarse basis Z (ndof x N_H, sparse): R_j^T X_j r_k for the rigid
    modes r_k of every floating subdomain (no global Dirichlet dof in Omega_j).

    Returns (Z, info) with info[j] = dict(lam, m, floating) (lam = 0 for the
    kept modes: they span the kernel of A_{Omega_j}).
    """
    ndof = A.shape[0]
    dmask = np.zeros(ndof, bool)
    dmask[np.asarray(p["dirichlet_dofs"], np.int64)] = True
    cols, info = [], []
    nc = decomp.ncomp(p)
    for s in subs:
        floating = not dmask[s.neu_dofs].any()
        m = (6 if nc == 3 else 1) if floating else 0
        if m:
            # the kernel of the Neumann problem: rigid displacements, or the
            # constants for the scalar problem
            R = (rigid_body_modes(p, s.neu_nodes) if nc == 3
                 else np.full((s.neu_nodes.size, 1), 1.0 / np.sqrt(s.neu_nodes.size)))
            for k in range(m):
                phi = np.zeros(ndof)
                phi[s.neu_dofs] = s.X * R[:, k]
                cols.append(phi)
        info.append(dict(lam=np.zeros(m), m=m, floating=floating))
    Z = sp.csc_matrix(np.array(cols).T) if cols else sp.csc_matrix((ndof, 0))
    return Z, info
