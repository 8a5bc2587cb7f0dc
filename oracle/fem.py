"""Trilinear hexahedral finite elements for anisotropic elasticity (Sec. 2).

The weak form a(u, v) = int sigma(u) : eps(v) dx = b(v) (Sec. 2, eq-fe) is
discretised with conforming trilinear (Q1) elements on a tensor-product mesh;
the vector basis is blocked per node (B = R^3, eqn:fe_matrix_system) and the
system is assembled element by element with Gaussian integration (end of
Sec. 2): here 2x2x2 Gauss-Legendre points (full integration).

Node n = i + (nx+1)(j + (ny+1)k), dof = 3n + c.  Local element node
a = ia + 2 ja + 4 ka sits at mesh node (ex+ia, ey+ja, ez+ka).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import material

GAUSS_1D = (-1.0 / np.sqrt(3.0), 1.0 / np.sqrt(3.0))   # weights 1, 1
CORNERS = np.array([(ia, ja, ka) for ka in (0, 1) for ja in (0, 1) for ia in (0, 1)])


def shape_grad_ref(xi, eta, zeta):
    """d N_a / d(xi, eta, zeta) for N_a = prod (1 + s_a t) / 2 on [-1, 1]^3."""
    s = 2.0 * CORNERS - 1.0          # (8, 3) corner signs
    fx = 0.5 * (1.0 + s[:, 0] * xi)
    fy = 0.5 * (1.0 + s[:, 1] * eta)
    fz = 0.5 * (1.0 + s[:, 2] * zeta)
    g = np.empty((8, 3))
    g[:, 0] = 0.5 * s[:, 0] * fy * fz
    g[:, 1] = fx * 0.5 * s[:, 1] * fz
    g[:, 2] = fx * fy * 0.5 * s[:, 2]
    return g


def strain_displacement(grad):
    """Voigt B matrix (6 x 24), rows (xx, yy, zz, yz, xz, xy), engineering shear."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = grad[a]
        c = 3 * a
        B[0, c + 0] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 1] = gz
        B[3, c + 2] = gy
        B[4, c + 0] = gz
        B[4, c + 2] = gx
        B[5, c + 0] = gy
        B[5, c + 1] = gx
    return B


def gauss_B(hx, hy, hz):
    """B at the 8 Gauss points of an hx x hy x hz box and det J (J diagonal)."""
    inv = np.array([2.0 / hx, 2.0 / hy, 2.0 / hz])
    Bs = []
    for zeta in GAUSS_1D:
        for eta in GAUSS_1D:
            for xi in GAUSS_1D:
                Bs.append(strain_displacement(shape_grad_ref(xi, eta, zeta) * inv))
    return np.array(Bs), hx * hy * hz / 8.0


def element_stiffness(Cv, hx, hy, hz):
    """K_e = sum_g w_g |J| B_g^T C B_g over 2x2x2 Gauss points (w_g = 1)."""
    Bs, detJ = gauss_B(hx, hy, hz)
    K = np.zeros((24, 24))
    for B in Bs:
        K += B.T @ Cv @ B * detJ
    return K


def element_dofs(nx, ny, ex, ey, ez):
    """Global dofs (24,) of element (ex, ey, ez), ordered 3a + c."""
    nnx, nny = nx + 1, ny + 1
    n = (ex + CORNERS[:, 0]) + nnx * ((ey + CORNERS[:, 1]) + nny * (ez + CORNERS[:, 2]))
    return (3 * n[:, None] + np.arange(3)[None, :]).reshape(-1)


def element_coords(p):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    e = np.arange(nx * ny * nz)
    return e % nx, (e // nx) % ny, e // (nx * ny)


def element_voigt_all(p):
    """Per-element global-frame Voigt stiffness (nel, 6, 6) (Sec. 2 eq-hooke)."""
    mats, em = p["materials"], p["elem_mat"]
    th = p["elem_theta"]
    ph = p["elem_phi"] if p.get("elem_phi") is not None else np.zeros_like(th)
    keys = np.stack([em.astype(np.float64), th, ph], axis=1)
    uk, inv = np.unique(keys, axis=0, return_inverse=True)
    Cu = np.array([material.element_stiffness_voigt(mats[int(k[0])], k[1], k[2])
                   for k in uk])
    return Cu[inv.reshape(-1)]


def element_stiffness_all(p, elems=None):
    """K_e (len(elems), 24, 24) for the given element ids (all if None).

    Elements sharing material, angles and box size share one K_e computation.
    """
    nx, ny = p["nx"], p["ny"]
    x, y, z = p["x"], p["y"], p["z"]
    if elems is None:
        elems = np.arange(nx * ny * p["nz"])
    elems = np.asarray(elems)
    ex, ey, ez = elems % nx, (elems // nx) % ny, elems // (nx * ny)
    hx, hy, hz = x[ex + 1] - x[ex], y[ey + 1] - y[ey], z[ez + 1] - z[ez]
    th = p["elem_theta"][elems]
    ph = (p["elem_phi"][elems] if p.get("elem_phi") is not None
          else np.zeros_like(th))
    keys = np.stack([p["elem_mat"][elems].astype(np.float64), th, ph,
                     hx, hy, hz], axis=1)
    uk, inv = np.unique(keys, axis=0, return_inverse=True)
    Ku = np.empty((len(uk), 24, 24))
    cache = {}
    for i, k in enumerate(uk):
        ck = (int(k[0]), k[1], k[2])
        if ck not in cache:
            cache[ck] = material.element_stiffness_voigt(p["materials"][ck[0]], ck[1], ck[2])
        Ku[i] = element_stiffness(cache[ck], k[3], k[4], k[5])
    return Ku, inv.reshape(-1), elems


def assemble_stiffness(p, elems=None, node_map=None, n_local_nodes=None):
    """A = sum_e K_e scattered by dof (Sec. 2, element-wise assembly).

    With node_map (global node -> local node, -1 outside) the matrix is built
    on the local node set only (used for subdomain Neumann matrices).
    Returns scipy CSR.
    """
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    Ku, inv, elems = element_stiffness_all(p, elems)
    ex, ey, ez = elems % nx, (elems // nx) % ny, elems // (nx * ny)
    nnx, nny = nx + 1, ny + 1
    nodes = ((ex[:, None] + CORNERS[None, :, 0])
             + nnx * ((ey[:, None] + CORNERS[None, :, 1])
                      + nny * (ez[:, None] + CORNERS[None, :, 2])))   # (E, 8)
    if node_map is not None:
        nodes = node_map[nodes]
        ndof = 3 * n_local_nodes
    else:
        ndof = 3 * nnx * nny * (nz + 1)
    dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(len(elems), 24)
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    vals = Ku[inv].reshape(-1)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(ndof, ndof)).tocsr()
    A.sum_duplicates()
    return A


def top_pressure_load(p):
    """Consistent nodal load of traction (0, 0, -q) on the face z = z_max.

    int_face N_a t dA = -q * hx * hy / 4 for each of the 4 top nodes of a
    bilinear face (Sec. 2 eq-fe boundary term; Sec. 5 Example 1 load).
    """
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x, y = p["x"], p["y"]
    q = p["top_pressure"]
    nnx, nny = nx + 1, ny + 1
    b = np.zeros(3 * nnx * nny * (nz + 1))
    for ey in range(ny):
        for ex in range(nx):
            f = -q * (x[ex + 1] - x[ex]) * (y[ey + 1] - y[ey]) / 4.0
            for dj in (0, 1):
                for di in (0, 1):
                    n = (ex + di) + nnx * ((ey + dj) + nny * nz)
                    b[3 * n + 2] += f
    if p.get("nodal_load") is not None:
        b += p["nodal_load"]
    return b


def apply_dirichlet(A, b, dofs, values, diag=1.0):
    """Symmetric elimination: b -= A[:, D] g; zero rows/cols D; A_DD = diag; b_D = g.

    Sec. 2 (eq-fctspace) fixes u_i = h_i on the Dirichlet part; eliminating
    symmetrically keeps A symmetric positive definite (eqn:fe_matrix_system).
    """
    n = A.shape[0]
    dofs = np.asarray(dofs, dtype=np.int64)
    g = np.zeros(n)
    g[dofs] = values
    b = b - A @ g
    mask = np.ones(n)
    mask[dofs] = 0.0
    P = sp.diags(mask)
    A = (P @ A @ P).tocsr()
    A = A + sp.diags(np.where(mask == 0.0, diag, 0.0))
    A = A.tocsr()
    A.eliminate_zeros()
    b[dofs] = values
    return A, b


def assemble_system(p):
    """Global A (CSR, Dirichlet eliminated) and load b (eqn:fe_matrix_system);
    the scalar Darcy problem (eq-fe-darcy) when p["kind"] == "darcy"."""
    if p.get("kind") == "darcy":
        from . import darcy
        return darcy.assemble_system(p)
    if p.get("element") == "serendipity":
        from . import serendipity
        return serendipity.assemble_system(p)
    A = assemble_stiffness(p)
    b = top_pressure_load(p)
    return apply_dirichlet(A, b, p["dirichlet_dofs"], p["dirichlet_values"])


def element_stresses(p, u):
    """Stress recovery: sigma_e = C_e B(centroid) u_e at every element (nel, 6).

    Voigt order (xx, yy, zz, yz, xz, xy); C_e is the rotated ply stiffness of
    the element (Sec. 2 constitutive law), B the strain-displacement matrix of
    the trilinear element at its centre (engineering shear strains).  The
    paper recovers stresses from the displacement solution for its failure
    analysis (Sec. 5); the centroid is the one point where the Q1 strain of a
    box element is the element average.
    """
    Cv = element_voigt_all(p)
    ex, ey, ez = element_coords(p)
    x, y, z = np.asarray(p["x"]), np.asarray(p["y"]), np.asarray(p["z"])
    g0 = shape_grad_ref(0.0, 0.0, 0.0)
    out = np.zeros((ex.size, 6))
    for e in range(ex.size):
        h = np.array([x[ex[e] + 1] - x[ex[e]], y[ey[e] + 1] - y[ey[e]], z[ez[e] + 1] - z[ez[e]]])
        B = strain_displacement(g0 * (2.0 / h))
        eps = B @ u[element_dofs(p["nx"], p["ny"], ex[e], ey[e], ez[e])]
        out[e] = Cv[e] @ eps
    return out
