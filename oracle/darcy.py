"""Scalar Darcy flow, the paper's subsurface application (Sec. on SPE10, eqn:Darcy).

-div(K grad u) = f in Omega, u = 0 on the face z = 0 and zero flux elsewhere,
K = diag(Kx, Ky, Kz) constant in each cell; Q1 (trilinear) elements on the
tensor-product grid, assembled element by element with 2x2x2 Gauss points
(eq-fe-darcy): A_ab = int K grad N_a . grad N_b dx, b_a = int f N_a dx.
One unknown per node (dof = node).  Test infrastructure only, like the rest
of the oracle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem


def element_matrix(kd, hx, hy, hz):
    """8 x 8 element matrix of the diagonal conductivity kd = (Kx, Ky, Kz)."""
    inv = np.array([2.0 / hx, 2.0 / hy, 2.0 / hz])
    detJ = hx * hy * hz / 8.0
    K = np.zeros((8, 8))
    for zeta in fem.GAUSS_1D:
        for eta in fem.GAUSS_1D:
            for xi in fem.GAUSS_1D:
                g = fem.shape_grad_ref(xi, eta, zeta) * inv        # (8, 3)
                K += (g * np.asarray(kd)[None, :]) @ g.T * detJ
    return K


def element_nodes(p, elems):
    nx, ny = p["nx"], p["ny"]
    nnx, nny = nx + 1, ny + 1
    ex, ey, ez = elems % nx, (elems // nx) % ny, elems // (nx * ny)
    c = fem.CORNERS
    return ((ex[:, None] + c[None, :, 0]) + nnx * ((ey[:, None] + c[None, :, 1])
                                                   + nny * (ez[:, None] + c[None, :, 2])))


def assemble_matrix(p, elems=None, node_map=None, n_local_nodes=None):
    """A over `elems` (all by default), optionally on a local node numbering."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    if elems is None:
        elems = np.arange(nx * ny * nz)
    elems = np.asarray(elems)
    x, y, z = np.asarray(p["x"]), np.asarray(p["y"]), np.asarray(p["z"])
    ex, ey, ez = elems % nx, (elems // nx) % ny, elems // (nx * ny)
    kxyz = np.asarray(p["perm"])[elems]                     # (ne, 3)
    nodes = element_nodes(p, elems)
    if node_map is not None:
        nodes = node_map[nodes]
        n = n_local_nodes
    else:
        n = (nx + 1) * (ny + 1) * (nz + 1)
    rows, cols, vals = [], [], []
    for e in range(elems.size):
        Ke = element_matrix(kxyz[e], x[ex[e] + 1] - x[ex[e]], y[ey[e] + 1] - y[ey[e]],
                            z[ez[e] + 1] - z[ez[e]])
        rows.append(np.repeat(nodes[e], 8))
        cols.append(np.tile(nodes[e], 8))
        vals.append(Ke.reshape(-1))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return A.tocsr()


def load(p):
    """b_a = int f N_a dx (uniform source f: f V_e / 8 per element node) + nodal_load."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x, y, z = np.asarray(p["x"]), np.asarray(p["y"]), np.asarray(p["z"])
    elems = np.arange(nx * ny * nz)
    ex, ey, ez = elems % nx, (elems // nx) % ny, elems // (nx * ny)
    vol = (x[ex + 1] - x[ex]) * (y[ey + 1] - y[ey]) * (z[ez + 1] - z[ez])
    b = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
    np.add.at(b, element_nodes(p, elems).reshape(-1), np.repeat(p["source"] * vol / 8.0, 8))
    if p.get("nodal_load") is not None:
        b += p["nodal_load"]
    return b


def assemble_system(p):
    """A (CSR, Dirichlet eliminated symmetrically) and b of eq-fe-darcy."""
    return fem.apply_dirichlet(assemble_matrix(p), load(p), p["dirichlet_dofs"],
                               p["dirichlet_values"])
