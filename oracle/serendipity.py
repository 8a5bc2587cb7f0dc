"""20-node serendipity hexahedra for anisotropic elasticity (Sec. 2, Sec. 5).

Test infrastructure only, like the rest of `oracle/`: a plain FP64 statement
of the paper's quadratic element (20-node serendipity, full Gaussian
integration) on tensor-product blocks, for checking a GPU element later.

Reference cube [-1, 1]^3 with the 8 corners and the 12 edge midpoints as
nodes.  Shape functions of the serendipity family:
  corner (s1, s2, s3 in {-1, 1}):
      N = (1 + s1 xi)(1 + s2 eta)(1 + s3 zeta)(s1 xi + s2 eta + s3 zeta - 2) / 8
  midpoint of an edge along xi (xi_i = 0):
      N = (1 - xi^2)(1 + s2 eta)(1 + s3 zeta) / 4        (and likewise along eta, zeta)
Full integration: 3 x 3 x 3 Gauss-Legendre points (exact for these products on
box elements).  Mesh nodes of an nx x ny x nz block are the points of the
doubled grid (2nx+1) x (2ny+1) x (2nz+1) with at most one odd coordinate
(corners: none, edge midpoints: one), numbered in lexicographic order with
the doubled x index fastest; dof = 3 n + c as for the trilinear element.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fem import element_voigt_all

_C = [(ia, ja, ka) for ka in (0, 1) for ja in (0, 1) for ia in (0, 1)]
_E = ([(1, 2 * j, 2 * k) for k in (0, 1) for j in (0, 1)] +      # edges along x
      [(2 * i, 1, 2 * k) for k in (0, 1) for i in (0, 1)] +      # edges along y
      [(2 * i, 2 * j, 1) for j in (0, 1) for i in (0, 1)])       # edges along z
# local nodes as doubled-grid offsets (0, 1, 2) inside the element
LOCAL_OFFSETS = np.array([(2 * a, 2 * b, 2 * c) for a, b, c in _C] + _E)
REF_NODES = LOCAL_OFFSETS - 1.0                                   # in [-1, 1]^3

GAUSS3 = (np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)]), np.array([5.0, 8.0, 5.0]) / 9.0)


def shape(xi, eta, zeta):
    """N_a (20,) at a point of the reference cube."""
    t = np.array([xi, eta, zeta])
    N = np.empty(20)
    for a, s in enumerate(REF_NODES):
        if a < 8:
            f = (1.0 + s * t)
            N[a] = f[0] * f[1] * f[2] * (s @ t - 2.0) / 8.0
        else:
            d = int(np.flatnonzero(s == 0.0)[0])        # the edge's axis
            o = [e for e in range(3) if e != d]
            N[a] = (1.0 - t[d] ** 2) * (1.0 + s[o[0]] * t[o[0]]) * (1.0 + s[o[1]] * t[o[1]]) / 4.0
    return N


def shape_grad(xi, eta, zeta):
    """dN_a / d(xi, eta, zeta) (20, 3)."""
    t = np.array([xi, eta, zeta])
    G = np.empty((20, 3))
    for a, s in enumerate(REF_NODES):
        if a < 8:
            f = 1.0 + s * t
            lin = s @ t - 2.0
            for d in range(3):
                o = [e for e in range(3) if e != d]
                G[a, d] = s[d] * f[o[0]] * f[o[1]] * (lin + f[d]) / 8.0
        else:
            d = int(np.flatnonzero(s == 0.0)[0])
            o = [e for e in range(3) if e != d]
            g0 = 1.0 + s[o[0]] * t[o[0]]
            g1 = 1.0 + s[o[1]] * t[o[1]]
            G[a, d] = -2.0 * t[d] * g0 * g1 / 4.0
            G[a, o[0]] = (1.0 - t[d] ** 2) * s[o[0]] * g1 / 4.0
            G[a, o[1]] = (1.0 - t[d] ** 2) * g0 * s[o[1]] / 4.0
    return G


def strain_displacement(grad):
    """Voigt B (6 x 60), rows (xx, yy, zz, yz, xz, xy), engineering shear."""
    B = np.zeros((6, 60))
    for a in range(20):
        gx, gy, gz = grad[a]
        c = 3 * a
        B[0, c] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 1] = gz
        B[3, c + 2] = gy
        B[4, c] = gz
        B[4, c + 2] = gx
        B[5, c] = gy
        B[5, c + 1] = gx
    return B


def element_stiffness(Cv, hx, hy, hz):
    """K_e (60 x 60) = sum_g w_g |J| B_g^T C B_g over 3 x 3 x 3 Gauss points."""
    pts, wts = GAUSS3
    inv = np.array([2.0 / hx, 2.0 / hy, 2.0 / hz])
    detJ = hx * hy * hz / 8.0
    K = np.zeros((60, 60))
    for k, zeta in enumerate(pts):
        for j, eta in enumerate(pts):
            for i, xi in enumerate(pts):
                B = strain_displacement(shape_grad(xi, eta, zeta) * inv)
                K += wts[i] * wts[j] * wts[k] * detJ * (B.T @ Cv @ B)
    return K


def node_map(nx, ny, nz):
    """Doubled-grid point -> node id (-1 where no node), and the node count."""
    I, J, K = np.meshgrid(np.arange(2 * nx + 1), np.arange(2 * ny + 1), np.arange(2 * nz + 1),
                          indexing="ij")
    odd = (I % 2) + (J % 2) + (K % 2)
    keep = odd <= 1
    ids = -np.ones(I.shape, dtype=np.int64)
    order = np.argsort((K * (2 * ny + 1) + J) * (2 * nx + 1) + I, axis=None)
    flat_keep = keep.reshape(-1)[order]
    idx = np.cumsum(flat_keep) - 1
    ids_flat = ids.reshape(-1)
    ids_flat[order[flat_keep]] = idx[flat_keep]
    return ids, int(flat_keep.sum())


def element_nodes(ids, ex, ey, ez):
    """Global node ids (20,) of element (ex, ey, ez) in local order."""
    o = LOCAL_OFFSETS
    return ids[2 * ex + o[:, 0], 2 * ey + o[:, 1], 2 * ez + o[:, 2]]


def node_coordinates(p):
    """(nnodes, 3) coordinates of the serendipity mesh of problem p."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ids, nn = node_map(nx, ny, nz)

    def doubled(v):
        v = np.asarray(v, dtype=np.float64)
        out = np.empty(2 * len(v) - 1)
        out[0::2] = v
        out[1::2] = 0.5 * (v[:-1] + v[1:])
        return out
    X, Y, Z = doubled(p["x"]), doubled(p["y"]), doubled(p["z"])
    xyz = np.empty((nn, 3))
    I, J, K = np.nonzero(ids >= 0)
    xyz[ids[I, J, K]] = np.stack([X[I], Y[J], Z[K]], axis=1)
    return xyz


def assemble_stiffness(p):
    """Unconstrained global stiffness (CSR, 3 nnodes square) of problem p's block
    meshed with serendipity elements and its per-element materials."""
    nn = nnodes(p)
    return assemble_stiffness_on(p, np.arange(p["nx"] * p["ny"] * p["nz"]),
                                 np.arange(nn), nn)


def face_shape(xi, eta):
    """The eight serendipity functions of a face (the element's z = +1 face
    restricted to it), in the order corners (as the element's 4 top corners)
    then mid-edges along x (eta = -1, +1) and along y (xi = -1, +1)."""
    s = np.array([(-1, -1), (1, -1), (-1, 1), (1, 1)], dtype=np.float64)
    N = np.empty(8)
    for a, (s1, s2) in enumerate(s):
        N[a] = (1 + s1 * xi) * (1 + s2 * eta) * (s1 * xi + s2 * eta - 1) / 4.0
    N[4] = (1 - xi ** 2) * (1 - eta) / 2.0
    N[5] = (1 - xi ** 2) * (1 + eta) / 2.0
    N[6] = (1 - xi) * (1 - eta ** 2) / 2.0
    N[7] = (1 + xi) * (1 - eta ** 2) / 2.0
    return N


# element-local nodes of the z = +1 face in face_shape's order
TOP_FACE = [4, 5, 6, 7, 10, 11, 14, 15]


def top_pressure_load(p):
    """Consistent nodal load of traction (0, 0, -q) on z = z_max: int_face N_a t dA
    with the 8-node face functions, 3 x 3 Gauss points (corners get -1/12 and
    mid-edges 1/3 of the face's force)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ids, nn = node_map(nx, ny, nz)
    x, y = np.asarray(p["x"], dtype=np.float64), np.asarray(p["y"], dtype=np.float64)
    q = p["top_pressure"]
    pts, wts = GAUSS3
    fN = np.zeros(8)
    for j, eta in enumerate(pts):
        for i, xi in enumerate(pts):
            fN += wts[i] * wts[j] * face_shape(xi, eta) / 4.0     # int over the unit face
    b = np.zeros(3 * nn)
    for ey in range(ny):
        for ex in range(nx):
            area = (x[ex + 1] - x[ex]) * (y[ey + 1] - y[ey])
            nodes = element_nodes(ids, ex, ey, nz - 1)[TOP_FACE]
            np.add.at(b, 3 * nodes + 2, -q * area * fN)
    return b


def clamp_dofs(p):
    """Dofs of the nodes on x = 0 (the cantilever's clamp)."""
    nodes = np.flatnonzero(node_coordinates(p)[:, 0] == np.asarray(p["x"])[0])
    return (3 * nodes[:, None] + np.arange(3)).reshape(-1)


def assemble_system(p):
    """Loaded on the top face, with the Dirichlet rows eliminated symmetrically as
    for the trilinear element: p's serendipity-numbered Dirichlet dofs when p is
    a serendipity problem, else the clamp at x = 0."""
    from .fem import apply_dirichlet
    A = assemble_stiffness(p)
    b = top_pressure_load(p)
    if p.get("element") == "serendipity":
        D = np.asarray(p["dirichlet_dofs"], np.int64)
        g = np.asarray(p["dirichlet_values"], np.float64)
    else:
        D = clamp_dofs(p)
        g = np.zeros(len(D))
    return apply_dirichlet(A, b, D, g)


def nnodes(p):
    return node_map(p["nx"], p["ny"], p["nz"])[1]


def box_nodes(p, dlo, dhi):
    """Sorted ids of the nodes whose doubled-grid coordinates lie in [dlo, dhi]."""
    ids, _ = node_map(p["nx"], p["ny"], p["nz"])
    sub = ids[dlo[0]:dhi[0] + 1, dlo[1]:dhi[1] + 1, dlo[2]:dhi[2] + 1]
    return np.sort(sub[sub >= 0].reshape(-1))


def assemble_stiffness_on(p, elems, node_map_local, n_local_nodes):
    """sum_e K_e over `elems` on a local node set (global node -> local id)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ids, _ = node_map(nx, ny, nz)
    Cv = element_voigt_all(p)
    x, y, z = (np.asarray(p[k], dtype=np.float64) for k in ("x", "y", "z"))
    rows, cols, vals = [], [], []
    cache = {}
    for e in np.asarray(elems):
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        h = (x[ex + 1] - x[ex], y[ey + 1] - y[ey], z[ez + 1] - z[ez])
        key = (Cv[e].tobytes(), h)
        Ke = cache.get(key)
        if Ke is None:
            Ke = element_stiffness(Cv[e], *h)
            cache[key] = Ke
        loc = node_map_local[element_nodes(ids, ex, ey, ez)]
        dofs = (3 * loc[:, None] + np.arange(3)).reshape(-1)
        rows.append(np.repeat(dofs, 60))
        cols.append(np.tile(dofs, 60))
        vals.append(Ke.reshape(-1))
    n = 3 * n_local_nodes
    if not rows:
        return sp.csr_matrix((n, n))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def problem(p):
    """A copy of the block problem p meshed with serendipity elements: the same
    geometry, materials, partition and load, with the clamp on x = 0 numbered on
    the serendipity mesh."""
    q = dict(p)
    q["element"] = "serendipity"
    D = clamp_dofs(q)
    q["dirichlet_dofs"] = D.astype(np.int32)
    q["dirichlet_values"] = np.zeros(len(D))
    return q
