"""Overlapping box decomposition and partition of unity (Sec. 3.1-3.3).

Sec. 3.1: non-overlapping subdomains Omega'_j resolved by the mesh, each
extended by O layers of elements to Omega_j; V_{h,0}(Omega_j) holds the FE
functions supported in Omega_j, i.e. zero on the artificial boundary
(points of the boundary of Omega_j that lie inside another subdomain).
Sec. 3.2 (Def. Subdomain Overlap): Omega_j^o is the part of Omega_j that lies
in another subdomain; read element-wise here: the elements of Omega_j that
also belong to some other Omega_k.
Sec. 3.3.1: the standard PoU X^(j) is diagonal, 1 / (number of subdomains
containing the dof), zero on the subdomain boundary, with global Dirichlet
conditions enforced (zero there as well).

Box split: an axis with n elements and p parts gives part k the elements
[floor(k n / p), floor((k + 1) n / p)).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def axis_split(n, p):
    return [(k * n // p, (k + 1) * n // p) for k in range(p)]


@dataclass
class Subdomain:
    index: int
    owned: tuple            # ((lo, hi) per axis), elements, half-open
    ebox: tuple             # element box of Omega_j, half-open per axis
    elems: np.ndarray       # element ids in Omega_j
    neu_nodes: np.ndarray   # all nodes of Omega_j (closure), sorted
    int_nodes: np.ndarray   # nodes of V_{h,0}(Omega_j), sorted
    neu_dofs: np.ndarray = field(default=None)
    int_dofs: np.ndarray = field(default=None)
    X: np.ndarray = field(default=None)          # PoU on neu_dofs
    ovl_elems: np.ndarray = field(default=None)  # elements of Omega_j^o


def _box_nodes(p, lo, hi):
    nnx, nny = p["nx"] + 1, p["ny"] + 1
    i = np.arange(lo[0], hi[0] + 1)
    j = np.arange(lo[1], hi[1] + 1)
    k = np.arange(lo[2], hi[2] + 1)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    return np.sort((I + nnx * (J + nny * K)).reshape(-1))


def _box_elems(p, lo, hi):
    nx, ny = p["nx"], p["ny"]
    i = np.arange(lo[0], hi[0])
    j = np.arange(lo[1], hi[1])
    k = np.arange(lo[2], hi[2])
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    return np.sort((I + nx * (J + ny * K)).reshape(-1))


def ncomp(p):
    """Unknowns per node: 1 for the scalar Darcy problem, 3 for elasticity."""
    return 1 if p.get("kind") == "darcy" else 3


def serendipity(p):
    return p.get("element") == "serendipity"


def nnodes(p):
    """Mesh nodes: the trilinear grid, or the 20-node serendipity mesh."""
    if serendipity(p):
        from . import serendipity as sd
        return sd.nnodes(p)
    return (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)


def dofs_of(nodes, nc=3):
    return (nc * nodes[:, None] + np.arange(nc)[None, :]).reshape(-1)


def partition(p):
    """Subdomains of the px x py x pz box split with overlap O (Sec. 3.1)."""
    px, py, pz, O = p["partition"]
    n = (p["nx"], p["ny"], p["nz"])
    splits = [axis_split(n[0], px), axis_split(n[1], py), axis_split(n[2], pz)]
    subs = []
    for jz in range(pz):
        for jy in range(py):
            for jx in range(px):
                owned = (splits[0][jx], splits[1][jy], splits[2][jz])
                ebox = tuple((max(0, a - O), min(n[d], b + O))
                             for d, (a, b) in enumerate(owned))
                elo = [e[0] for e in ebox]
                ehi = [e[1] for e in ebox]
                if serendipity(p):
                    # nodes in doubled-grid coordinates: V_{h,0} keeps the edge
                    # midpoints of the first layer, drops those on the boundary
                    from . import serendipity as sd
                    neu = sd.box_nodes(p, [2 * e for e in elo], [2 * e for e in ehi])
                    dlo = [2 * elo[d] + (1 if elo[d] > 0 else 0) for d in range(3)]
                    dhi = [2 * ehi[d] - (1 if ehi[d] < n[d] else 0) for d in range(3)]
                    intn = sd.box_nodes(p, dlo, dhi)
                else:
                    neu = _box_nodes(p, elo, ehi)
                    ilo = [elo[d] + (1 if elo[d] > 0 else 0) for d in range(3)]
                    ihi = [ehi[d] - (1 if ehi[d] < n[d] else 0) for d in range(3)]
                    intn = _box_nodes(p, ilo, ihi)
                s = Subdomain(index=len(subs), owned=owned, ebox=ebox,
                              elems=_box_elems(p, elo, ehi),
                              neu_nodes=neu, int_nodes=intn)
                s.neu_dofs = dofs_of(neu, ncomp(p))
                s.int_dofs = dofs_of(intn, ncomp(p))
                subs.append(s)
    if p.get("pou", "standard") == "sarkis":
        _pou_sarkis(p, subs)
    else:
        _pou(p, subs)
    _overlap(p, subs)
    return subs


def node_layers(p):
    """(nnodes, 3) node positions in element layers along each axis: the grid
    index of a trilinear node, half the doubled-grid index of a serendipity
    node (edge midpoints sit half a layer in)."""
    if serendipity(p):
        from . import serendipity as sd
        ids, nn = sd.node_map(p["nx"], p["ny"], p["nz"])
        out = np.empty((nn, 3))
        I, J, K = np.nonzero(ids >= 0)
        out[ids[I, J, K]] = 0.5 * np.stack([I, J, K], axis=1)
        return out
    nnx, nny = p["nx"] + 1, p["ny"] + 1
    m = np.arange(nnodes(p))
    return np.stack([m % nnx, (m // nnx) % nny, m // (nnx * nny)], axis=1).astype(np.float64)


def _pou_sarkis(p, subs):
    """Sarkis's PoU (Sec. 3.2 and Sec. 3.3.1 offer it beside the standard one):
    X_j(n) = d_j(n) / sum_k d_k(n), d_j the distance from node n to the
    artificial boundary of Omega_j (the part of its boundary inside the
    domain), counted in element layers, so that the weight ramps linearly
    across the overlap on any element grading.  For a box and a point inside
    it the distance to a face is the distance to the face's plane, so d_j is
    the least over the artificial faces.  Zero on the artificial boundary and
    on global Dirichlet dofs; with one layer of overlap it equals the standard
    PoU."""
    n = (p["nx"], p["ny"], p["nz"])
    pos = node_layers(p)
    nc = ncomp(p)
    dist = []
    for s in subs:
        c = pos[s.neu_nodes]
        d = np.full(s.neu_nodes.size, np.inf)
        for a in range(3):
            lo, hi = s.ebox[a]
            if lo > 0:
                d = np.minimum(d, c[:, a] - lo)
            if hi < n[a]:
                d = np.minimum(d, hi - c[:, a])
        d[~np.isfinite(d)] = 1.0               # no artificial face: the whole domain
        dist.append(d)
    total = np.zeros(nnodes(p))
    for s, d in zip(subs, dist):
        total[s.neu_nodes] += d
    dir_mask = np.zeros(nc * nnodes(p), bool)
    dir_mask[np.asarray(p["dirichlet_dofs"], np.int64)] = True
    for s, d in zip(subs, dist):
        X = np.repeat(d / total[s.neu_nodes], nc)
        X[dir_mask[s.neu_dofs]] = 0.0
        s.X = X


def _pou(p, subs):
    """Standard PoU (Sec. 3.3.1): 1/multiplicity on V_{h,0}(Omega_j) dofs."""
    ndof = ncomp(p) * nnodes(p)
    mult = np.zeros(ndof)
    for s in subs:
        mult[s.int_dofs] += 1.0
    dir_mask = np.zeros(ndof, bool)
    dir_mask[np.asarray(p["dirichlet_dofs"], np.int64)] = True
    for s in subs:
        X = np.zeros(s.neu_dofs.size)
        inside = np.isin(s.neu_dofs, s.int_dofs)
        X[inside] = 1.0 / mult[s.neu_dofs[inside]]
        X[dir_mask[s.neu_dofs]] = 0.0
        s.X = X


def _overlap(p, subs):
    """Elements of Omega_j that also lie in another subdomain (Def. overlap)."""
    nel = p["nx"] * p["ny"] * p["nz"]
    count = np.zeros(nel, np.int64)
    for s in subs:
        count[s.elems] += 1
    for s in subs:
        s.ovl_elems = s.elems[count[s.elems] >= 2]


def pou_sum(p, subs):
    """sum_j R_j^T X_j R_j 1 (Def. Partition of Unity, applied to v = 1)."""
    ndof = ncomp(p) * nnodes(p)
    v = np.zeros(ndof)
    for s in subs:
        v[s.neu_dofs] += s.X
    return v
