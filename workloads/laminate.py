"""Laminated cantilever blocks on tensor-product hex meshes (synthetic inputs).

Units: mm, N, MPa.  Node n = i + (nx+1)*(j + (ny+1)*k), dof = 3*n + c.
Element e = ex + nx*(ey + ny*ez).

Material constants are the paper's (Section 5): orthotropic plies with
E11=162 GPa, E22=E33=10 GPa, G12=G13=5.2 GPa, G23=3.5 GPa, nu12=nu13=0.35,
nu23=0.5, ply thickness 0.23 mm; isotropic resin interlayers E=10 GPa,
nu=0.35, thickness 0.02 mm.  A material is the 9-vector
(E1, E2, E3, G12, G13, G23, nu12, nu13, nu23); an isotropic material repeats
E and nu and uses G = E / (2 (1 + nu)).

The layer-to-element rule, the in-plane element size (0.5 mm), the ply-angle
convention and the wrinkle shape are readings stated where the paper is silent
(Section 5 gives only the stacking sequences and thicknesses).
"""
from __future__ import annotations

import math

import numpy as np

# (E1, E2, E3, G12, G13, G23, nu12, nu13, nu23) in MPa
PLY = (162000.0, 10000.0, 10000.0, 5200.0, 5200.0, 3500.0, 0.35, 0.35, 0.5)
_E_RESIN, _NU_RESIN = 10000.0, 0.35
_G_RESIN = _E_RESIN / (2.0 * (1.0 + _NU_RESIN))
RESIN = (_E_RESIN, _E_RESIN, _E_RESIN, _G_RESIN, _G_RESIN, _G_RESIN,
         _NU_RESIN, _NU_RESIN, _NU_RESIN)

PLY_T = 0.23     # mm
RESIN_T = 0.02   # mm
H_INPLANE = 0.5  # mm, in-plane element edge


def layer_cake(nz, ply_angles_deg, resin_between, ply_t=PLY_T, resin_t=RESIN_T):
    """Split nz element layers over a stack of plies (and optional resin).

    Layers bottom-up: ply0, [resin], ply1, [resin], ... .  Each resin layer gets
    one element; the remaining elements go to the plies as evenly as possible,
    the lowest plies taking one extra when the split is uneven.

    Returns (z_nodes[nz+1], elem_layer_kind[nz] (0 ply, 1 resin),
    elem_layer_angle_deg[nz], elem_layer_index[nz]).
    """
    n_ply = len(ply_angles_deg)
    n_resin = n_ply - 1 if resin_between else 0
    n_ply_el = nz - n_resin
    if n_ply_el < n_ply:
        raise ValueError("nz too small for the stack")
    base, extra = divmod(n_ply_el, n_ply)
    dz, kind, ang, lay = [], [], [], []
    layer = 0
    for p in range(n_ply):
        ne = base + (1 if p < extra else 0)
        for _ in range(ne):
            dz.append(ply_t / ne)
            kind.append(0)
            ang.append(float(ply_angles_deg[p]))
            lay.append(layer)
        layer += 1
        if resin_between and p < n_ply - 1:
            dz.append(resin_t)
            kind.append(1)
            ang.append(0.0)
            lay.append(layer)
            layer += 1
    z = np.concatenate([[0.0], np.cumsum(dz)])
    return z, np.array(kind, np.int32), np.array(ang), np.array(lay, np.int32)


def make_block(nx, ny, nz, ply_angles_deg, resin_between=False, h=H_INPLANE,
               pressure=1.0, partition=(2, 2, 2, 1), modes=None,
               wrinkle=None, contrast=None, clamp="x0", name="block"):
    """Build one laminated cantilever block problem as plain arrays.

    wrinkle: None or (amplitude_deg, width_in_elements): out-of-plane fibre
      angle phi(x, y) = A * exp(-r^2 / (2 w^2)) about the block centre,
      evaluated at element centroids, applied to every ply.
    contrast: None or factor c: materials of odd layers get E and G scaled by
      c (isotropic copies of the resin scaled), used for contrast sweeps.
    clamp: "x0" clamps u=0 at x=0 (the paper's cantilever);
      "none" leaves the block unconstrained.
    """
    z, kind, ang, lay = layer_cake(nz, ply_angles_deg, resin_between)
    x = np.arange(nx + 1, dtype=np.float64) * h
    y = np.arange(ny + 1, dtype=np.float64) * h
    nel = nx * ny * nz
    ez = np.repeat(np.arange(nz), nx * ny)
    ey = np.tile(np.repeat(np.arange(ny), nx), nz)
    ex = np.tile(np.arange(nx), ny * nz)
    mats = [PLY, RESIN]
    elem_mat = kind[ez].astype(np.int32)
    if contrast is not None:
        c = float(contrast)
        scaled = tuple(v * c for v in PLY[:6]) + PLY[6:]
        mats.append(scaled)
        odd = (lay[ez] % 2 == 1) & (elem_mat == 0)
        elem_mat = np.where(odd, 2, elem_mat).astype(np.int32)
        scaled_r = tuple(v * c for v in RESIN[:6]) + RESIN[6:]
        mats.append(scaled_r)
        oddr = (lay[ez] % 2 == 1) & (kind[ez] == 1)
        elem_mat = np.where(oddr, 3, elem_mat).astype(np.int32)
    theta = np.deg2rad(ang[ez]).astype(np.float64)
    theta = np.where(kind[ez] == 1, 0.0, theta)
    phi = np.zeros(nel)
    if wrinkle is not None:
        amp, width = wrinkle
        xc = 0.5 * (x[ex] + x[ex + 1])
        yc = 0.5 * (y[ey] + y[ey + 1])
        w = width * h
        r2 = (xc - 0.5 * x[-1]) ** 2 + (yc - 0.5 * y[-1]) ** 2
        phi = np.deg2rad(amp) * np.exp(-r2 / (2.0 * w * w))
        phi = np.where(kind[ez] == 1, 0.0, phi)
    nnx, nny, nnz = nx + 1, ny + 1, nz + 1
    if clamp == "x0":
        nodes = np.array([i + nnx * (j + nny * k)
                          for k in range(nnz) for j in range(nny) for i in (0,)],
                         dtype=np.int64)
        dofs = (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)
        dofs = np.sort(dofs).astype(np.int32)
    elif clamp == "none":
        dofs = np.zeros(0, np.int32)
    else:
        raise ValueError(clamp)
    if modes is None:
        modes = dict(fixed_modes=6, threshold=0.0, max_modes=20, shift=-0.01)
    return dict(
        name=name, nx=nx, ny=ny, nz=nz, x=x, y=y, z=z,
        materials=np.array(mats, dtype=np.float64),
        elem_mat=elem_mat, elem_theta=theta, elem_phi=phi,
        dirichlet_dofs=dofs, dirichlet_values=np.zeros(dofs.size),
        top_pressure=float(pressure), nodal_load=None,
        partition=tuple(int(v) for v in partition), modes=dict(modes),
    )


CONFIG_NAMES = ("c1", "c2", "c3", "tiny", "small")


def config(name, **over):
    """The standard synthetic workloads.

    c1: 8x8x8 block, 4 plies [0/90/90/0] (2 elements each), 2x2x2 subdomains,
        overlap 1, 6 GenEO modes per subdomain, FP64 PCG to 1e-8.
    c2: 64x32x24 block, 12 plies drawn from {0, +-45, 90} (seed 1) with 11
        one-element resin interlayers, 4x4x2 subdomains, overlap 1,
        threshold rule with a cap of 20 modes.
    c3: 128x64x48 block, 24 plies (seed 2), 2 elements each, Gaussian fibre
        wrinkle (8 degrees, width 10 elements), 8x4x4 subdomains, cap 20.
    tiny: 4x3x2 block, 2 plies, 2x1x1 subdomains (fast CPU pins).
    small: 12x8x6 block, 3 plies + 2 resin, 3x2x1 subdomains.
    """
    thr = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)
    if name == "c1":
        kw = dict(nx=8, ny=8, nz=8, ply_angles_deg=[0, 90, 90, 0],
                  partition=(2, 2, 2, 1),
                  modes=dict(fixed_modes=6, threshold=0.0, max_modes=20,
                             shift=-0.01))
    elif name == "c2":
        rng = np.random.default_rng(1)
        ang = rng.choice([0.0, 45.0, -45.0, 90.0], size=12)
        kw = dict(nx=64, ny=32, nz=24, ply_angles_deg=ang, resin_between=True,
                  partition=(4, 4, 2, 1), modes=thr)
    elif name == "c3":
        rng = np.random.default_rng(2)
        ang = rng.choice([0.0, 45.0, -45.0, 90.0], size=24)
        kw = dict(nx=128, ny=64, nz=48, ply_angles_deg=ang,
                  partition=(8, 4, 4, 1), modes=thr, wrinkle=(8.0, 10.0))
    elif name == "tiny":
        kw = dict(nx=4, ny=3, nz=2, ply_angles_deg=[30, -60],
                  partition=(2, 1, 1, 1),
                  modes=dict(fixed_modes=6, threshold=0.0, max_modes=20,
                             shift=-0.01))
    elif name == "small":
        kw = dict(nx=12, ny=8, nz=6, ply_angles_deg=[0, 45, 90],
                  resin_between=True, partition=(3, 2, 1, 1), modes=thr)
    else:
        raise KeyError(name)
    kw.update(over)
    kw.setdefault("name", name)
    return make_block(**kw)


def problem_summary(p):
    nn = (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)
    return dict(name=p["name"], elements=p["nx"] * p["ny"] * p["nz"],
                nodes=nn, dofs=3 * nn, partition=list(p["partition"]),
                modes=dict(p["modes"]))
