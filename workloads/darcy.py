"""Synthetic layered permeability for the scalar Darcy problem (inputs only).

Stand-in for the SPE10 permeability data, which is not available here: a
tensor-product grid of cells 20 x 10 x 2 (ft) like SPE10's, log10 Kx drawn
from a Gaussian field with mean -1 and standard deviation 1.5, correlated
over about 20 cells in-plane and 2 cells vertically (the field is white noise
smoothed by separable Gaussian filters and rescaled), with every third layer
made a channelised layer (a meandering high-permeability channel of width 4
cells cut into a low-permeability background) so that the contrast reaches
about 1e6; Ky = Kx and Kz = 0.1 Kx.  The pressure is fixed to zero on the
bottom face z = 0 and the source is f = 1.
"""
from __future__ import annotations

import numpy as np

CELL = (20.0, 10.0, 2.0)   # ft, the SPE10 cell size


def _smooth(a, axis, ell):
    """Circular Gaussian smoothing of `a` along `axis` with length ell (cells)."""
    n = a.shape[axis]
    k = np.fft.fftfreq(n)
    filt = np.exp(-0.5 * (2.0 * np.pi * k * ell) ** 2)
    shape = [1] * a.ndim
    shape[axis] = n
    return np.real(np.fft.ifft(np.fft.fft(a, axis=axis) * filt.reshape(shape), axis=axis))


def permeability(nx, ny, nz, seed=5, mean=-1.0, std=1.5, ell_xy=20.0, ell_z=2.0):
    """(nel, 3) array of (Kx, Ky, Kz), element e = ex + nx (ey + ny ez)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((nz, ny, nx))
    g = _smooth(_smooth(_smooth(g, 2, ell_xy), 1, ell_xy), 0, ell_z)
    sd = g.std()
    g = (g - g.mean()) / sd if sd > 0 else np.zeros_like(g)     # one cell: the mean field
    logk = mean + std * g
    # channelised layers: every third layer, a meandering channel of width 4
    xs = np.arange(nx)
    for k in range(1, nz, 3):
        centre = nx / 2 + 0.3 * nx * np.sin(2 * np.pi * np.arange(ny) / max(ny, 1) + k)
        inside = np.abs(xs[None, :] - centre[:, None]) < 2.0
        logk[k] = np.where(inside, 2.0, -4.0)
    kx = 10.0 ** logk.reshape(-1)
    return np.stack([kx, kx, 0.1 * kx], axis=1)


def make_darcy(nx, ny, nz, seed=5, partition=(2, 2, 1, 1), modes=None, source=1.0,
               name="darcy"):
    """A Darcy problem dict (kind "darcy", one unknown per node)."""
    x = np.arange(nx + 1) * CELL[0]
    y = np.arange(ny + 1) * CELL[1]
    z = np.arange(nz + 1) * CELL[2]
    nnx, nny = nx + 1, ny + 1
    bottom = np.arange(nnx * nny, dtype=np.int32)          # nodes of the face z = 0
    if modes is None:
        modes = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)
    return dict(kind="darcy", name=name, nx=nx, ny=ny, nz=nz, x=x, y=y, z=z,
                perm=permeability(nx, ny, nz, seed), dirichlet_dofs=bottom,
                dirichlet_values=np.zeros(bottom.size), source=float(source),
                nodal_load=None, partition=tuple(int(v) for v in partition),
                modes=dict(modes))


def darcy_config(name, **over):
    """d-tiny: 6x5x4, 2x1x1 subdomains; d-small: 16x12x9, 2x2x1 (the paper decomposes
    SPE10 in-plane, full height); d-large: 36x64x24, 1x2x1 (30,525 interior unknowns per
    subdomain, more than a local vector held whole in shared memory allows); d-spe10: the
    SPE10 grid 60x220x85, 6x18x1 (subdomains of 10 x 12 x 85 cells)."""
    if name == "d-tiny":
        kw = dict(nx=6, ny=5, nz=4, partition=(2, 1, 1, 1))
    elif name == "d-small":
        kw = dict(nx=16, ny=12, nz=9, partition=(2, 2, 1, 1))
    elif name == "d-large":
        kw = dict(nx=36, ny=64, nz=24, partition=(1, 2, 1, 1))
    elif name == "d-spe10":
        kw = dict(nx=60, ny=220, nz=85, partition=(6, 18, 1, 1))
    else:
        raise KeyError(name)
    kw.update(over)
    kw.setdefault("name", name)
    return make_darcy(**kw)
