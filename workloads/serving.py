"""Request streams for the serving loop (synthetic inputs).

A stream mixes laminated blocks of uneven size: the number of unknowns is
drawn log-uniformly between `dof_lo` and `dof_hi`, the block keeps the
8:4:3 proportions of the standard workloads, the stacking is a random
sequence of {0, +-45, 90} plies of two elements each, and the partition gives
subdomains of about 16 x 8 x 12 elements (the size of the 64x32x24 workload's
subdomains) with overlap 1 and the threshold mode rule capped at 20.  A share
of the requests repeats an earlier structure with a new load (another top
pressure), which the server can answer from resident factors.  With
`darcy_frac` > 0 that share of the new structures is instead a scalar Darcy
block (one unknown per node) with the layered permeability of
`workloads.darcy`, the same log-uniform unknown count, SPE10-like 60:220:85
proportions and an in-plane decomposition over the full height (about 10 x 12
cells per subdomain: narrow bands, so cheap band factorisations);
with `darcy_grid="spe10"` every new Darcy structure is instead the full
60 x 220 x 85-cell SPE10 grid (1,159,366 unknowns, 6 x 18 subdomains) with its
own seeded permeability.  Arrival times are a Poisson process.
"""
from __future__ import annotations

import math

import numpy as np

from .darcy import make_darcy
from .laminate import make_block

SUB_ELEMS = (16, 8, 12)


def block_for_dofs(dofs, rng, name):
    """A laminate block with about `dofs` unknowns in 8:4:3 proportions."""
    a = max((dofs / 288.0) ** (1.0 / 3.0), 1.0)
    nx, ny = max(4, int(round(8 * a))), max(2, int(round(4 * a)))
    nplies = max(2, int(round(3 * a)) // 2)
    nz = 2 * nplies
    ang = rng.choice([0.0, 45.0, -45.0, 90.0], size=nplies)
    part = tuple(max(1, min(n // 2, int(math.ceil(n / s))))
                 for n, s in zip((nx, ny, nz), SUB_ELEMS)) + (1,)
    modes = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)
    return make_block(nx, ny, nz, ang, partition=part, modes=modes, name=name)


def darcy_for_dofs(dofs, rng, name):
    """A Darcy block with about `dofs` unknowns in SPE10's 60:220:85 proportions."""
    a = max((dofs / (60.0 * 220.0 * 85.0)) ** (1.0 / 3.0), 0.05)
    nx, ny, nz = max(4, round(60 * a)), max(4, round(220 * a)), max(3, round(85 * a))
    part = (max(1, min(nx // 2, math.ceil(nx / 10))), max(1, min(ny // 2, math.ceil(ny / 12))), 1, 1)
    return make_darcy(nx, ny, nz, seed=int(rng.integers(1 << 30)), partition=part, name=name)


def request_stream(n, seed=4, dof_lo=2e4, dof_hi=2e6, repeat_frac=0.25, rate_hz=None,
                   darcy_frac=0.0, darcy_grid=None):
    """n requests as (key, problem, arrival_offset_s).

    Without a rate every offset is 0 (a burst); with one, offsets are the
    cumulative sums of exponential gaps of mean 1/rate_hz.
    """
    rng = np.random.default_rng(seed)
    structures = []
    out = []
    t = 0.0
    for i in range(n):
        if structures and rng.random() < repeat_frac:
            key, base = structures[int(rng.integers(len(structures)))]
            p = dict(base)
            p["source" if p.get("kind") == "darcy" else "top_pressure"] = float(rng.uniform(0.5, 2.0))
            p["name"] = f"{key}+load{i}"
        else:
            dofs = math.exp(rng.uniform(math.log(dof_lo), math.log(dof_hi)))
            key = f"s{i}"
            if darcy_frac > 0 and rng.random() < darcy_frac:
                if darcy_grid == "spe10":
                    p = make_darcy(60, 220, 85, seed=int(rng.integers(1 << 30)),
                                   partition=(6, 18, 1, 1), name=key)
                else:
                    p = darcy_for_dofs(dofs, rng, key)
                p["source"] = float(rng.uniform(0.5, 2.0))
            else:
                p = block_for_dofs(dofs, rng, key)
                p["top_pressure"] = float(rng.uniform(0.5, 2.0))
            structures.append((key, p))
        out.append((key, p, t))
        if rate_hz:
            t += float(rng.exponential(1.0 / rate_hz))
    return out


def dofs_of(p):
    nc = 1 if p.get("kind") == "darcy" else 3
    return nc * (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)
