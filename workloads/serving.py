"""Request streams for the serving loop (synthetic inputs).

A stream mixes laminated blocks of uneven size: the number of unknowns is
drawn log-uniformly between `dof_lo` and `dof_hi`, the block keeps the
8:4:3 proportions of the standard workloads, the stacking is a random
sequence of {0, +-45, 90} plies of two elements each, and the partition gives
subdomains of about 16 x 8 x 12 elements (the size of the 64x32x24 workload's
subdomains) with overlap 1 and the threshold mode rule capped at 20.  A share
of the requests repeats an earlier structure with a new load (another top
pressure), which the server can answer from resident factors.  Arrival times
are a Poisson process.
"""
from __future__ import annotations

import math

import numpy as np

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


def request_stream(n, seed=4, dof_lo=2e4, dof_hi=2e6, repeat_frac=0.25, rate_hz=None):
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
            p["top_pressure"] = float(rng.uniform(0.5, 2.0))
            p["name"] = f"{key}+load{i}"
        else:
            dofs = math.exp(rng.uniform(math.log(dof_lo), math.log(dof_hi)))
            key = f"s{i}"
            p = block_for_dofs(dofs, rng, key)
            p["top_pressure"] = float(rng.uniform(0.5, 2.0))
            structures.append((key, p))
        out.append((key, p, t))
        if rate_hz:
            t += float(rng.exponential(1.0 / rate_hz))
    return out


def dofs_of(p):
    return 3 * (p["nx"] + 1) * (p["ny"] + 1) * (p["nz"] + 1)
