"""Batches of uneven laminated blocks for the batched-solve workload.

Each block (seeded) draws its element count log-uniformly in [8e3, 1e5], a ply
count uniformly in 4..24 with one or two elements per ply through the
thickness, an in-plane aspect nx / ny uniformly in [1, 3], a stacking sequence
from {0, +-45, 90}, and a subdomain count log-uniformly in [2, 64]; the count
is raised where a subdomain would hold more than `max_sub_elems` elements
(which bounds the local band systems), and split over x and y in proportion
to the block (z too for thick blocks).  Overlap 1, the threshold mode rule
with at most 20 modes per subdomain.
"""
from __future__ import annotations

import math

import numpy as np

from .laminate import make_block

MODES = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)


def batch_block(rng, name, el_lo=8e3, el_hi=1e5, max_sub_elems=4000):
    n_el = math.exp(rng.uniform(math.log(el_lo), math.log(el_hi)))
    nplies = int(rng.integers(4, 25))
    nz = nplies * int(rng.integers(1, 3))
    aspect = rng.uniform(1.0, 3.0)
    area = n_el / nz
    nx = max(4, int(round(math.sqrt(area * aspect))))
    ny = max(4, int(round(area / nx)))
    ang = rng.choice([0.0, 45.0, -45.0, 90.0], size=nplies)
    parts = int(round(math.exp(rng.uniform(math.log(2), math.log(64)))))
    parts = max(parts, math.ceil(nx * ny * nz / max_sub_elems))
    pz = 2 if (nz >= 8 and parts >= 8) else 1
    pxy = math.ceil(parts / pz)
    px = max(1, min(nx // 2, int(round(math.sqrt(pxy * nx / ny)))))
    py = max(1, min(ny // 2, math.ceil(pxy / px)))
    # a subdomain may still exceed the bound when an axis is capped at 2 elements per part
    while math.ceil(nx / px) * math.ceil(ny / py) * math.ceil(nz / pz) > max_sub_elems:
        if px < nx // 2:
            px += 1
        elif py < ny // 2:
            py += 1
        elif pz < nz // 2:
            pz += 1
        else:
            break
    return make_block(nx, ny, nz, ang, partition=(px, py, pz, 1), modes=dict(MODES), name=name)


def batch_blocks(n, seed=3, **kw):
    """n blocks of the batch (the first n of the seeded sequence)."""
    rng = np.random.default_rng(seed)
    return [batch_block(rng, f"b{i}", **kw) for i in range(n)]
