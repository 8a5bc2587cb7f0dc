"""Pins against the figures the paper prints for its flat-plate example
(Sec. 5, Example 1; Table 1), stored in tests/golden/example1_plate.json.

Geometry: twelve plies of the stacking sequence with eleven resin interlayers
add up to the printed thickness, and the base mesh (20 x 5 elements in plane,
two per ply and one per interlayer) has the printed element count.  The
printed unknown count equals three unknowns on every vertex of that mesh: the
trilinear mesh of the oracle gives it exactly, the 20-node mesh would give
far more (its count is checked against the closed form instead).  Table 1:
the ZEM coarse space has six rigid modes per subdomain without a clamped
dof, and the printed dimensions for 4, 8, 16 and 32 subdomains are met by
in-plane grids 2x2, 8x1, 8x2 and 8x4 on the clamped plate (the table does not
state the grids; N - dim/6 = 2, 1, 2, 4 subdomains touch the clamp).
"""
import json
import os

import numpy as np
import pytest

from oracle import decomp, fem, geneo, serendipity as sd
from workloads.laminate import make_block

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "example1_plate.json")))
GRIDS = {4: (2, 2), 8: (8, 1), 16: (8, 2), 32: (8, 4)}


def _plate(partition=(1, 1, 1, 1)):
    m = GOLD["base_mesh"]
    nply = len(GOLD["stacking_deg"])
    nz = m["elements_per_ply"] * nply + m["elements_per_resin"] * GOLD["resin_layers"]
    p = make_block(m["nx"], m["ny"], nz, GOLD["stacking_deg"], resin_between=True,
                   partition=partition)
    lx, ly = GOLD["plate_mm"]
    p["x"] = np.linspace(0.0, lx, m["nx"] + 1)
    p["y"] = np.linspace(0.0, ly, m["ny"] + 1)
    return p


def test_thickness_and_layer_map():
    p = _plate()
    assert abs(p["z"][-1] - GOLD["total_thickness_mm"]) <= 1e-12
    dz = np.diff(p["z"])
    nres = GOLD["resin_layers"]
    assert np.sum(np.isclose(dz, GOLD["resin_thickness_mm"], rtol=0, atol=1e-14)) == nres
    assert np.allclose(dz[dz > 0.05], GOLD["ply_thickness_mm"] / 2, rtol=0, atol=1e-14)


def test_base_mesh_counts():
    p = _plate()
    assert p["nx"] * p["ny"] * p["nz"] == GOLD["base_elements"]
    A = fem.assemble_stiffness(p)
    assert A.shape[0] == GOLD["base_dof"]
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ser = 3 * sd.nnodes(p)
    assert ser == 3 * ((nx + 1) * (ny + 1) * (nz + 1) + nx * (ny + 1) * (nz + 1)
                       + ny * (nx + 1) * (nz + 1) + nz * (nx + 1) * (ny + 1))
    assert ser != GOLD["base_dof"]


@pytest.mark.parametrize("n", sorted(GRIDS))
def test_table1_zem_dimension(n):
    px, py = GRIDS[n]
    p = _plate((px, py, 1, 1))
    A, _ = fem.assemble_system(p)
    subs = decomp.partition(p)
    assert len(subs) == n
    Z, info = geneo.zem_space(p, subs, A)
    assert Z.shape[1] == GOLD["table1_zem_dim"][str(n)]
    touching = sum(1 for s in subs if s.ebox[0][0] == 0)
    assert [d["m"] for d in info].count(0) == touching
