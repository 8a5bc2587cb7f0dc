"""Pins for the oracle's Sarkis partition of unity (Sec. 3.2; Sec. 3.3.1).

X_j(n) = d_j(n) / sum_k d_k(n) with d_j the distance, in element layers, from
node n to the artificial boundary of Omega_j.  Pins: it sums to one on free
dofs (and is zero on clamped ones) for overlaps 2 and 3 on both meshes; with
one layer of overlap it is the standard multiplicity PoU exactly, also on a
graded laminate split through its thickness; across an overlap of two layers
it ramps 1, 3/4, 1/2, 1/4, 0 (and through the edge midpoints of the 20-node
mesh at the quarter steps between); and, as the paper reports, GenEO-PCG
needs at most one iteration more or less than with the standard PoU.
"""
import numpy as np
import pytest

import workloads
from oracle import decomp, serendipity as sd, solver
from workloads.laminate import make_block


def _free(p, v):
    free = np.ones(v.size, bool)
    free[p["dirichlet_dofs"]] = False
    return free


@pytest.mark.parametrize("overlap", [2, 3])
@pytest.mark.parametrize("element", ["trilinear", "serendipity"])
def test_sums_to_one(overlap, element):
    p = make_block(9, 7, 6, [0.0, 90.0, 45.0], resin_between=True, partition=(3, 2, 1, overlap))
    p = sd.problem(p) if element == "serendipity" else p
    p["pou"] = "sarkis"
    subs = decomp.partition(p)
    v = decomp.pou_sum(p, subs)
    free = _free(p, v)
    assert np.abs(v[free] - 1.0).max() <= 4e-16
    assert np.all(v[~free] == 0.0)
    for s in subs:
        assert np.all((s.X >= 0.0) & (s.X <= 1.0))
        art = ~np.isin(s.neu_dofs, s.int_dofs)
        assert np.all(s.X[art] == 0.0)


def test_one_layer_is_the_standard_pou():
    # graded element sizes through the thickness (plies and resin) and a split in z
    p = make_block(6, 4, 7, [0.0, 90.0, 0.0, 90.0], resin_between=True, partition=(2, 2, 2, 1))
    std = decomp.partition(p)
    sar = decomp.partition(dict(p, pou="sarkis"))
    for a, b in zip(std, sar):
        assert np.array_equal(a.X, b.X)


def test_linear_ramp_across_two_layers():
    p = make_block(8, 2, 2, [0.0, 90.0], partition=(2, 1, 1, 2), clamp="none")
    p["pou"] = "sarkis"
    s1, s2 = decomp.partition(p)            # Omega_1 = [0, 6], Omega_2 = [2, 8] in x layers
    nnx = p["nx"] + 1
    for s, want in ((s1, {2: 1.0, 3: 0.75, 4: 0.5, 5: 0.25, 6: 0.0}),
                    (s2, {2: 0.0, 3: 0.25, 4: 0.5, 5: 0.75, 6: 1.0})):
        i = s.neu_nodes % nnx
        Xn = s.X.reshape(-1, 3)[:, 0]
        for k, w in want.items():
            assert np.all(Xn[i == k] == w), (s.index, k)
    q = sd.problem(make_block(8, 2, 2, [0.0, 90.0], partition=(2, 1, 1, 2), clamp="none"))
    q["pou"] = "sarkis"
    t1, _ = decomp.partition(q)
    ids, _ = sd.node_map(8, 2, 2)
    X1 = np.zeros(ids.max() + 1)
    X1[t1.neu_nodes] = t1.X.reshape(-1, 3)[:, 0]
    for di, w in ((7, 0.625), (9, 0.375), (11, 0.125)):        # edge midpoints along x
        col = ids[di, 0::2, 0::2]
        assert np.all(X1[col[col >= 0]] == w)


def test_iterations_close_to_the_standard_pou():
    p = workloads.config("small")
    p["partition"] = tuple(p["partition"][:3]) + (2,)
    it = [solver.solve(dict(p, pou=k), precond="geneo", tol=1e-8)["iterations"]
          for k in ("standard", "sarkis")]
    assert abs(it[0] - it[1]) <= 1, it
