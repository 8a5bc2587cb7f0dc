"""Pins for the oracle's overlapping decomposition and PoU (Sec. 3.1-3.3.1)."""
import numpy as np
import pytest

from oracle import decomp
import workloads


@pytest.mark.parametrize("name", ["tiny", "small", "c1"])
def test_pou_identity_exact(name):
    # Def. Partition of Unity applied to v = 1: sum_j R_j^T X_j R_j 1 = 1 on free dofs.
    p = workloads.config(name)
    subs = decomp.partition(p)
    v = decomp.pou_sum(p, subs)
    free = np.ones(v.size, bool)
    free[p["dirichlet_dofs"]] = False
    assert np.array_equal(v[free], np.ones(free.sum()))
    assert np.all(v[~free] == 0.0)


def test_pou_identity_outside_overlap():
    # Sec. 3.2: restricted to Omega_j minus the overlap, Xi_j is the identity.
    p = workloads.config("small", clamp="none")
    subs = decomp.partition(p)
    for s in subs:
        others = set()
        for t in subs:
            if t is not s:
                others.update(t.neu_nodes.tolist())
        own = np.array([n not in others for n in s.neu_nodes])
        Xn = s.X.reshape(-1, 3)
        assert np.all(Xn[own] == 1.0)
        # zero on the artificial boundary
        art = ~np.isin(s.neu_nodes, s.int_nodes)
        assert np.all(Xn[art] == 0.0)


def test_owned_boxes_tile_the_mesh_and_overlap_elements():
    p = workloads.config("tiny")        # 4x3x2, split 2x1x1, overlap 1
    subs = decomp.partition(p)
    owned = []
    for s in subs:
        (a0, a1), (b0, b1), (c0, c1) = s.owned
        owned += [ex + 4 * (ey + 3 * ez) for ez in range(c0, c1)
                  for ey in range(b0, b1) for ex in range(a0, a1)]
    assert sorted(owned) == list(range(24))
    # Omega_0 = x-elements [0, 3), Omega_1 = [1, 4): overlap is x-elements 1 and 2
    for s in subs:
        ex = s.ovl_elems % 4
        assert sorted(set(ex.tolist())) == [1, 2]
        assert s.ovl_elems.size == 2 * 3 * 2


def test_subdomain_sizes_match_closed_form():
    # Interior subdomains of c2 (64x32x24, 4x4x2, O=1): closure 19x11x14 nodes,
    # V_{h,0} part 17x9x13 nodes.
    p = workloads.config("c2")
    subs = decomp.partition(p)
    assert max(s.neu_dofs.size for s in subs) == 3 * 19 * 11 * 14
    assert max(s.int_dofs.size for s in subs) == 3 * 17 * 9 * 13
    assert len(subs) == 32
