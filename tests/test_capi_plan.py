"""The library's subdomain plan (host-only, no GPU) against the oracle's
decomposition (Sec. 3.1), on the CPU.

For the standard workloads and seeded random boxes (ragged parts, parts of
one element, overlaps 1-3): every subdomain's element box, its interior node
box (V_{h,0}(Omega_j)) and its unknown counts match the oracle's element and
node sets; the band half-width of each factor, in 32-row tiles, covers the
widest coupling of two nodes of one element in the box's node numbering
(Omega_j's longest axis slowest), found by brute force; and a partition is refused
exactly when a part would be empty or a node would lie in the interiors of
more than four parts of one axis.
"""
import numpy as np
import pytest

import paper_1901_05188_gb300 as pkg
import workloads
from oracle import decomp
from workloads.laminate import make_block


def _plan(p):
    keep = []
    mesh = pkg.GeneoSolver.mesh_of(p, keep)
    return pkg.geneo_plan_subdomains(mesh, pkg.GeneoSolver.partition_of(p),
                                     pkg.GeneoSolver.unknowns_per_node(p))


def _box_nodes(p, lo, hi):
    nnx, nny = p["nx"] + 1, p["ny"] + 1
    i, j, k = (np.arange(lo[d], hi[d] + 1) for d in range(3))
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    return np.sort((I + nnx * (J + nny * K)).ravel())


def _half_band_dofs(ext, order, nc):
    """Brute force: number the box's nodes with the axes in `order` (fastest
    first) and take the widest index distance between two nodes of one element
    (offsets in {-1, 0, 1} per axis), in unknowns."""
    n = [int(ext[a]) for a in order]
    stride = [1, n[0], n[0] * n[1]]
    widest = 0
    for off in np.ndindex(3, 3, 3):
        d = [o - 1 for o in off]
        if any(d[a] != 0 and n[a] < 2 for a in range(3)):
            continue
        widest = max(widest, abs(sum(d[a] * stride[a] for a in range(3))))
    return nc * widest + nc - 1


def _check(p):
    plan = _plan(p)
    subs = decomp.partition(p)
    nc = decomp.ncomp(p)
    assert plan.shape == (len(subs), pkg.PLAN_INTS)
    for r, s in zip(plan, subs):
        assert [tuple(r[[d, 3 + d]]) for d in range(3)] == [tuple(e) for e in s.ebox]
        assert np.array_equal(_box_nodes(p, r[6:9], r[9:12]), s.int_nodes)
        assert np.array_equal(_box_nodes(p, r[0:3], r[3:6]), s.neu_nodes)
        assert r[12] == nc * s.int_nodes.size and r[14] == nc * s.neu_nodes.size
        # both boxes are numbered with Omega_j's axes by increasing node extent
        # (the longest axis slowest; ties in axis order)
        ext_neu = r[3:6] - r[0:3] + 1
        order = sorted(range(3), key=lambda a: (ext_neu[a], a))
        for n_dofs, w, ext in ((r[12], r[13], r[9:12] - r[6:9] + 1), (r[14], r[15], ext_neu)):
            nt = (n_dofs + 31) // 32
            assert w == min((_half_band_dofs(ext, order, nc) + 31) // 32, nt - 1)


@pytest.mark.parametrize("name", ["tiny", "small", "c1", "c2", "c3"])
def test_plan_of_the_workloads(name):
    _check(workloads.config(name))


def test_plan_of_a_darcy_block():
    from workloads.darcy import darcy_config
    _check(darcy_config("d-small"))


def _random(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ne = [int(v) for v in rng.integers(1, 9, size=3)]
        parts = [int(rng.integers(1, m + 1)) for m in ne]
        out.append((ne, parts, int(rng.integers(1, 4))))
    return out


@pytest.mark.parametrize("case", _random(40, 31))
def test_plan_of_random_partitions(case):
    ne, parts, O = case
    p = make_block(*ne, [0.0, 90.0][: min(2, ne[2])], partition=(*parts, O))
    # the refusal rule: more than four parts of one axis hold a node in their interior
    too_wide = False
    for n, k in zip(ne, parts):
        cnt = np.zeros(n + 1, int)
        for lo, hi in decomp.axis_split(n, k):
            elo, ehi = max(0, lo - O), min(n, hi + O)
            cnt[elo + (elo > 0): ehi - (ehi < n) + 1] += 1
        too_wide |= cnt.max() > 4
    if too_wide:
        with pytest.raises(pkg.GeneoError) as ei:
            _plan(p)
        assert ei.value.status == 1
    else:
        _check(p)


@pytest.mark.parametrize("name", ["small", "c1", "c2", "d-small"])
def test_setup_estimate_covers_the_planned_factors(name):
    # The host-only set-up estimate (used to admit requests by device memory)
    # must hold at least the band factor pools of the plan: per subdomain
    # nt (w + 1) tiles of 32 x 32 for L and for L^T, interior factors in the
    # chosen precision, the Neumann factors of the GenEO eigensolve in FP64.
    if name.startswith("d-"):
        from workloads.darcy import darcy_config
        p = darcy_config(name)
    else:
        p = workloads.config(name)
    plan = _plan(p)
    keep = []
    mesh = pkg.GeneoSolver.mesh_of(p, keep)
    tiles = lambda n, w: ((n + 31) // 32) * (w + 1) * 1024
    int_elems = sum(tiles(int(r[12]), int(r[13])) for r in plan)
    neu_elems = sum(tiles(int(r[14]), int(r[15])) for r in plan)
    for prec, size in ((pkg.GENEO_FP64, 8), (pkg.GENEO_MIXED_FP32, 4)):
        _, setup = pkg.geneo_estimate_workspace_bytes(mesh, pkg.GeneoSolver.partition_of(p),
                                                      pkg.GeneoSolver.modes_of(p), prec,
                                                      pkg.GeneoSolver.unknowns_per_node(p))
        assert setup >= 2 * int_elems * size + 2 * neu_elems * 8, (prec, setup)


@pytest.mark.parametrize("case", _random(10, 32))
def test_plan_of_random_darcy_partitions(case):
    # one unknown per node: the same boxes, unknown counts and band widths in
    # scalar unknowns
    from workloads.darcy import make_darcy
    ne, parts, O = case
    p = make_darcy(*ne, seed=1, partition=(*parts, O))
    try:
        _check(p)
    except pkg.GeneoError as e:
        assert e.status == 1
        for n, k in zip(ne, parts):
            cnt = np.zeros(n + 1, int)
            for lo, hi in decomp.axis_split(n, k):
                elo, ehi = max(0, lo - O), min(n, hi + O)
                cnt[elo + (elo > 0): ehi - (ehi < n) + 1] += 1
            if cnt.max() > 4:
                break
        else:
            raise
