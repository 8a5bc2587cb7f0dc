"""Randomised pins for the oracle's decomposition (Sec. 3.1-3.3.1).

Seeded random boxes, part counts up to the element count per axis (ragged
splits, parts of one element) and overlaps from 1 to 3 (wider than some
parts): each subdomain's closure and V_{h,0} node sets equal brute force on
the element-node incidence, and both partitions of unity sum to one on free
dofs, on the trilinear mesh and (for a few cases) on the 20-node mesh.
"""
import numpy as np
import pytest

from oracle import decomp, serendipity as sd
from workloads.laminate import make_block

from test_oracle_serendipity_geneo import _incidence


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny, nz = (int(v) for v in rng.integers(1, 7, size=3))
        parts = [int(rng.integers(1, m + 1)) for m in (nx, ny, nz)]
        O = int(rng.integers(1, 4))
        clamp = "x0" if rng.random() < 0.7 else "none"
        out.append((nx, ny, nz, parts, O, clamp))
    return out


@pytest.mark.parametrize("case", _cases(24, 11) + [(3, 2, 2, [3, 2, 2], 2, "x0")])
def test_random_partitions_trilinear(case):
    _check(*case, serend=False)


@pytest.mark.parametrize("case", _cases(5, 12))
def test_random_partitions_serendipity(case):
    _check(*case, serend=True)


def _check(nx, ny, nz, parts, O, clamp, serend):
    p = make_block(nx, ny, nz, [0.0, 90.0][: max(1, min(2, nz))], partition=(*parts, O), clamp=clamp)
    if serend:
        p = sd.problem(p) if clamp == "x0" else dict(p, element="serendipity",
                                                        dirichlet_dofs=np.zeros(0, np.int32),
                                                        dirichlet_values=np.zeros(0))
    en, adj = _incidence(p)
    for pou in ("standard", "sarkis"):
        q = dict(p, pou=pou)
        subs = decomp.partition(q)
        assert len(subs) == parts[0] * parts[1] * parts[2]
        covered = np.zeros(len(adj), bool)
        for s in subs:
            el = set(s.elems.tolist())
            assert s.neu_nodes.tolist() == sorted({int(n) for e in el for n in en[e]})
            assert s.int_nodes.tolist() == sorted(n for n in range(len(adj)) if adj[n] <= el)
            covered[s.int_nodes] = True
        assert covered.all()
        v = decomp.pou_sum(q, subs)
        free = np.ones(v.size, bool)
        free[np.asarray(q["dirichlet_dofs"], np.int64)] = False
        terms = np.zeros(v.size)
        for s in subs:
            terms[s.neu_dofs] += s.X > 0
        # a sum of k rounded weights is within k ulps of one
        assert np.all(np.abs(v[free] - 1.0) <= terms[free] * np.finfo(float).eps)
        assert np.all(v[~free] == 0.0)
