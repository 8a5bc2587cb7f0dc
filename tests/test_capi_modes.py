"""The library's GenEO mode rules (host-only) against the oracle's, on the CPU
(Sec. 3.2).

Default thresholds: per subdomain equal to the oracle's diam / width reading
(1e-14 relative) on the workloads, the Example 1 plate and graded random
meshes.  Mode selection: on seeded random ascending eigenvalue lists with
zero clusters, near-ties, exact pairs and infinities, under fixed counts,
thresholds and caps, the same mode count as the oracle's rule.
"""
import numpy as np
import pytest

import paper_1901_05188_gb300 as pkg
import workloads
from oracle import decomp, geneo
from workloads.laminate import make_block


def _taus(p):
    keep = []
    mesh = pkg.GeneoSolver.mesh_of(p, keep)
    return pkg.geneo_default_thresholds(mesh, pkg.GeneoSolver.partition_of(p))


def _graded(seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) for v in rng.integers(2, 9, size=3))
    parts = [int(rng.integers(1, max(1, m // 2) + 1)) for m in (nx, ny, nz)]
    p = make_block(nx, ny, nz, [0.0, 90.0][: min(2, nz)], partition=(*parts, int(rng.integers(1, 3))))
    for k, n in (("x", nx), ("y", ny), ("z", nz)):
        p[k] = np.concatenate([[0.0], np.cumsum(rng.uniform(0.02, 3.0, size=n))])
    return p


@pytest.mark.parametrize("p", [workloads.config(n) for n in ("tiny", "small", "c1", "c2")]
                         + [_graded(s) for s in range(12)])
def test_default_thresholds(p):
    subs = decomp.partition(p)
    got = _taus(p)
    want = np.array([geneo.threshold(p, s) for s in subs])
    assert np.allclose(got, want, rtol=1e-14, atol=0)


def _lists(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        k = int(rng.integers(1, 30))
        lam = np.sort(rng.exponential(0.5, size=k))
        nz = int(rng.integers(0, min(7, k) + 1))
        lam[:nz] = rng.uniform(-1e-13, 1e-13, size=nz)            # a zero cluster
        lam = np.sort(lam)
        for _ in range(int(rng.integers(0, 3))):                     # exact and near pairs
            i = int(rng.integers(0, k - 1)) if k > 1 else 0
            if k > 1:
                lam[i + 1] = lam[i] * (1 + rng.choice([0.0, 5e-7, 2e-6, 1e-3]))
        lam = np.sort(lam)
        ninf = int(rng.integers(0, 3))
        if ninf:
            lam[-ninf:] = np.inf
        out.append(lam)
    return out


@pytest.mark.parametrize("seed", range(4))
def test_select_modes(seed):
    rng = np.random.default_rng(100 + seed)
    for lam in _lists(60, seed):
        fixed = int(rng.choice([0, 0, 3, 6, 9]))
        cap = int(rng.integers(1, 25))
        tau = float(rng.choice([0.0, 0.05, 0.3, 1.0, 10.0]))
        modes = pkg.geneo_modes(fixed, 0.0, cap, -0.01)
        assert pkg.geneo_select_modes(lam, modes, tau) == geneo.select_modes(lam, fixed, tau, cap), \
            (lam, fixed, tau, cap)


def test_select_modes_refuses_bad_caps():
    lam = np.array([0.0, 0.1, 0.2, 0.3])
    for fixed, cap in ((0, 0), (0, -3), (0, 33), (-1, 20), (33, 20)):
        with pytest.raises(pkg.GeneoError) as e:
            pkg.geneo_select_modes(lam, pkg.geneo_modes(fixed, 0.0, cap, -0.01), 1.0)
        assert e.value.status == 1, (fixed, cap)
    # a fixed count ignores the cap
    assert pkg.geneo_select_modes(lam, pkg.geneo_modes(2, 0.0, 0, -0.01), 1.0) == 2
