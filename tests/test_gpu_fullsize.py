"""Full-size workload (64x32x24 laminate, 160,875 dofs, 4x4x2 subdomains) on
the GPU in the launch configuration bench.py times, against the oracle's
stored summary (tests/golden/c2_oracle.json, written by make_golden.py from
oracle/ only): iteration count within +-2, GenEO mode counts and eigenvalues
(1e-7 relative), coarse dimension, and the displacement at the stored sample
of dofs within 1e-6 relative L2 (FP64) / 1e-6 (mixed precision)."""
import json
import os

import numpy as np
import pytest

import workloads

from gpu_common import check_against_golden, require_gpu

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c2_oracle.json")


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.fixture(scope="module")
def gold():
    return json.load(open(GOLD))


def samples(u, g):
    return u[::g["sample_stride"]][:len(g["u_samples"])]


def test_c2_fp64_matches_oracle(pkg, gold):
    p = workloads.config("c2")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_FP64)
    u, st = s.solve(tol=1e-8, max_it=2000)
    modes, lam, nh = s.coarse_info()
    assert nh == gold["n_coarse"]
    assert list(modes) == gold["modes"]
    for j, ref in enumerate(gold["lambdas"]):
        ref = np.asarray(ref)
        k = min(len(ref), modes[j] + 1)
        got = lam[j, :k]
        assert np.all(np.abs(got - ref[:k]) <= 1e-7 * np.maximum(np.abs(ref[:k]), 1e-2)), j
    assert abs(st["iterations"] - gold["iterations"]) <= 2
    ref = np.asarray(gold["u_samples"])
    assert np.linalg.norm(samples(u, gold) - ref) <= 1e-6 * np.linalg.norm(ref)
    assert abs(np.linalg.norm(u) - gold["u_norm"]) <= 1e-6 * gold["u_norm"]
    check_against_golden(u, st, gold)
    assert st["rel_res_true"] <= 2e-8
    s.close()


def test_c2_mixed_precision_matches_oracle(pkg, gold):
    p = workloads.config("c2")
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p, pkg.GENEO_MIXED_FP32)
    u, st = s.solve(tol=1e-8, max_it=2000)
    ref = np.asarray(gold["u_samples"])
    err = np.linalg.norm(samples(u, gold) - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err
    check_against_golden(u, st, gold, s.coarse_info())
    assert st["rel_res_true"] <= 2e-8
    assert st["flexible"] == 1
    s.close()
