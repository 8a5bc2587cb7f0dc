"""Stress recovery on the GPU (geneo_element_stress) against the oracle.

Same element stiffnesses and the same centre strains on both sides: 1e-12
relative to the largest stress, for the displacement of a solve on layered
and wrinkled blocks and for a linear field (uniform strain), with host and
device arrays.
"""
import numpy as np
import pytest

import workloads
from oracle import fem

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.mark.parametrize("name,over", [("small", {}), ("c1", {}), ("small", {"wrinkle": (8.0, 3.0)})])
def test_stress_of_a_solution_matches_oracle(pkg, name, over):
    p = workloads.config(name, **over)
    s = pkg.GeneoSolver()
    s.assemble(p)
    s.setup(p)
    u, _ = s.solve(tol=1e-8)
    sig = s.element_stress(u)
    ref = fem.element_stresses(p, u)
    assert sig.shape == ref.shape
    assert np.abs(sig - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_stress_of_linear_field_on_device(pkg):
    import torch
    p = workloads.config("small")
    Z, Y, X = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    Xn = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    G = np.array([[0.01, -0.02, 0.005], [0.003, 0.02, -0.01], [0.004, 0.007, -0.015]])
    u = (Xn @ G.T).reshape(-1)
    s = pkg.GeneoSolver()
    s.assemble(p)
    sig = s.element_stress(torch.from_numpy(u).cuda()).cpu().numpy()
    ref = fem.element_stresses(p, u)
    assert np.abs(sig - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()
