"""The batched-solve workload: sizes, plies and partitions within its recipe."""
import math

import numpy as np

from workloads.batch import batch_blocks


def test_batch_recipe():
    blocks = batch_blocks(64, seed=3)
    els = np.array([p["nx"] * p["ny"] * p["nz"] for p in blocks])
    assert els.min() >= 0.6 * 8e3 and els.max() <= 1.4 * 1e5
    assert els.max() / els.min() > 4                     # uneven
    for p in blocks:
        px, py, pz, ov = p["partition"]
        assert ov == 1 and px * py * pz >= 2
        sub = math.ceil(p["nx"] / px) * math.ceil(p["ny"] / py) * math.ceil(p["nz"] / pz)
        assert sub <= 4000                               # bounded local band systems
        assert min(p["nx"] // px, p["ny"] // py, p["nz"] // pz) >= 2
        plies = np.unique(np.asarray(p["elem_theta"]).round(9))
        assert 1 <= len(plies) <= 4                      # angles from {0, +-45, 90}


def test_batch_is_seeded():
    a, b = batch_blocks(4, seed=3), batch_blocks(4, seed=3)
    for p, q in zip(a, b):
        assert (p["nx"], p["ny"], p["nz"], p["partition"]) == (q["nx"], q["ny"], q["nz"], q["partition"])
        assert np.array_equal(p["elem_theta"], q["elem_theta"])
