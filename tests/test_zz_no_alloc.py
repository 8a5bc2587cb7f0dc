"""The allocation-free SpMV + dot entry point against the regular one.

geneo_spmv_dot_noalloc serves callers that cannot allocate device memory; its
scratch is a static device array.  Two calls in a row (the second reuses the
scratch left by the first) must give the same y as geneo_spmv and the same
x . y as the host dot product of x and that y, within the SpMV parity
tolerance used elsewhere (1e-13 relative).  Collected last (file name) so a
stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

import workloads

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_spmv_dot_matches_regular_entry_point():
    pkg = require_gpu()
    import torch
    p = workloads.config("c1")
    s = pkg.GeneoSolver()
    s.assemble(p)
    rp, col, val, b = s.system()
    dev = torch.device("cuda", torch.cuda.current_device())
    d_rp = torch.as_tensor(rp, device=dev)
    d_col = torch.as_tensor(col, device=dev)
    d_val = torch.as_tensor(val.reshape(-1), device=dev)
    rng = np.random.default_rng(7)
    for call in range(2):
        x = rng.normal(size=s.ndof)
        y_ref = s.spmv(x)                      # existing entry point
        d_x = torch.as_tensor(x, device=dev)
        d_y = torch.full((s.ndof,), np.nan, dtype=torch.float64, device=dev)
        d_xy = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev).cuda_stream
        pkg.geneo_spmv_dot_noalloc(s.nnode, d_rp, d_col, d_val, d_x, d_y, d_xy,
                                   stream or None)
        torch.cuda.synchronize(dev)
        y = d_y.cpu().numpy()
        assert np.linalg.norm(y - y_ref) <= 1e-13 * np.linalg.norm(y_ref), call
        xy_ref = float(x @ y_ref)
        assert abs(float(d_xy.cpu()[0]) - xy_ref) <= 1e-12 * abs(xy_ref), call
    s.close()


def test_noalloc_rejects_oversized_input():
    pkg = require_gpu()
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.zeros(4, dtype=torch.float64, device=dev)
    ti = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(pkg.GeneoError) as e:
        pkg.geneo_spmv_dot_noalloc(524288 + 1, ti, ti, t, t, t, t)
    assert e.value.status == 2
    assert "524288" in str(e.value)
