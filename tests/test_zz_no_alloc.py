"""The allocation-free SpMV + dot entry point against the regular one and the oracle.

geneo_spmv_dot_noalloc serves callers that cannot allocate device memory (a
fixed device-memory budget handed out by a host framework, a real-time loop
that must stay out of the CUDA allocator, a plug-in given only someone else's
buffers); its scratch is a static device array.  Two calls in a row (the
second reuses the scratch left by the first) must give the same y as
geneo_spmv, the same y as the FP64 oracle's assembled A times x, and the same
x . y as the host dot product, within the SpMV parity tolerance used
elsewhere (1e-13 relative).  A hand-built BSR whose rows hold 64 blocks checks
rows far longer than the library's own 27-block rows against a numpy product.
Collected last (file name) so a stop-at-first-failure run has already run
every other test.
"""
import numpy as np
import pytest

import workloads

from gpu_common import bsr_to_csr, require_gpu

pytestmark = pytest.mark.gpu


def _call(pkg, torch, dev, n, d_rp, d_col, d_val, x):
    d_x = torch.as_tensor(x, device=dev)
    d_y = torch.full((3 * n,), np.nan, dtype=torch.float64, device=dev)
    d_xy = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    pkg.geneo_spmv_dot_noalloc(n, d_rp, d_col, d_val, d_x, d_y, d_xy, stream or None)
    torch.cuda.synchronize(dev)
    return d_y.cpu().numpy(), float(d_xy.cpu()[0])


def test_noalloc_spmv_dot_matches_regular_entry_point_and_oracle():
    pkg = require_gpu()
    import torch
    from oracle import fem
    p = workloads.config("c1")
    A_oracle = fem.assemble_system(p)[0].tocsr()
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
        y, xy = _call(pkg, torch, dev, s.nnode, d_rp, d_col, d_val, x)
        assert np.linalg.norm(y - y_ref) <= 1e-13 * np.linalg.norm(y_ref), call
        y_or = A_oracle @ x
        assert np.linalg.norm(y - y_or) <= 1e-13 * np.linalg.norm(y_or), call
        xy_ref = float(x @ y_ref)
        assert abs(xy - xy_ref) <= 1e-12 * abs(xy_ref), call
    s.close()


def test_noalloc_long_rows_against_numpy():
    pkg = require_gpu()
    import torch
    rng = np.random.default_rng(11)
    n, per_row = 200, 64                       # 576 entries per row, > 512
    col = np.concatenate([np.sort(rng.choice(n, per_row, replace=False))
                          for _ in range(n)]).astype(np.int32)
    rp = (per_row * np.arange(n + 1)).astype(np.int32)
    val = rng.normal(size=(n * per_row, 3, 3))
    A = bsr_to_csr(rp, col, val, n)
    dev = torch.device("cuda", torch.cuda.current_device())
    d_rp = torch.as_tensor(rp, device=dev)
    d_col = torch.as_tensor(col, device=dev)
    d_val = torch.as_tensor(val.reshape(-1), device=dev)
    for call in range(2):
        x = rng.normal(size=3 * n)
        y, xy = _call(pkg, torch, dev, n, d_rp, d_col, d_val, x)
        y_ref = A @ x
        assert np.linalg.norm(y - y_ref) <= 1e-13 * np.linalg.norm(y_ref), call
        assert abs(xy - float(x @ y_ref)) <= 1e-12 * np.abs(x * y_ref).sum(), call


def test_noalloc_rejects_oversized_and_in_place_input():
    pkg = require_gpu()
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.zeros(4, dtype=torch.float64, device=dev)
    ti = torch.zeros(4, dtype=torch.int32, device=dev)
    with pytest.raises(pkg.GeneoError) as e:
        pkg.geneo_spmv_dot_noalloc(524288 + 1, ti, ti, t, t, t, t)
    assert e.value.status == 2
    assert "524288" in str(e.value)
    v = torch.zeros(6, dtype=torch.float64, device=dev)
    rp = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    col = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    val = torch.zeros(18, dtype=torch.float64, device=dev)
    xy = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.GeneoError) as e:
        pkg.geneo_spmv_dot_noalloc(2, rp, col, val, v, v, xy)
    assert e.value.status == 1
    assert "overlap" in str(e.value)
