"""Shared helpers for the GPU parity tests (imported by tests marked gpu)."""
import numpy as np
import pytest
import scipy.sparse as sp


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05188_gb300 as pkg
    pkg.load(build_if_missing=True)
    return pkg


def bsr_to_csr(rp, col, val, n):
    """Expand the library's 3x3 BSR into a scipy CSR matrix."""
    nb = len(col)
    rows = np.repeat(np.arange(n), np.diff(rp))
    R = (3 * rows[:, None, None] + np.arange(3)[None, :, None]).repeat(3, axis=2)
    Cc = (3 * col[:, None, None] + np.arange(3)[None, None, :]).repeat(3, axis=1)
    return sp.csr_matrix((val.reshape(-1), (R.reshape(-1), Cc.reshape(-1))), shape=(3 * n, 3 * n))


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
