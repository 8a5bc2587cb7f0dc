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


def bsr_to_csr(rp, col, val, n, nc=3):
    """Expand the library's nc x nc block BSR into a scipy CSR matrix."""
    rows = np.repeat(np.arange(n), np.diff(rp))
    R = (nc * rows[:, None, None] + np.arange(nc)[None, :, None]).repeat(nc, axis=2)
    Cc = (nc * col[:, None, None] + np.arange(nc)[None, None, :]).repeat(nc, axis=1)
    return sp.csr_matrix((val.reshape(-1), (R.reshape(-1), Cc.reshape(-1))), shape=(nc * n, nc * n))


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
