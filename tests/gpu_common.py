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


def check_against_golden(u, st, gold, coarse=None, u_tol=1e-6):
    """Compare a GPU solve with an oracle summary written by make_golden.py:
    the displacement at the stored samples (relative L2), the norm of every
    consecutive chunk of dofs (largest deviation relative to the largest
    chunk norm, so every dof is covered), the norm of u, the iteration count
    (+-2) and, given coarse = (modes, lambdas, n_coarse), the coarse
    dimension, the per-subdomain mode counts and eigenvalues (1e-7 relative,
    floor 1e-2)."""
    ref = np.asarray(gold["u_samples"])
    us = u[::gold["sample_stride"]][:ref.size]
    err = np.linalg.norm(us - ref) / np.linalg.norm(ref)
    assert err <= u_tol, ("samples", err)
    assert abs(np.linalg.norm(u) - gold["u_norm"]) <= u_tol * gold["u_norm"]
    if "u_chunk_norms" in gold:
        ch = int(gold["chunk"])
        cn = np.sqrt(np.add.reduceat(u * u, np.arange(0, u.size, ch)))
        rc = np.asarray(gold["u_chunk_norms"])
        assert cn.size == rc.size
        dev = np.max(np.abs(cn - rc)) / np.max(rc)
        assert dev <= u_tol, ("chunk norms", dev)
    assert abs(st["iterations"] - gold["iterations"]) <= 2, (st["iterations"], gold["iterations"])
    if coarse is not None:
        modes, lam, nh = coarse
        assert nh == gold["n_coarse"]
        assert list(modes) == gold["modes"]
        for j, lref in enumerate(gold["lambdas"]):
            lref = np.asarray(lref)
            k = min(len(lref), modes[j] + 1)
            got = lam[j, :k]
            assert np.all(np.abs(got - lref[:k]) <= 1e-7 * np.maximum(np.abs(lref[:k]), 1e-2)), j
    return err


# The set-up's default Ritz acceptance: residual <= EIG_TOL * theta
# (theta = mu = 1 / (lambda - sigma), the shift-invert eigenvalue).
EIG_TOL = 1e-5


def span_tolerance(modes, lambdas, shift, eig_tol=EIG_TOL):
    """Largest angle the Ritz acceptance allows between the kept eigenvectors
    and the exact ones: eig_tol * mu_k over the gap to the first dropped
    mode, maximised over subdomains and kept modes (at least 1e-5), from the
    oracle's eigenvalues."""
    worst = 1e-5
    for m, lam in zip(modes, lambdas):
        lam = np.asarray(lam, dtype=float)
        if 0 < m < lam.size and np.isfinite(lam[m]):
            mu = 1.0 / (lam - shift)
            worst = max(worst, max(eig_tol * mu[k] / (mu[k] - mu[m]) for k in range(m)))
    return worst
