"""Subdomain matrices of the GenEO set-up vs the oracle (Sec. 3.1, Sec. 3.3.2).

A_j = R_j A R_j^T, S_j = A_{Omega_j} - sigma X_j A_{Omega_j^o} X_j and
B_j = X_j A_{Omega_j^o} X_j are compared entry by entry (1e-12 relative to
max |entry|) after mapping the GPU's band numbering to global dofs.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import decomp, fem, geneo

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.mark.parametrize("name", ["tiny", "small", "c1"])
def test_local_matrices_match_oracle(pkg, name):
    p = workloads.config(name)
    s = pkg.GeneoSolver()
    s.assemble(p)
    try:
        s.setup(p, pkg.GENEO_FP64)
    except pkg.GeneoError:
        pass          # the matrices are checked even if a later set-up step fails
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    sigma = p["modes"]["shift"]
    for j, sd in enumerate(subs):
        Aj, gd = s.local_matrix(j, 0)
        ref = A[gd][:, gd].toarray()
        assert np.abs(Aj - ref).max() <= 1e-12 * np.abs(ref).max(), ("A_j", j)
        An, Ao = geneo.local_matrices(p, sd)
        Xd = sp.diags(sd.X)
        B = (Xd @ Ao @ Xd).toarray()
        Sref = An.toarray() - sigma * B
        # oracle local order = sorted global dofs of the closure of Omega_j
        Sg, gdn = s.local_matrix(j, 1)
        pos = np.searchsorted(sd.neu_dofs, gdn)
        assert np.array_equal(sd.neu_dofs[pos], gdn)
        Sr = Sref[np.ix_(pos, pos)]
        assert np.abs(Sg - Sr).max() <= 1e-12 * np.abs(Sr).max(), ("S_j", j)
        Bg, _ = s.local_matrix(j, 2)
        Br = B[np.ix_(pos, pos)]
        assert np.abs(Bg - Br).max() <= 1e-12 * max(np.abs(Br).max(), 1e-300), ("B_j", j)
        assert np.linalg.eigvalsh(Sg).min() > 0
    s.close()


@pytest.mark.parametrize("name,kind", [("tiny", 3), ("tiny", 4), ("c1", 3), ("c1", 4)])
def test_band_cholesky_matches_dense(pkg, name, kind):
    # The tile Cholesky (Sec. 3.3.3 exact local solves) against LAPACK on the
    # same matrix: off-diagonal blocks of L and inverted diagonal blocks.
    p = workloads.config(name)
    s = pkg.GeneoSolver()
    s.assemble(p)
    try:
        s.setup(p, pkg.GENEO_FP64)
    except pkg.GeneoError:
        pass
    for j in range(len(decomp.partition(p))):
        M, gd = s.local_matrix(j, kind - 3)
        F, _ = s.local_matrix(j, kind)
        L = np.linalg.cholesky(M)
        n = M.shape[0]
        nt = (n + 31) // 32
        for I in range(nt):
            r0, r1 = 32 * I, min(n, 32 * I + 32)
            Dinv = np.linalg.inv(L[r0:r1, r0:r1])
            assert np.abs(F[r0:r1, r0:r1] - Dinv).max() <= 1e-9 * np.abs(Dinv).max(), (j, I)
            if I > 0:
                off = F[r0:r1, :r0]
                ref = L[r0:r1, :r0]
                assert np.abs(off - ref).max() <= 1e-9 * np.abs(L).max(), (j, I)
    s.close()
