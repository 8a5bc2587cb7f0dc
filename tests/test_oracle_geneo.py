"""Pins for the oracle's GenEO eigenproblems and coarse space (Sec. 3.2-3.3)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import decomp, fem, geneo
import workloads

from test_oracle_fem import rigid_modes


def _floating_and_clamped(p):
    subs = decomp.partition(p)
    fl = [s for s in subs if s.ebox[0][0] > 0]
    cl = [s for s in subs if s.ebox[0][0] == 0]
    return subs, fl, cl


def _local(p, s):
    A, Ao = geneo.local_matrices(p, s)
    Xd = sp.diags(s.X)
    return A, (Xd @ Ao @ Xd).tocsr()


def test_floating_subdomain_has_six_rigid_zero_modes():
    p = workloads.config("c1")
    subs, fl, cl = _floating_and_clamped(p)
    s = fl[0]
    A, B = _local(p, s)
    lam, P = geneo.eigenpairs(A, B, 8, -0.01, "dense")
    assert np.all(np.abs(lam[:6]) < 1e-9)
    assert lam[6] > 1e-3
    nnx, nny = p["nx"] + 1, p["ny"] + 1
    n = s.neu_nodes
    X = np.stack([p["x"][n % nnx], p["y"][(n // nnx) % nny], p["z"][n // (nnx * nny)]], 1)
    R = rigid_modes(X)
    ang = sla.subspace_angles(P[:, :6], R)
    assert ang.max() < 1e-8
    # clamped subdomains have no zero modes
    A, B = _local(p, cl[0])
    lam, _ = geneo.eigenpairs(A, B, 3, -0.01, "dense")
    assert lam[0] > 1e-4


def test_eigenpairs_satisfy_the_generalised_problem():
    p = workloads.config("c1")
    subs = decomp.partition(p)
    for s in subs[:2]:
        A, B = _local(p, s)
        lam, P = geneo.eigenpairs(A, B, 10, -0.01, "dense")
        assert np.allclose(np.linalg.norm(P, axis=0), 1.0)
        res = A @ P - (B @ P) * lam[None, :]
        assert np.abs(res).max() < 1e-8 * abs(A).max()
        assert np.all(np.diff(lam) >= -1e-12)


def test_eigenvalues_independent_of_shift():
    p = workloads.config("c1")
    subs = decomp.partition(p)
    s = subs[1]
    A, B = _local(p, s)
    l1, _ = geneo.eigenpairs(A, B, 12, -1e-3, "dense")
    l2, _ = geneo.eigenpairs(A, B, 12, -1e-1, "dense")
    big = np.abs(l1) > 1e-6
    assert np.allclose(l1[big], l2[big], rtol=1e-8)
    assert np.all(np.abs(l2[~big]) < 1e-8)


def test_dense_and_arpack_agree():
    p = workloads.config("small")
    subs = decomp.partition(p)
    s = subs[0]
    A, B = _local(p, s)
    ld, Pd = geneo.eigenpairs(A, B, 8, -0.01, "dense")
    la, Pa = geneo.eigenpairs(A, B, 8, -0.01, "arpack")
    assert np.allclose(ld, la, rtol=1e-8, atol=1e-10)
    ang = sla.subspace_angles(Pd[:, :7], Pa[:, :7])
    assert ang.max() < 1e-6


def test_select_modes_rules():
    lam = np.array([0.0, 0.0, 0.1, 0.2, 0.2, 0.5, 3.0])
    assert geneo.select_modes(lam, 0, 0.3, 20) == 5
    assert geneo.select_modes(lam, 0, 0.3, 4) == 3      # cap cuts the 0.2 pair
    assert geneo.select_modes(lam, 0, 0.3, 2) == 2
    assert geneo.select_modes(lam, 0, 0.3, 1) == 0      # cut inside the zero pair
    assert geneo.select_modes(lam, 2, 0.0, 20) == 2
    assert geneo.select_modes(lam, 0, 10.0, 20) == 7
    # neighbours 1e-3 apart (relative) are distinct eigenvalues, not a cluster
    near = np.array([0.1, 0.2, 0.3, 0.3003, 0.9])
    assert geneo.select_modes(near, 0, 10.0, 3) == 3
    assert geneo.select_modes(near, 3, 0.0, 20) == 3


def test_cap_inside_a_degenerate_pair_drops_it():
    # The middle subdomain of a 3 x 3 in-plane split of a square isotropic block
    # is symmetric under quarter turns about z, so past its six rigid modes
    # GenEO eigenvalues come in equal pairs; a cap or a fixed count that would
    # split a pair keeps neither of the two (the kept span must be unique).
    import scipy.sparse as sp
    from workloads.laminate import RESIN, make_block
    p = make_block(6, 6, 2, [0.0], partition=(3, 3, 1, 1), clamp="none")
    p["materials"] = np.array([RESIN, RESIN], dtype=np.float64)
    p["x"], p["y"], p["z"] = np.linspace(0, 6, 7), np.linspace(0, 6, 7), np.linspace(0, 2, 3)
    subs = decomp.partition(p)
    mid = subs[4]
    A, Ao = geneo.local_matrices(p, mid)
    Xd = sp.diags(mid.X)
    lam, _ = geneo.eigenpairs(A, (Xd @ Ao @ Xd).tocsr(), 12, -0.01, "dense")
    assert abs(lam[8] - lam[9]) <= 1e-10 * lam[9] and lam[9] < lam[10] * (1 - 1e-3)
    Ag = fem.assemble_stiffness(p)
    for rule, want in (((0, 1e9, 9), 8), ((0, 1e9, 10), 10), ((9, 0.0, 20), 8)):
        p["modes"] = dict(fixed_modes=rule[0], threshold=rule[1], max_modes=rule[2], shift=-0.01)
        _, info = geneo.coarse_space(p, subs, Ag, "dense")
        assert info[4]["m"] == want, (rule, info[4]["m"])


def test_threshold_closed_form():
    p = workloads.config("c1")
    subs = decomp.partition(p)
    s = subs[0]            # elements [0, 5)^3: 2.5 x 2.5 x 5*0.115 mm, O = 1
    d = 0.5 * np.sqrt(2.5 ** 2 + 2.5 ** 2 + (5 * 0.115) ** 2)
    assert geneo.threshold(p, s) == pytest.approx(d / 0.115, rel=1e-12)


def test_coarse_matrix_block_sparsity_and_symmetry():
    # (A_H)_{il} = 0 when the supports of Phi_i and Phi_l do not overlap (Sec. 3.3.3).
    p = workloads.config("small", partition=(3, 2, 1, 1),
                         modes=dict(fixed_modes=7, threshold=0.0, max_modes=20, shift=-0.01))
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Z, info = geneo.coarse_space(p, subs, A)
    AH = geneo.coarse_matrix(A, Z)
    assert np.allclose(AH, AH.T, rtol=0, atol=1e-12 * np.abs(AH).max())
    assert all(d["m"] == 7 for d in info)
    owner = np.repeat(np.arange(len(subs)), [d["m"] for d in info])
    for i in range(AH.shape[0]):
        for l in range(AH.shape[1]):
            si, sl = subs[owner[i]], subs[owner[l]]
            if np.intersect1d(si.neu_nodes, sl.neu_nodes).size == 0:
                assert AH[i, l] == 0.0
    # subdomains 0 and 2 (x-blocks 0 and 2 of 3) do not overlap: a zero block exists
    assert np.any(AH == 0.0)
    sla.cholesky(AH, lower=True)
