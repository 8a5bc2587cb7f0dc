"""Pins for the oracle's scalar Darcy problem (the SPE10 application, eqn:Darcy).

Element matrix: symmetric, constants in its kernel, and the energy of a
linear field g.x equals V sum_d K_d g_d^2 exactly (2x2x2 Gauss is exact for
the Q1 bilinear terms on boxes).  Global matrix: exactly one zero eigenvalue
(the constants) before the Dirichlet condition, SPD after.  Patch test: with
homogeneous K a linear field on the whole boundary and f = 0 is reproduced
at every node.  Load: the consistent source integrates to f times the volume.
Solvers: PCG with the GenEO preconditioner equals a dense direct solve; on a
partition with a floating subdomain its only zero-energy GenEO mode is the
constant, which is also the ZEM mode; iterations order AS > GenEO.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import darcy, decomp, geneo, solver
from workloads.darcy import darcy_config, make_darcy


def test_element_matrix_closed_forms():
    kd = (3.0, 0.5, 0.02)
    h = (2.0, 1.5, 0.25)
    K = darcy.element_matrix(kd, *h)
    assert np.allclose(K, K.T, atol=1e-14 * abs(K).max())
    assert np.abs(K.sum(axis=1)).max() <= 1e-13 * abs(K).max()
    corners = np.array([(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]) * np.array(h)
    g = np.array([0.7, -1.3, 2.1])
    u = corners @ g
    vol = h[0] * h[1] * h[2]
    assert abs(u @ K @ u - vol * np.dot(kd, g * g)) <= 1e-12 * vol * np.dot(kd, g * g)


def test_global_matrix_kernel_is_the_constants():
    p = darcy_config("d-tiny")
    A = darcy.assemble_matrix(p).toarray()
    assert np.allclose(A, A.T, atol=1e-13 * abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert abs(ev[0]) <= 1e-10 * ev[-1] and ev[1] > 1e-12 * ev[-1]
    assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-12 * abs(A).max()
    Ac, _ = darcy.assemble_system(p)
    np.linalg.cholesky(Ac.toarray())


def test_patch_test_linear_field():
    p = make_darcy(5, 4, 3, seed=1)
    p["perm"][:] = np.array([2.0, 0.7, 0.05])          # homogeneous anisotropic K
    p["source"] = 0.0
    nnx, nny, nnz = p["nx"] + 1, p["ny"] + 1, p["nz"] + 1
    Zc, Yc, Xc = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    g = np.array([0.01, -0.03, 0.2])
    u_ex = (np.stack([Xc.ravel(), Yc.ravel(), Zc.ravel()], 1) @ g) + 1.5
    I, J, K = np.meshgrid(np.arange(nnx), np.arange(nny), np.arange(nnz), indexing="ij")
    bnd = (I == 0) | (I == nnx - 1) | (J == 0) | (J == nny - 1) | (K == 0) | (K == nnz - 1)
    nodes = np.sort((I + nnx * (J + nny * K))[bnd]).astype(np.int32)
    p["dirichlet_dofs"] = nodes
    p["dirichlet_values"] = u_ex[nodes]
    A, b = darcy.assemble_system(p)
    u = sp.linalg.spsolve(A.tocsc(), b)
    assert np.abs(u - u_ex).max() <= 1e-12 * np.abs(u_ex).max()


def test_source_integrates_to_volume():
    p = darcy_config("d-small")
    vol = p["x"][-1] * p["y"][-1] * p["z"][-1]
    assert abs(darcy.load(p).sum() - p["source"] * vol) <= 1e-12 * vol


def test_pcg_matches_direct_solve():
    p = darcy_config("d-tiny")
    A, b = darcy.assemble_system(p)
    u_d = np.linalg.solve(A.toarray(), b)
    r = solver.solve(p, precond="geneo", tol=1e-12)
    assert np.linalg.norm(r["u"] - u_d) <= 1e-9 * np.linalg.norm(u_d)


def test_floating_subdomain_zero_mode_is_constant():
    p = darcy_config("d-tiny", partition=(1, 1, 2, 1))    # the upper half floats
    subs = decomp.partition(p)
    top = [s for s in subs if s.ebox[2][0] > 0][0]
    A, Ao = geneo.local_matrices(p, top)
    Xd = sp.diags(top.X)
    lam, P = geneo.eigenpairs(A, (Xd @ Ao @ Xd).tocsr(), 4, -0.01, "dense")
    assert abs(lam[0]) < 1e-9 and lam[1] > 1e-6
    one = np.ones((P.shape[0], 1))
    assert sla.subspace_angles(P[:, :1], one).max() < 1e-8
    Az, _ = darcy.assemble_system(p)
    Z, info = geneo.zem_space(p, subs, Az)
    assert [d["m"] for d in info] == [0, 1]


def test_iterations_as_greater_than_geneo():
    p = darcy_config("d-small")
    it = {k: solver.solve(p, precond=k, tol=1e-8)["iterations"] for k in ("as", "geneo")}
    assert it["as"] > it["geneo"], it


def test_global_energy_of_linear_field_heterogeneous():
    # On the unconstrained matrix the energy of a linear field g.x is
    # sum_e V_e sum_d K_{e,d} g_d^2 exactly, for a per-cell K and a graded mesh
    # with different spacings per axis: it ties every cell to its own K
    # components and its own edge lengths.
    p = make_darcy(5, 4, 3, seed=2)
    p["x"] = np.cumsum(np.r_[0.0, [1.0, 1.5, 0.7, 2.0, 1.1]])
    p["y"] = np.cumsum(np.r_[0.0, [0.4, 0.9, 0.6, 1.3]])
    p["z"] = np.cumsum(np.r_[0.0, [0.2, 0.05, 0.3]])
    Zc, Yc, Xc = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    g = np.array([0.8, -1.7, 2.3])
    u = np.stack([Xc.ravel(), Yc.ravel(), Zc.ravel()], 1) @ g
    nx, ny = p["nx"], p["ny"]
    e = np.arange(nx * ny * p["nz"])
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    vol = np.diff(p["x"])[ex] * np.diff(p["y"])[ey] * np.diff(p["z"])[ez]
    K = np.random.default_rng(9).uniform(0.1, 10.0, size=(e.size, 3))   # Kx, Ky, Kz all distinct
    p["perm"] = K
    A = darcy.assemble_matrix(p)
    want = np.sum(vol * (K @ (g * g)))
    assert abs(u @ (A @ u) - want) <= 1e-12 * want
