"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP64 path): assembly entries 1e-12 relative to max |A|, the load
exactly up to rounding (1e-13); one preconditioner application 1e-9 relative
(different but exact factorisations of the same SPD matrices); GenEO
eigenvalues 1e-7 relative (Lanczos vs dense/ARPACK); coarse span principal
angles within the Ritz acceptance's bound (residual 1e-5 theta over the gap to the
first dropped mode, at least 1e-5); solutions 1e-6 relative L2 with iteration counts within +-2.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import decomp, fem, geneo, krylov, solver as osolver

from gpu_common import bsr_to_csr, rel, require_gpu, span_tolerance

pytestmark = pytest.mark.gpu

CASES = ["tiny", "small", "c1"]


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


def make(pkg, p):
    s = pkg.GeneoSolver()
    s.assemble(p)
    return s


@pytest.mark.parametrize("name", CASES)
def test_assembly_matches_oracle(pkg, name):
    p = workloads.config(name)
    s = make(pkg, p)
    rp, col, val, b = s.system()
    A = bsr_to_csr(rp, col, val, s.nnode)
    Ao, bo = fem.assemble_system(p)
    D = (A - Ao).toarray() if s.ndof < 4000 else (A - Ao)
    scale = abs(Ao).max()
    assert abs(D).max() <= 1e-12 * scale
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()
    # structure: 27-point pattern, sorted columns
    assert rp[-1] == s.nnzb and np.all(np.diff(rp) <= 27)
    s.close()


def test_assembly_wrinkled_anisotropic_block(pkg):
    p = workloads.config("small", wrinkle=(8.0, 3.0))
    s = make(pkg, p)
    rp, col, val, b = s.system()
    A = bsr_to_csr(rp, col, val, s.nnode)
    Ao, bo = fem.assemble_system(p)
    assert abs(A - Ao).max() <= 1e-12 * abs(Ao).max()
    s.close()


def test_nonhomogeneous_dirichlet_patch(pkg):
    # Patch test through the GPU assembly: linear field on the boundary.
    p = workloads.config("small", ply_angles_deg=[30, 30, 30], resin_between=False)
    p["elem_theta"][:] = np.deg2rad(30.0)
    p["elem_mat"][:] = 0
    p["top_pressure"] = 0.0
    nnx, nny, nnz = p["nx"] + 1, p["ny"] + 1, p["nz"] + 1
    Zc, Yc, Xc = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    X = np.stack([Xc.ravel(), Yc.ravel(), Zc.ravel()], axis=1)
    G = np.array([[0.01, -0.02, 0.005], [0.003, 0.02, -0.01], [0.004, 0.007, -0.015]])
    u_ex = (X @ G.T).reshape(-1)
    I, J, K = np.meshgrid(np.arange(nnx), np.arange(nny), np.arange(nnz), indexing="ij")
    bnd = ((I == 0) | (I == nnx - 1) | (J == 0) | (J == nny - 1) | (K == 0) | (K == nnz - 1))
    bn = np.sort((I + nnx * (J + nny * K))[bnd])
    dofs = (3 * bn[:, None] + np.arange(3)).reshape(-1)
    p["dirichlet_dofs"] = dofs.astype(np.int32)
    p["dirichlet_values"] = u_ex[dofs]
    s = make(pkg, p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, pkg.GENEO_COARSE_NONE)
    u, st = s.solve(tol=1e-13, max_it=3000)
    assert np.abs(u - u_ex).max() <= 1e-9 * np.abs(u_ex).max()
    s.close()


@pytest.mark.parametrize("name", CASES)
def test_spmv_matches_oracle(pkg, name):
    p = workloads.config(name)
    s = make(pkg, p)
    Ao, _ = fem.assemble_system(p)
    x = np.random.default_rng(0).normal(size=s.ndof)
    assert rel(s.spmv(x), Ao @ x) <= 1e-13
    s.close()


@pytest.mark.parametrize("name", CASES)
def test_one_level_schwarz_apply_matches_oracle(pkg, name):
    p = workloads.config(name)
    s = make(pkg, p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, pkg.GENEO_COARSE_NONE)
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    M = krylov.OneLevelAS(A, subs)
    r = np.random.default_rng(1).normal(size=s.ndof)
    r[p["dirichlet_dofs"]] = 0.0
    assert rel(s.apply_preconditioner(r), M(r)) <= 1e-9
    s.close()


def test_pou_weighted_one_level_apply(pkg):
    p = workloads.config("small")
    s = make(pkg, p)
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS_POU, pkg.GENEO_COARSE_NONE)
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    M = krylov.OneLevelAS(A, subs, weight="pou")
    r = np.random.default_rng(2).normal(size=s.ndof)
    r[p["dirichlet_dofs"]] = 0.0
    assert rel(s.apply_preconditioner(r), M(r)) <= 1e-9
    s.close()


@pytest.mark.parametrize("name", ["tiny", "small", "c1"])
def test_geneo_eigenvalues_and_span(pkg, name):
    p = workloads.config(name)
    s = make(pkg, p)
    s.setup(p, pkg.GENEO_FP64)
    modes, lam, nh = s.coarse_info()
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Zo, info = geneo.coarse_space(p, subs, A, "dense")
    assert list(modes) == [d["m"] for d in info]
    for j, d in enumerate(info):
        lo = d["lam"]
        k = min(len(lo), lam.shape[1])
        fin = np.isfinite(lo[:k])
        # all kept modes and the first dropped one agree
        kk = min(int(modes[j]) + 1, int(fin.sum()))
        ref = lo[:kk]
        got = lam[j, :kk]
        tol = 1e-7 * np.maximum(np.abs(ref), 1e-2)
        assert np.all(np.abs(got - ref) <= tol), (j, got, ref)
    Phi, AH = s.coarse()
    assert Phi.shape[1] == nh == Zo.shape[1]
    if nh:
        ang = sla.subspace_angles(Phi, Zo.toarray())
        assert ang.max() <= span_tolerance([d["m"] for d in info], [d["lam"] for d in info],
                                           p["modes"]["shift"])
        # A_H = Phi^T A Phi (Sec. 3.3.3) for the GPU's own basis
        AHr = Phi.T @ (A @ Phi)
        assert np.abs(AH - AHr).max() <= 1e-10 * np.abs(AHr).max()
    s.close()


@pytest.mark.parametrize("name", ["small", "c1"])
def test_two_level_apply_matches_oracle(pkg, name):
    p = workloads.config(name)
    s = make(pkg, p)
    s.setup(p, pkg.GENEO_FP64)
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Zo, _ = geneo.coarse_space(p, subs, A, "dense")
    M = krylov.TwoLevelAS(A, subs, Zo)
    r = np.random.default_rng(3).normal(size=s.ndof)
    r[p["dirichlet_dofs"]] = 0.0
    assert rel(s.apply_preconditioner(r), M(r)) <= 1e-7
    s.close()


@pytest.mark.parametrize("name,pre", [("tiny", "geneo"), ("small", "geneo"), ("c1", "geneo"),
                                      ("c1", "as"), ("small", "as")])
def test_fp64_solve_matches_oracle(pkg, name, pre):
    p = workloads.config(name)
    s = make(pkg, p)
    coarse = pkg.GENEO_COARSE_GENEO if pre == "geneo" else pkg.GENEO_COARSE_NONE
    s.setup(p, pkg.GENEO_FP64, pkg.GENEO_AS, coarse)
    u, st = s.solve(tol=1e-8, max_it=2000)
    ref = osolver.solve(p, precond=pre, tol=1e-8)
    assert rel(u, ref["u"]) <= 1e-6
    assert abs(st["iterations"] - ref["iterations"]) <= 2, (st["iterations"], ref["iterations"])
    assert st["rel_res_true"] <= 2e-8
    if ref["kappa"]:
        assert st["kappa_est"] == pytest.approx(ref["kappa"], rel=0.05)
    s.close()


@pytest.mark.parametrize("name", ["small", "c1"])
def test_mixed_precision_solve_matches_oracle(pkg, name):
    p = workloads.config(name)
    s = make(pkg, p)
    s.setup(p, pkg.GENEO_MIXED_FP32)
    u, st = s.solve(tol=1e-10, max_it=2000)
    ref = osolver.solve(p, precond="geneo", tol=1e-10)
    assert st["flexible"] == 1
    assert rel(u, ref["u"]) <= 1e-6
    assert st["rel_res_true"] <= 2e-10
    s.close()


def test_unpreconditioned_is_rejected_before_setup(pkg):
    p = workloads.config("tiny")
    s = make(pkg, p)
    with pytest.raises(pkg.GeneoError):
        s.solve()
    s.close()
