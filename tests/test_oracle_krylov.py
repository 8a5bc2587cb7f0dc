"""Pins for the oracle's Schwarz preconditioners and (F)PCG (Sec. 3.1)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import decomp, fem, geneo, krylov, solver
import workloads


def dense_op(M, n):
    return np.column_stack([M(e) for e in np.eye(n)])


def test_cg_terminates_in_k_steps_for_k_distinct_eigenvalues():
    # Exact-arithmetic property of CG: k distinct eigenvalues -> k iterations.
    d = np.repeat([1.0, 3.0, 10.0, 25.0], 50)
    A = sp.diags(d).tocsr()
    b = np.random.default_rng(0).normal(size=d.size)
    x, info = krylov.pcg(A, b, tol=1e-12, maxit=50)
    assert info["iterations"] == 4
    assert np.allclose(x, b / d, rtol=1e-10)


@pytest.mark.parametrize("pre", ["none", "as", "geneo"])
def test_pcg_matches_dense_direct_solve(pre):
    p = workloads.config("c1")
    r = solver.solve(p, precond=pre, tol=1e-12)
    u_direct = np.linalg.solve(r["A"].toarray(), r["b"])
    assert np.linalg.norm(r["u"] - u_direct) <= 1e-10 * np.linalg.norm(u_direct)


def test_single_subdomain_is_exact_in_one_iteration():
    p = workloads.config("small", partition=(1, 1, 1, 1),
                         modes=dict(fixed_modes=2, threshold=0.0, max_modes=20, shift=-0.01))
    for pre in ("as", "geneo"):
        r = solver.solve(p, precond=pre, tol=1e-8)
        assert r["iterations"] == 1


def test_zero_modes_reduces_to_one_level():
    p = workloads.config("small")
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    M1 = krylov.OneLevelAS(A, subs)
    M2 = krylov.TwoLevelAS(A, subs, sp.csc_matrix((A.shape[0], 0)))
    r = np.random.default_rng(1).normal(size=A.shape[0])
    assert np.array_equal(M1(r), M2(r))


def test_coarse_correction_is_a_projection():
    p = workloads.config("tiny")
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Z, info = geneo.coarse_space(p, subs, A)
    M2 = krylov.TwoLevelAS(A, subs, Z)
    n = A.shape[0]
    P = dense_op(lambda v: M2.coarse(A @ v), n)
    assert np.allclose(P @ P, P, atol=1e-9)
    assert np.linalg.matrix_rank(P, tol=1e-8) == Z.shape[1]


def test_two_level_preconditioner_is_spd():
    p = workloads.config("tiny")
    A, b = fem.assemble_system(p)
    subs = decomp.partition(p)
    Z, _ = geneo.coarse_space(p, subs, A)
    M = dense_op(krylov.TwoLevelAS(A, subs, Z), A.shape[0])
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_lanczos_kappa_matches_dense_spectrum():
    p = workloads.config("c1")
    r = solver.solve(p, precond="geneo", tol=1e-14, maxit=500)
    A = r["A"].toarray()
    M = dense_op(r["M"], A.shape[0])
    ev = np.sort(np.real(sla.eigvals(M @ A)))
    kappa = ev[-1] / ev[0]
    assert r["kappa"] == pytest.approx(kappa, rel=0.02)


def test_flexible_cg_equals_pcg_for_fixed_spd_preconditioner():
    p = workloads.config("c1")
    st = solver.setup(p, precond="geneo")
    x1, i1 = krylov.pcg(st["A"], st["b"], st["M"], tol=1e-8)
    x2, i2 = krylov.pcg(st["A"], st["b"], st["M"], tol=1e-8, flexible=True)
    assert abs(i1["iterations"] - i2["iterations"]) <= 1
    assert np.linalg.norm(x1 - x2) <= 1e-7 * np.linalg.norm(x1)


def test_pou_weighted_schwarz_with_flexible_cg_converges():
    p = workloads.config("c1")
    r = solver.solve(p, precond="geneo", weight="pou", tol=1e-8)
    u = np.linalg.solve(r["A"].toarray(), r["b"])
    assert r["true_rel_res"] < 2e-8
    assert np.linalg.norm(r["u"] - u) <= 1e-6 * np.linalg.norm(u)


def test_pou_weighted_one_level_is_the_plain_one_over_multiplicity():
    # With the standard PoU every subdomain holding a free dof in its interior
    # weighs it by 1/multiplicity, so sum_j R_j^T X_j A_j^-1 R_j r is the plain
    # one-level sum divided by the multiplicity, dof by dof.
    p = workloads.config("small")
    A, _ = fem.assemble_system(p)
    subs = decomp.partition(p)
    mult = np.zeros(A.shape[0])
    for s in subs:
        mult[s.int_dofs] += 1.0
    free = np.ones(A.shape[0], bool)
    free[p["dirichlet_dofs"]] = False
    assert mult[free].max() >= 4
    r = np.random.default_rng(5).normal(size=A.shape[0])
    plain = krylov.OneLevelAS(A, subs, "none")(r)
    weighted = krylov.OneLevelAS(A, subs, "pou")(r)
    assert np.abs(weighted[free] * mult[free] - plain[free]).max() <= 1e-12 * np.abs(plain).max()
    assert np.all(weighted[~free] == 0.0)


def test_geneo_condition_insensitive_to_contrast():
    # Sec. 3.2 bound: kappa stays bounded as the layer stiffness contrast grows.
    md = dict(fixed_modes=0, threshold=0.0, max_modes=20, shift=-0.01)
    kg, ka = [], []
    for c in (1e2, 1e4, 1e6):
        p = workloads.config("c1", contrast=c, modes=md)
        st = solver.setup(p, precond="geneo")
        A = st["A"].toarray()
        ev = np.sort(np.real(sla.eigvals(dense_op(st["M"], A.shape[0]) @ A)))
        kg.append(ev[-1] / ev[0])
        st1 = solver.setup(p, precond="as")
        ev1 = np.sort(np.real(sla.eigvals(dense_op(st1["M"], A.shape[0]) @ A)))
        ka.append(ev1[-1] / ev1[0])
    assert max(kg) / min(kg) < 2.0
    assert all(g < a / 10 for g, a in zip(kg, ka))
