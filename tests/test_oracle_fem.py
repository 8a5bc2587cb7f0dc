"""Pins for the oracle's Q1 elements, assembly, BCs and load (Sec. 2)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import fem, material
import workloads


def rigid_modes(coords):
    """6 rigid-body displacement fields at the given node coordinates."""
    n = coords.shape[0]
    R = np.zeros((3 * n, 6))
    for c in range(3):
        R[c::3, c] = 1.0
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    # rotations omega x r for omega = e_x, e_y, e_z
    R[1::3, 3], R[2::3, 3] = -z, y
    R[0::3, 4], R[2::3, 4] = z, -x
    R[0::3, 5], R[1::3, 5] = -y, x
    return R


def box_coords(hx, hy, hz):
    return fem.CORNERS * np.array([hx, hy, hz], float)


def test_shape_functions_partition_and_linear_reproduction():
    rng = np.random.default_rng(0)
    for _ in range(5):
        xi = rng.uniform(-1, 1, 3)
        g = fem.shape_grad_ref(*xi)
        assert np.allclose(g.sum(axis=0), 0, atol=1e-15)
        # sum_a grad N_a (x) X_a = identity on the reference cube (X_a = corner signs)
        s = 2.0 * fem.CORNERS - 1.0
        assert np.allclose(s.T @ g, np.eye(3), atol=1e-14)


@pytest.mark.parametrize("th,ph", [(0.0, 0.0), (0.6, 0.0), (1.1, 0.3)])
def test_element_stiffness_symmetry_rigid_null_space(th, ph):
    Cv = material.element_stiffness_voigt(workloads.PLY, th, ph)
    hx, hy, hz = 0.5, 0.5, 0.115
    K = fem.element_stiffness(Cv, hx, hy, hz)
    assert np.allclose(K, K.T, rtol=0, atol=1e-9 * np.abs(K).max())
    R = rigid_modes(box_coords(hx, hy, hz))
    assert np.abs(K @ R).max() <= 1e-12 * np.abs(K).max() * np.abs(R).max() * 24
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6
    assert ev.min() > -1e-10 * ev.max()


def test_uniform_strain_energy_exact():
    # u = eps0 . x  gives the element energy V eps0^T C eps0 exactly.
    rng = np.random.default_rng(3)
    Cv = material.element_stiffness_voigt(workloads.PLY, 0.4, 0.1)
    hx, hy, hz = 0.7, 0.3, 0.05
    K = fem.element_stiffness(Cv, hx, hy, hz)
    E = rng.normal(size=(3, 3))
    E = 0.5 * (E + E.T)
    X = box_coords(hx, hy, hz)
    u = (X @ E.T).reshape(-1)
    ev = np.array([E[0, 0], E[1, 1], E[2, 2], 2 * E[1, 2], 2 * E[0, 2], 2 * E[0, 1]])
    assert u @ K @ u == pytest.approx(hx * hy * hz * ev @ Cv @ ev, rel=1e-12)


def test_assembly_matches_element_loop():
    p = workloads.config("tiny")
    A = fem.assemble_stiffness(p).toarray()
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    Cel = fem.element_voigt_all(p)
    D = np.zeros_like(A)
    e = 0
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                d = fem.element_dofs(nx, ny, ex, ey, ez)
                hx = p["x"][ex + 1] - p["x"][ex]
                hy = p["y"][ey + 1] - p["y"][ey]
                hz = p["z"][ez + 1] - p["z"][ez]
                D[np.ix_(d, d)] += fem.element_stiffness(Cel[e], hx, hy, hz)
                e += 1
    assert np.allclose(A, D, rtol=0, atol=1e-10 * np.abs(D).max())


def test_unconstrained_global_null_space_is_rigid():
    p = workloads.config("tiny", clamp="none")
    A = fem.assemble_stiffness(p).toarray()
    ev = np.linalg.eigvalsh(A)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 6
    nnx, nny, nnz = p["nx"] + 1, p["ny"] + 1, p["nz"] + 1
    Zc, Yc, Xc = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    R = rigid_modes(np.stack([Xc.ravel(), Yc.ravel(), Zc.ravel()], axis=1))
    assert np.linalg.norm(A @ R) <= 1e-13 * np.linalg.norm(A, 2) * np.linalg.norm(R)


def test_patch_test_linear_field_reproduced():
    # Homogeneous anisotropic material, graded z mesh: Dirichlet data of a
    # linear field on the whole boundary gives that field at every node.
    p = workloads.config("small", ply_angles_deg=[37, 37, 37], resin_between=False)
    p["elem_theta"][:] = np.deg2rad(37.0)
    p["elem_mat"][:] = 0
    dz = np.diff(p["z"]) * (1.0 + 0.5 * np.sin(np.arange(p["nz"]) + 0.3))
    p["z"] = np.concatenate([[0.0], np.cumsum(dz)])  # graded, still increasing
    assert np.all(np.diff(p["z"]) > 0)
    p["top_pressure"] = 0.0
    nnx, nny, nnz = p["nx"] + 1, p["ny"] + 1, p["nz"] + 1
    Zc, Yc, Xc = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    X = np.stack([Xc.ravel(), Yc.ravel(), Zc.ravel()], axis=1)
    G = np.array([[0.01, -0.02, 0.005], [0.003, 0.02, -0.01], [0.004, 0.007, -0.015]])
    c = np.array([0.1, -0.2, 0.3])
    u_ex = (X @ G.T + c).reshape(-1)
    I, J, K = np.meshgrid(np.arange(nnx), np.arange(nny), np.arange(nnz), indexing="ij")
    bnd = ((I == 0) | (I == nnx - 1) | (J == 0) | (J == nny - 1) | (K == 0) | (K == nnz - 1))
    bnodes = np.sort((I + nnx * (J + nny * K))[bnd])
    dofs = (3 * bnodes[:, None] + np.arange(3)).reshape(-1)
    p["dirichlet_dofs"] = dofs.astype(np.int32)
    p["dirichlet_values"] = u_ex[dofs]
    A, b = fem.assemble_system(p)
    u = spla.spsolve(A.tocsc(), b)
    assert np.abs(u - u_ex).max() <= 1e-12 * np.abs(u_ex).max()


def test_constrained_matrix_spd():
    p = workloads.config("c1")
    A, b = fem.assemble_system(p)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T, rtol=0, atol=1e-12 * np.abs(Ad).max())
    sla.cholesky(Ad, lower=True)


def test_top_pressure_total_load_and_symmetry():
    p = workloads.config("c1")
    b = fem.top_pressure_load(p)
    Lx, Ly = p["x"][-1] - p["x"][0], p["y"][-1] - p["y"][0]
    assert b[2::3].sum() == pytest.approx(-p["top_pressure"] * Lx * Ly, rel=1e-14)
    assert np.all(b[0::3] == 0) and np.all(b[1::3] == 0)
    # mirror symmetry about the mid-plane of y
    nnx, nny, nnz = p["nx"] + 1, p["ny"] + 1, p["nz"] + 1
    bz = b[2::3].reshape(nnz, nny, nnx)
    assert np.allclose(bz, bz[:, ::-1, :])
    # only top-face nodes are loaded
    assert np.all(bz[:-1] == 0)


def _fibre_strain(Cv, d):
    """Normal strain along unit d under the uniaxial stress d (x) d."""
    sig = np.array([d[0] ** 2, d[1] ** 2, d[2] ** 2, d[1] * d[2], d[0] * d[2], d[0] * d[1]])
    e = np.linalg.solve(Cv, sig)                     # engineering shear strains
    return (d[0] ** 2 * e[0] + d[1] ** 2 * e[1] + d[2] ** 2 * e[2]
            + d[1] * d[2] * e[3] + d[0] * d[2] * e[4] + d[0] * d[1] * e[5])


def test_element_material_follows_the_fibre():
    # Every ply element of a wrinkled block is stiff (E1) along its fibre
    # (cos t cos f, sin t cos f, -sin f) for its own ply angle t and wrinkle
    # angle f: the element stiffness takes the angles with their signs.
    p = workloads.config("small", wrinkle=(8.0, 3.0))
    Cv = fem.element_voigt_all(p)
    E1 = p["materials"][0][0]
    ply = np.flatnonzero(p["elem_mat"] == 0)
    assert np.abs(p["elem_phi"][ply]).max() > 0.05 and np.ptp(p["elem_theta"][ply]) > 0.5
    for e in ply[:: max(1, ply.size // 40)]:
        t, f = p["elem_theta"][e], p["elem_phi"][e]
        d = np.array([np.cos(t) * np.cos(f), np.sin(t) * np.cos(f), -np.sin(f)])
        assert _fibre_strain(Cv[e], d) == pytest.approx(1.0 / E1, rel=1e-10)
    # and the element stiffness matrices are built from those same C_e
    x, y, z = p["x"], p["y"], p["z"]
    nx, ny = p["nx"], p["ny"]
    Ku, inv, elems = fem.element_stiffness_all(p)
    for e in ply[:: max(1, ply.size // 10)]:
        ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
        Ke = fem.element_stiffness(Cv[e], x[ex + 1] - x[ex], y[ey + 1] - y[ey], z[ez + 1] - z[ez])
        got = Ku[inv[np.flatnonzero(elems == e)[0]]]
        assert np.abs(got - Ke).max() <= 1e-12 * np.abs(Ke).max()
