"""Pins for the oracle's 20-node serendipity element (the paper's element, Sec. 5).

Shape functions: Kronecker property at the nodes, and exact reproduction of
the 20 monomials that span the serendipity space (any dropped term or wrong
sign in one of the 20 functions breaks it); gradients against central
differences.  Element stiffness: symmetric, exactly six zero eigenvalues
(rigid modes), and the strain energy of a quadratic displacement field
(linear strain) equal to its integral evaluated independently of the element
(Gauss rule of higher order on the field itself).  Mesh: node count in closed
form, exactly six zero eigenvalues of the unconstrained global matrix, and a
patch test (linear boundary data, homogeneous material: exact interior
field).  Against the trilinear element: on a coarse cantilever mesh the
quadratic element's tip deflection is much closer to a fine-mesh reference.
"""
import itertools

import numpy as np
import scipy.sparse.linalg as spla

from oracle import fem, material, serendipity as sd
from workloads.laminate import PLY, make_block

MONOMIALS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2),
             (1, 1, 0), (0, 1, 1), (1, 0, 1), (2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1),
             (1, 0, 2), (0, 1, 2), (1, 1, 1), (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def test_kronecker_and_serendipity_span():
    for b, xb in enumerate(sd.REF_NODES):
        N = sd.shape(*xb)
        assert np.allclose(N, np.eye(20)[b], atol=1e-14)
    rng = np.random.default_rng(0)
    for _ in range(20):
        t = rng.uniform(-1, 1, 3)
        N = sd.shape(*t)
        for m in MONOMIALS:
            at_nodes = np.prod(sd.REF_NODES ** np.array(m), axis=1)
            assert abs(N @ at_nodes - np.prod(t ** np.array(m))) <= 1e-13


def test_gradients_are_derivatives():
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        t = rng.uniform(-1, 1, 3)
        G = sd.shape_grad(*t)
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fd = (sd.shape(*(t + e)) - sd.shape(*(t - e))) / (2 * h)
            assert np.abs(G[:, d] - fd).max() <= 1e-8


def _ply_C():
    # the paper's ply at 30 degrees: a fully anisotropic 6 x 6 stiffness in the global frame
    return material.element_stiffness_voigt(PLY, np.deg2rad(30.0), 0.0)


def test_element_stiffness_rigid_modes_and_quadratic_energy():
    C = _ply_C()
    h = np.array([0.5, 0.7, 0.23])
    K = sd.element_stiffness(C, *h)
    assert np.allclose(K, K.T, atol=1e-12 * abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert np.all(np.abs(ev[:6]) <= 1e-10 * ev[-1]) and ev[6] > 1e-6 * ev[-1]
    # u(x) quadratic -> eps linear: energy by the element vs a 5-point Gauss rule on the field
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(3, 10))            # u_c = Q[c] . (1, x, y, z, x^2, y^2, z^2, xy, yz, xz)

    def basis(x):
        return np.array([1, x[0], x[1], x[2], x[0] ** 2, x[1] ** 2, x[2] ** 2,
                         x[0] * x[1], x[1] * x[2], x[0] * x[2]])

    def grad_basis(x):
        g = np.zeros((10, 3))
        g[1, 0] = g[2, 1] = g[3, 2] = 1.0
        g[4, 0], g[5, 1], g[6, 2] = 2 * x[0], 2 * x[1], 2 * x[2]
        g[7] = (x[1], x[0], 0.0)
        g[8] = (0.0, x[2], x[1])
        g[9] = (x[2], 0.0, x[0])
        return g

    nodes = (sd.REF_NODES + 1.0) * 0.5 * h
    u = np.array([Q @ basis(xn) for xn in nodes]).reshape(-1)
    e_elem = 0.5 * u @ K @ u
    pts, wts = np.polynomial.legendre.leggauss(5)
    e_ref = 0.0
    for (i, a), (j, b), (k, c) in itertools.product(enumerate(pts), repeat=3):
        x = (np.array([a, b, c]) + 1.0) * 0.5 * h
        Gu = Q @ grad_basis(x)                  # du_c / dx_d
        eps = np.array([Gu[0, 0], Gu[1, 1], Gu[2, 2], Gu[1, 2] + Gu[2, 1], Gu[0, 2] + Gu[2, 0],
                        Gu[0, 1] + Gu[1, 0]])
        e_ref += wts[i] * wts[j] * wts[k] * 0.5 * eps @ C @ eps
    e_ref *= h.prod() / 8.0
    assert abs(e_elem - e_ref) <= 1e-11 * abs(e_ref)


def test_mesh_nodes_and_global_rigid_modes():
    p = make_block(3, 2, 2, [0.0, 90.0], partition=(1, 1, 1, 1))
    ids, nn = sd.node_map(3, 2, 2)
    nx, ny, nz = 3, 2, 2
    assert nn == ((nx + 1) * (ny + 1) * (nz + 1) + nx * (ny + 1) * (nz + 1)
                  + ny * (nx + 1) * (nz + 1) + nz * (nx + 1) * (ny + 1))
    assert sorted(ids[ids >= 0]) == list(range(nn))
    A = sd.assemble_stiffness(p).toarray()
    ev = np.linalg.eigvalsh(A)
    assert np.all(np.abs(ev[:6]) <= 1e-9 * ev[-1]) and ev[6] > 1e-7 * ev[-1]


def test_patch_linear_field():
    p = make_block(3, 2, 2, [0.0, 0.0], partition=(1, 1, 1, 1))
    A = sd.assemble_stiffness(p)
    xyz = sd.node_coordinates(p)
    G = np.array([[0.01, -0.02, 0.003], [0.004, 0.02, -0.01], [-0.005, 0.001, 0.015]])
    u_ex = (xyz @ G.T + np.array([0.1, -0.2, 0.05])).reshape(-1)
    lo, hi = xyz.min(0), xyz.max(0)
    bnd = np.any((np.abs(xyz - lo) < 1e-12) | (np.abs(xyz - hi) < 1e-12), axis=1)
    D = (3 * np.flatnonzero(bnd)[:, None] + np.arange(3)).reshape(-1)
    F = np.setdiff1d(np.arange(A.shape[0]), D)
    rhs = -A[F][:, D] @ u_ex[D]
    uF = spla.spsolve(A[F][:, F].tocsc(), rhs)
    assert np.abs(uF - u_ex[F]).max() <= 1e-12 * np.abs(u_ex).max()


def _tip_deflection(p, A, xyz):
    x0 = xyz[:, 0] < 1e-12
    D = (3 * np.flatnonzero(x0)[:, None] + np.arange(3)).reshape(-1)
    b = np.zeros(A.shape[0])
    top = np.abs(xyz[:, 2] - xyz[:, 2].max()) < 1e-12
    b[3 * np.flatnonzero(top) + 2] = -1.0 / top.sum()      # unit total downward load on the top
    F = np.setdiff1d(np.arange(A.shape[0]), D)
    u = np.zeros(A.shape[0])
    u[F] = spla.spsolve(A[F][:, F].tocsc(), b[F])
    tip = np.abs(xyz[:, 0] - xyz[:, 0].max()) < 1e-12
    return u[3 * np.flatnonzero(tip) + 2].mean()


def test_quadratic_element_beats_trilinear_on_a_coarse_cantilever():
    # the same 8 x 1 x 1 beam, one element through the thickness and the width;
    # reference: the serendipity element on a 32 x 2 x 4 mesh
    def beam(nx, ny, nz):
        q = make_block(nx, ny, nz, [0.0], partition=(1, 1, 1, 1))
        q["x"] = np.linspace(0.0, 8.0, nx + 1)
        q["y"] = np.linspace(0.0, 1.0, ny + 1)
        q["z"] = np.linspace(0.0, 1.0, nz + 1)
        return q

    def ser(q):
        return _tip_deflection(q, sd.assemble_stiffness(q), sd.node_coordinates(q))

    def q1(q):
        A = fem.assemble_stiffness(q)
        Z, Y, X = np.meshgrid(q["z"], q["y"], q["x"], indexing="ij")
        return _tip_deflection(q, A, np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1))

    ref = ser(beam(32, 2, 4))
    coarse = beam(8, 1, 1)
    assert abs(ser(coarse) - ref) < 0.5 * abs(q1(coarse) - ref)


def test_face_functions_are_the_element_functions_on_the_face():
    rng = np.random.default_rng(4)
    others = [a for a in range(20) if a not in sd.TOP_FACE]
    for _ in range(10):
        xi, eta = rng.uniform(-1, 1, 2)
        N = sd.shape(xi, eta, 1.0)
        assert np.allclose(N[sd.TOP_FACE], sd.face_shape(xi, eta), atol=1e-14)
        assert np.abs(N[others]).max() <= 1e-14


def test_top_load_total_and_pattern():
    p = make_block(3, 2, 2, [0.0, 90.0], partition=(1, 1, 1, 1))
    b = sd.top_pressure_load(p)
    Lx, Ly = p["x"][-1] - p["x"][0], p["y"][-1] - p["y"][0]
    assert abs(b.sum() + p["top_pressure"] * Lx * Ly) <= 1e-12 * Lx * Ly
    assert np.all(b[0::3] == 0.0) and np.all(b[1::3] == 0.0)
    xyz = sd.node_coordinates(p)
    top = np.abs(xyz[:, 2] - xyz[:, 2].max()) < 1e-12
    assert np.all(b[2::3][~top] == 0.0)
    # a corner of the top face lies in one element and takes -1/12 of its face's downward
    # force -q * hx * hy: +q * hx * hy / 12
    hx, hy = p["x"][1] - p["x"][0], p["y"][1] - p["y"][0]
    corner = np.flatnonzero(top & (xyz[:, 0] == p["x"][0]) & (xyz[:, 1] == p["y"][0]))[0]
    assert abs(b[3 * corner + 2] - p["top_pressure"] * hx * hy / 12.0) <= 1e-15


def test_clamped_system_is_spd_and_solves():
    p = make_block(3, 2, 2, [0.0, 90.0], partition=(1, 1, 1, 1))
    A, b = sd.assemble_system(p)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T, atol=1e-12 * abs(Ad).max())
    np.linalg.cholesky(Ad)
    u = np.linalg.solve(Ad, b)
    D = sd.clamp_dofs(p)
    assert np.all(u[D] == 0.0) and u[2::3].min() < 0.0       # clamped, and the block bends down
