"""Pins for the oracle's stress recovery (Sec. 2 constitutive law, Sec. 5).

A linear displacement field u = G x has the uniform strain sym(G), so every
element's stress must equal C_e eps(G) with the engineering-shear Voigt strain
written out by hand here; a rigid rotation carries no stress; a pure shear
field excites only its own Voigt component.
"""
import numpy as np

import workloads
from oracle import fem


def _nodes(p):
    Z, Y, X = np.meshgrid(p["z"], p["y"], p["x"], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def test_linear_field_gives_c_times_uniform_strain():
    p = workloads.config("small", wrinkle=(8.0, 3.0))
    X = _nodes(p)
    G = np.array([[0.01, -0.02, 0.005], [0.003, 0.02, -0.01], [0.004, 0.007, -0.015]])
    u = (X @ G.T).reshape(-1)
    eps = np.array([G[0, 0], G[1, 1], G[2, 2], G[1, 2] + G[2, 1], G[0, 2] + G[2, 0],
                    G[0, 1] + G[1, 0]])
    sig = fem.element_stresses(p, u)
    ref = np.einsum("eij,j->ei", fem.element_voigt_all(p), eps)
    assert np.abs(sig - ref).max() <= 1e-12 * np.abs(ref).max()


def test_rigid_rotation_is_stress_free():
    p = workloads.config("c1")
    X = _nodes(p) - 1.0
    w = np.array([0.3, -0.2, 0.5])
    u = np.cross(w, X).reshape(-1)
    sig = fem.element_stresses(p, u)
    scale = np.abs(fem.element_voigt_all(p)).max() * np.abs(u).max()
    assert np.abs(sig).max() <= 1e-12 * scale


def test_pure_shear_excites_its_component():
    # isotropic material: u = (0, 0, a x) gives gamma_xz = a, so sigma_xz = G a
    p = workloads.config("tiny")
    p["materials"] = np.array([list(workloads.RESIN)])
    p["elem_mat"][:] = 0
    p["elem_theta"][:] = 0.0
    X = _nodes(p)
    a = 1e-3
    u = np.zeros_like(X)
    u[:, 2] = a * X[:, 0]
    sig = fem.element_stresses(p, u.reshape(-1))
    Gm = workloads.RESIN[3]
    assert np.allclose(sig[:, 4], Gm * a, rtol=1e-12, atol=0)
    assert np.abs(np.delete(sig, 4, axis=1)).max() <= 1e-12 * Gm * a


def test_centroid_value_of_a_varying_strain():
    # u = (a x y, b y z, c z x) lies in the trilinear space, so it is
    # interpolated exactly; its strain varies linearly across each element and
    # the recovered stress is C_e times the strain at the element's centre
    # (eps_xx = a y, eps_yy = b z, eps_zz = c x, gamma_xy = a x,
    # gamma_yz = b y, gamma_xz = c z there).
    p = workloads.config("small", wrinkle=(8.0, 3.0))
    X = _nodes(p)
    a, b, c = 0.004, -0.003, 0.002
    u = np.stack([a * X[:, 0] * X[:, 1], b * X[:, 1] * X[:, 2], c * X[:, 2] * X[:, 0]], 1).reshape(-1)
    ex, ey, ez = fem.element_coords(p)
    x, y, z = (np.asarray(p[k]) for k in ("x", "y", "z"))
    xc, yc, zc = 0.5 * (x[ex] + x[ex + 1]), 0.5 * (y[ey] + y[ey + 1]), 0.5 * (z[ez] + z[ez + 1])
    eps = np.stack([a * yc, b * zc, c * xc, b * yc, c * zc, a * xc], axis=1)
    ref = np.einsum("eij,ej->ei", fem.element_voigt_all(p), eps)
    sig = fem.element_stresses(p, u)
    assert np.abs(sig - ref).max() <= 1e-11 * np.abs(ref).max()
