"""Pins for the oracle's material law (Sec. 2 eq-hooke, Sec. 5 constants)."""
import numpy as np
import pytest

from oracle import material as M
import workloads

PLY = workloads.PLY


def kelvin(Cv):
    """Kelvin (Mandel) form: shear rows/cols scaled by sqrt(2) -> orthonormal basis."""
    s = np.array([1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2)])
    return Cv * s[:, None] * s[None, :]


def test_uniaxial_stress_engineering_constants():
    # A unit stress sigma_11 gives strains 1/E1, -nu12/E1, -nu13/E1 by the
    # definition of the engineering constants.
    E1, E2, E3, G12, G13, G23, nu12, nu13, nu23 = PLY
    C = M.stiffness_voigt(PLY)
    eps = np.linalg.solve(C, np.array([1.0, 0, 0, 0, 0, 0]))
    assert np.allclose(eps, [1 / E1, -nu12 / E1, -nu13 / E1, 0, 0, 0], rtol=1e-12, atol=0)
    eps = np.linalg.solve(C, np.array([0, 1.0, 0, 0, 0, 0]))
    assert np.allclose(eps, [-nu12 / E1, 1 / E2, -nu23 / E2, 0, 0, 0], rtol=1e-12, atol=1e-20)
    for k, G in ((3, G23), (4, G13), (5, G12)):
        sig = np.zeros(6)
        sig[k] = 1.0
        eps = np.linalg.solve(C, sig)
        assert eps[k] == pytest.approx(1 / G, rel=1e-12)
        assert np.allclose(np.delete(eps, k), 0, atol=1e-20)


def test_uniaxial_stress_general_orthotropic():
    # Nine distinct constants (E2 != E3, G13 != G12, ...), so that an engineering
    # constant divided by the wrong modulus cannot hide behind the ply's
    # transverse isotropy: sigma_kk = 1 gives eps_kk = 1/E_k and, for i != k,
    # eps_ii = -nu_ki / E_k with nu_ki = nu_ik E_k / E_i for i < k.
    E1, E2, E3 = 140000.0, 9000.0, 6000.0
    G12, G13, G23 = 4800.0, 4100.0, 2700.0
    nu12, nu13, nu23 = 0.31, 0.27, 0.45
    mat = (E1, E2, E3, G12, G13, G23, nu12, nu13, nu23)
    C = M.stiffness_voigt(mat)
    E = (E1, E2, E3)
    nu = {(0, 1): nu12, (0, 2): nu13, (1, 2): nu23}
    for k in range(3):
        sig = np.zeros(6)
        sig[k] = 1.0
        eps = np.linalg.solve(C, sig)
        want = np.zeros(6)
        want[k] = 1.0 / E[k]
        for i in range(3):
            if i != k:
                nu_ki = nu[(k, i)] if k < i else nu[(i, k)] * E[k] / E[i]
                want[i] = -nu_ki / E[k]
        assert np.allclose(eps, want, rtol=1e-12, atol=1e-22), k


def test_isotropic_two_routes_agree():
    E, nu = 10000.0, 0.35
    G = E / (2 * (1 + nu))
    a = M.stiffness_voigt((E, E, E, G, G, G, nu, nu, nu))
    b = M.lame_isotropic(E, nu)
    assert np.allclose(a, b, rtol=1e-12)


def test_rotation_identity_and_90_degrees():
    C = M.stiffness_voigt(PLY)
    assert np.allclose(M.element_stiffness_voigt(PLY, 0.0, 0.0), C, rtol=1e-14, atol=1e-9)
    R = M.element_stiffness_voigt(PLY, np.pi / 2)
    assert R[0, 0] == pytest.approx(C[1, 1], rel=1e-12)
    assert R[1, 1] == pytest.approx(C[0, 0], rel=1e-12)
    assert R[2, 2] == pytest.approx(C[2, 2], rel=1e-12)
    assert R[3, 3] == pytest.approx(C[4, 4], rel=1e-12)
    assert R[4, 4] == pytest.approx(C[3, 3], rel=1e-12)
    assert R[5, 5] == pytest.approx(C[5, 5], rel=1e-12)
    assert R[0, 2] == pytest.approx(C[1, 2], rel=1e-12)


def test_fibre_direction_convention():
    th, ph = 0.7, 0.2
    Q = M.rotation(th, ph)
    assert np.allclose(Q @ [1, 0, 0], [np.cos(th) * np.cos(ph), np.sin(th) * np.cos(ph), -np.sin(ph)])
    assert np.allclose(Q.T @ Q, np.eye(3), atol=1e-15)


def test_directional_modulus_along_fibre():
    # Young's modulus measured along the rotated fibre equals E1.
    rng = np.random.default_rng(0)
    for _ in range(5):
        th, ph = rng.uniform(-np.pi, np.pi), rng.uniform(-0.5, 0.5)
        C4 = M.element_stiffness_tensor(PLY, th, ph)
        Cv = M.tensor_to_voigt(C4)
        Sv = np.linalg.inv(Cv)
        n = M.rotation(th, ph) @ [1.0, 0, 0]
        # stress n (x) n in Voigt form (no factor on shear stresses)
        sig = np.array([n[0] ** 2, n[1] ** 2, n[2] ** 2, n[1] * n[2], n[0] * n[2], n[0] * n[1]])
        eps = Sv @ sig
        # normal strain along n: eps_ij n_i n_j with engineering shear halved
        e = eps[0] * n[0] ** 2 + eps[1] * n[1] ** 2 + eps[2] * n[2] ** 2 \
            + eps[3] * n[1] * n[2] + eps[4] * n[0] * n[2] + eps[5] * n[0] * n[1]
        assert 1.0 / e == pytest.approx(PLY[0], rel=1e-10)


def test_kelvin_invariants_and_spd():
    C = M.stiffness_voigt(PLY)
    ev0 = np.linalg.eigvalsh(kelvin(C))
    assert ev0.min() > 0
    rng = np.random.default_rng(1)
    for _ in range(10):
        R = M.element_stiffness_voigt(PLY, rng.uniform(-3, 3), rng.uniform(-1, 1))
        assert np.allclose(R, R.T, rtol=0, atol=1e-9)
        ev = np.linalg.eigvalsh(kelvin(R))
        assert np.allclose(ev, ev0, rtol=1e-12)
