"""Material law: generalised Hooke's law with orthotropic plies (Sec. 2).

Sec. 2 (eq-hooke) gives sigma_ij = C_ijkl eps_kl with C symmetric positive
definite; a ply is orthotropic with 9 constants plus an orientation, rotated
with standard tensor rotations; resin is isotropic with 2 Lame parameters.

Voigt order (11, 22, 33, 23, 13, 12) with engineering shear strains.
"""
from __future__ import annotations

import numpy as np

VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def compliance_orthotropic(E1, E2, E3, G12, G13, G23, nu12, nu13, nu23):
    """6x6 compliance S (strain = S stress) in material axes (Sec. 2, 9 constants)."""
    S = np.zeros((6, 6))
    S[0, 0] = 1.0 / E1
    S[1, 1] = 1.0 / E2
    S[2, 2] = 1.0 / E3
    S[0, 1] = S[1, 0] = -nu12 / E1
    S[0, 2] = S[2, 0] = -nu13 / E1
    S[1, 2] = S[2, 1] = -nu23 / E2
    S[3, 3] = 1.0 / G23
    S[4, 4] = 1.0 / G13
    S[5, 5] = 1.0 / G12
    return S


def stiffness_voigt(mat9):
    """6x6 Voigt stiffness C = S^-1 from (E1,E2,E3,G12,G13,G23,nu12,nu13,nu23)."""
    return np.linalg.inv(compliance_orthotropic(*mat9))


def lame_isotropic(E, nu):
    """Isotropic stiffness from the two Lame parameters (Sec. 2, resin)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


def voigt_to_tensor(Cv):
    """4th-order C_ijkl from the 6x6 Voigt matrix (engineering shear)."""
    C = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            v = Cv[I, J]
            C[i, j, k, l] = C[j, i, k, l] = C[i, j, l, k] = C[j, i, l, k] = v
    return C


def tensor_to_voigt(C):
    Cv = np.zeros((6, 6))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            Cv[I, J] = C[i, j, k, l]
    return Cv


def rotation(theta, phi=0.0):
    """Direction cosines Q (material axes -> global) for a ply.

    Reading of "standard tensor rotations" (Sec. 2): the in-plane ply angle
    theta turns about +z from +x toward +y; the wrinkle angle phi then tilts
    the fibre out of plane about the ply's transverse in-plane axis:
    Q = R_z(theta) R_y(phi); the fibre direction is Q e1.
    """
    c, s = np.cos(theta), np.sin(theta)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    cp, sp = np.cos(phi), np.sin(phi)
    Ry = np.array([[cp, 0.0, sp], [0.0, 1.0, 0.0], [-sp, 0.0, cp]])
    return Rz @ Ry


def rotate_tensor(C, Q):
    """C'_ijkl = Q_ip Q_jq Q_kr Q_ls C_pqrs (tensor transformation law)."""
    return np.einsum("ip,jq,kr,ls,pqrs->ijkl", Q, Q, Q, Q, C)


def element_stiffness_tensor(mat9, theta, phi=0.0):
    """Global-frame 4th-order stiffness of one element (Sec. 2, eq-hooke)."""
    Cv = stiffness_voigt(mat9)
    return rotate_tensor(voigt_to_tensor(Cv), rotation(theta, phi))


def element_stiffness_voigt(mat9, theta, phi=0.0):
    return tensor_to_voigt(element_stiffness_tensor(mat9, theta, phi))
