"""Orthotropic ply stiffness and its rotation into the laminate frame.

Hooke's law sigma_ij = C_ijkl eps_kl (Eq. eq-hooke).  A ply is a homogeneous
orthotropic material given by nine engineering constants, oriented in the
global frame by a rotation of the fourth-order tensor about the laminate
normal z (Sec. 5.1, "standard tensor rotations").

Conventions (the paper does not fix them): Voigt order 11, 22, 33, 23, 13, 12
with engineering shear strains; the fibre axis of a ply at angle theta is
(cos theta, sin theta, 0), theta measured from x toward y about +z.  On a
curved laminate (the C-section spar) each element carries its own reference
frame (a0, a1, a2); the fibre is then cos theta a0 + sin theta a1 and the
normal a2, the same rotation applied in the element's frame.
"""
import numpy as np

VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def compliance(E):
    """6x6 Voigt compliance of an orthotropic ply in its material axes.

    E = (E11, E22, E33, G12, G13, G23, nu12, nu13, nu23).
    """
    E11, E22, E33, G12, G13, G23, nu12, nu13, nu23 = E
    S = np.zeros((6, 6))
    S[0, 0], S[1, 1], S[2, 2] = 1.0 / E11, 1.0 / E22, 1.0 / E33
    S[0, 1] = S[1, 0] = -nu12 / E11
    S[0, 2] = S[2, 0] = -nu13 / E11
    S[1, 2] = S[2, 1] = -nu23 / E22
    S[3, 3], S[4, 4], S[5, 5] = 1.0 / G23, 1.0 / G13, 1.0 / G12
    return S


def voigt_to_tensor(Cv):
    """Fourth-order tensor C_ijkl from a 6x6 Voigt stiffness (engineering shear)."""
    C = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(VOIGT_PAIRS):
        for J, (k, l) in enumerate(VOIGT_PAIRS):
            for a, b in ((i, j), (j, i)):
                for c, d in ((k, l), (l, k)):
                    C[a, b, c, d] = Cv[I, J]
    return C


def tensor_to_voigt(C):
    Cv = np.zeros((6, 6))
    for I, (i, j) in enumerate(VOIGT_PAIRS):
        for J, (k, l) in enumerate(VOIGT_PAIRS):
            Cv[I, J] = C[i, j, k, l]
    return Cv


def ply_tensor(E):
    """C_ijkl of the ply in its material axes: the inverse of the compliance."""
    return voigt_to_tensor(np.linalg.inv(compliance(E)))


def rotation_z(theta_deg):
    """Columns are the material axes (fibre, in-plane transverse, normal) in global coordinates."""
    t = np.deg2rad(theta_deg)
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def material_axes(theta_deg, frame=None):
    """Columns: fibre, in-plane transverse and normal axes in global coordinates.

    ``frame`` (rows a0, a1, a2, orthonormal and right-handed) is the ply's
    reference frame: the fibre lies at angle theta from a0 toward a1 in the
    a0-a1 plane and a2 is the laminate normal.  ``None`` is the box beam's
    frame (x, y, z), where this is ``rotation_z``.
    """
    Rz = rotation_z(theta_deg)
    if frame is None:
        return Rz
    return np.asarray(frame, dtype=np.float64).T @ Rz


def rotated_tensor(E, theta_deg, frame=None):
    """Global-frame C_ijkl = R_ip R_jq R_kr R_ls C0_pqrs of a ply at angle theta
    (R = ``material_axes(theta, frame)``)."""
    R = material_axes(theta_deg, frame)
    return np.einsum("ip,jq,kr,ls,pqrs->ijkl", R, R, R, R, ply_tensor(E))


def isotropic_constants(E, nu):
    """Nine engineering constants of an isotropic material."""
    G = E / (2.0 * (1.0 + nu))
    return (E, E, E, G, G, G, nu, nu, nu)
