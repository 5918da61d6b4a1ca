"""Pins of the oracle's material, element, load and fine solve against closed
forms and invariants (linear elasticity, Sec. 2 of the paper)."""
import numpy as np
import pytest

from oracle.assemble import assemble_global
from oracle.element import brick_corners, hex_stiffness, shape_values, CORNERS
from oracle.fine import solve_fine
from oracle.material import (isotropic_constants, rotated_tensor, rotation_z,
                             tensor_to_voigt, compliance)
from oracle.mesh import BeamMesh
from workloads import material_constants

E = material_constants()
E11, E22, E33, G12, G13, G23, nu12, nu13, nu23 = E


def strain_from_stress(C, sig):
    """Solve C : eps = sig for the symmetric strain tensor (through Voigt form)."""
    Cv = tensor_to_voigt(C)
    sv = np.array([sig[0, 0], sig[1, 1], sig[2, 2], sig[1, 2], sig[0, 2], sig[0, 1]])
    e = np.linalg.solve(Cv, sv)             # engineering shear strains
    return np.array([[e[0], e[5] / 2, e[4] / 2], [e[5] / 2, e[1], e[3] / 2], [e[4] / 2, e[3] / 2, e[2]]])


@pytest.mark.parametrize("theta", [0.0, 30.0, -45.0, 90.0, 17.3])
def test_ply_engineering_constants_in_rotated_frame(theta):
    """Uniaxial and shear stress states along the rotated material axes return
    the nine engineering constants (pins C, its inverse relation and the rotation)."""
    C = rotated_tensor(E, theta)
    R = rotation_z(theta)
    n, t, z = R[:, 0], R[:, 1], R[:, 2]
    s0 = 7.0
    eps = strain_from_stress(C, s0 * np.outer(n, n))
    assert np.isclose(n @ eps @ n, s0 / E11, rtol=1e-12)
    assert np.isclose(t @ eps @ t, -nu12 * s0 / E11, rtol=1e-10)
    assert np.isclose(z @ eps @ z, -nu13 * s0 / E11, rtol=1e-10)
    assert abs(n @ eps @ t) < 1e-14 * s0
    eps = strain_from_stress(C, s0 * np.outer(t, t))
    assert np.isclose(t @ eps @ t, s0 / E22, rtol=1e-12)
    assert np.isclose(z @ eps @ z, -nu23 * s0 / E22, rtol=1e-10)
    for (a, b), G in (((n, t), G12), ((n, z), G13), ((t, z), G23)):
        eps = strain_from_stress(C, s0 * (np.outer(a, b) + np.outer(b, a)))
        assert np.isclose(2 * a @ eps @ b, s0 / G, rtol=1e-12)


def test_tensor_symmetries_and_spd():
    for theta in (0.0, 33.0, 90.0):
        C = rotated_tensor(E, theta)
        assert np.allclose(C, C.transpose(1, 0, 2, 3), atol=1e-9)
        assert np.allclose(C, C.transpose(2, 3, 0, 1), atol=1e-9)
        # Mandel form: spectrum is rotation invariant and positive
        m = np.array([1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(2)])
        M = tensor_to_voigt(C) * np.outer(m, m)
        ev = np.linalg.eigvalsh(M)
        ev0 = np.linalg.eigvalsh(tensor_to_voigt(rotated_tensor(E, 0.0)) * np.outer(m, m))
        assert ev.min() > 0
        assert np.allclose(ev, ev0, rtol=1e-12)


def test_axis_swap_and_mirror():
    C0, C90 = rotated_tensor(E, 0.0), rotated_tensor(E, 90.0)
    assert np.isclose(C90[0, 0, 0, 0], C0[1, 1, 1, 1], rtol=1e-12)
    assert np.isclose(C90[1, 1, 1, 1], C0[0, 0, 0, 0], rtol=1e-12)
    assert np.isclose(C90[0, 2, 0, 2], C0[1, 2, 1, 2], rtol=1e-12)
    # theta -> -theta mirrors y: entries change sign with an odd number of y indices
    Cp, Cm = rotated_tensor(E, 25.0), rotated_tensor(E, -25.0)
    idx = np.indices((3, 3, 3, 3))
    sign = (-1.0) ** (idx == 1).sum(0)
    assert np.allclose(Cm, sign * Cp, atol=1e-9)


def test_isotropic_rotation_invariant():
    Ei = isotropic_constants(1e5, 0.3)
    lam_, mu_ = 1e5 * 0.3 / (1.3 * 0.4), 1e5 / 2.6
    d = np.eye(3)
    Ciso = lam_ * np.einsum("ij,kl->ijkl", d, d) + mu_ * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    for th in (0.0, 40.0):
        assert np.allclose(rotated_tensor(Ei, th), Ciso, rtol=1e-12, atol=1e-7)


def rigid_modes(X):
    c = X.mean(0)
    R = []
    for a in range(3):
        v = np.zeros((8, 3))
        v[:, a] = 1.0
        R.append(v.ravel())
    for w in np.eye(3):
        R.append(np.cross(w, X - c).ravel())
    return np.array(R).T


def test_element_null_space_and_symmetry():
    X = brick_corners(0, 0, 0, 2.0, 2.0, 0.25)
    K = hex_stiffness(X, rotated_tensor(E, 30.0))
    assert np.allclose(K, K.T, rtol=0, atol=1e-10 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert (np.abs(ev[:6]) < 1e-12 * ev[-1]).all()
    assert ev[6] > 1e-8 * ev[-1]
    assert np.abs(K @ rigid_modes(X)).max() < 1e-10 * np.abs(K).max()


def test_element_energy_against_independent_quadrature():
    """u^T K_e u equals int eps(u):C:eps(u) evaluated with a 5x5x5 rule and
    strains from central differences of the trilinear interpolant."""
    rng = np.random.default_rng(3)
    hx, hy, hz = 2.0, 1.5, 0.25
    X = brick_corners(0.3, -1.0, 2.0, hx, hy, hz)
    C = rotated_tensor(E, -27.0)
    K = hex_stiffness(X, C)
    x, w = np.polynomial.legendre.leggauss(5)
    for _ in range(3):
        u = rng.standard_normal((8, 3))

        def disp(xi):
            return shape_values(xi) @ u
        energy = 0.0
        h = 1e-3
        for a in range(5):
            for b in range(5):
                for c in range(5):
                    xi = np.array([x[a], x[b], x[c]])
                    G = np.zeros((3, 3))   # du_i/dx_j
                    for j, hj in enumerate((hx, hy, hz)):
                        e = np.zeros(3)
                        e[j] = h
                        G[:, j] = (disp(xi + e) - disp(xi - e)) / (2 * h) * (2.0 / hj)
                    eps = 0.5 * (G + G.T)
                    energy += np.einsum("ij,ijkl,kl->", eps, C, eps) * w[a] * w[b] * w[c] * hx * hy * hz / 8
        assert np.isclose(u.ravel() @ K @ u.ravel(), energy, rtol=1e-9)


def test_face_load_total_and_nodal_split():
    m = BeamMesh(3, 4, 5, 2.0, 1.5, 0.25)
    b = m.compression_load(2.0)
    assert np.isclose(b[0::3].sum(), -2.0 * 4 * 1.5 * 5 * 0.25, rtol=1e-14)
    assert np.abs(b[1::3]).max() == 0 and np.abs(b[2::3]).max() == 0
    inner = m.node_id(3, 2, 2)
    corner = m.node_id(3, 0, 0)
    assert np.isclose(b[3 * inner], -2.0 * 1.5 * 0.25, rtol=1e-14)
    assert np.isclose(b[3 * corner], -2.0 * 1.5 * 0.25 / 4, rtol=1e-14)
    assert np.count_nonzero(b) == 5 * 6


def test_patch_test_linear_field_reproduced():
    """Constant strain in a homogeneous anisotropic body: prescribing u = G x + c
    on the boundary, the interior FE solution is the same linear field."""
    m = BeamMesh(4, 3, 3, 1.0, 1.3, 0.7)
    ang = np.full((4, 3, 3), 30.0)
    A = assemble_global(m, ang, E).toarray()
    rng = np.random.default_rng(0)
    G, c = rng.standard_normal((3, 3)) * 1e-3, rng.standard_normal(3)
    ijk = np.array(m.node_ijk(np.arange(m.n_nodes))).T
    xyz = m.coords(np.arange(m.n_nodes))
    u_lin = (xyz @ G.T + c).ravel()
    bnd = ((ijk[:, 0] == 0) | (ijk[:, 0] == 4) | (ijk[:, 1] == 0) | (ijk[:, 1] == 3) |
           (ijk[:, 2] == 0) | (ijk[:, 2] == 3))
    bd = (3 * np.nonzero(bnd)[0][:, None] + np.arange(3)).ravel()
    idof = np.setdiff1d(np.arange(m.n_dof), bd)
    ui = np.linalg.solve(A[np.ix_(idof, idof)], -A[np.ix_(idof, bd)] @ u_lin[bd])
    assert np.abs(ui - u_lin[idof]).max() < 1e-12 * np.abs(u_lin).max()


def test_global_unconstrained_rigid_modes():
    m = BeamMesh(3, 2, 2, 2.0, 2.0, 0.25)
    ang = np.random.default_rng(1).uniform(-90, 90, (3, 2, 2))
    A = assemble_global(m, ang, E).toarray()
    ev = np.linalg.eigvalsh(A)
    assert (np.abs(ev[:6]) < 1e-11 * ev[-1]).all() and ev[6] > 1e-9 * ev[-1]


def test_euler_bernoulli_cantilever():
    """Isotropic slender cantilever with an end shear load P: the FE tip deflection
    increases monotonically under refinement toward the Timoshenko value
    PL^3/(3EI) + PL/(kappa G A) (kappa = 5/6) and is within 3 % on the finest mesh
    (full integration locks on coarse meshes, so convergence is from below)."""
    Ei = isotropic_constants(1e5, 0.3)
    P, L, H = 1.0, 200.0, 10.0
    I = H ** 4 / 12
    d_ref = P * L ** 3 / (3 * 1e5 * I) + P * L / (5 / 6 * 1e5 / 2.6 * H * H)
    prev, out = 0.0, []
    for n in (2, 4, 8):
        NX = 20 * n
        m = BeamMesh(NX, n, n, L / NX, H / n, H / n)
        A = assemble_global(m, np.zeros((NX, n, n)), Ei)
        u = solve_fine(m, A, m.face_load((0.0, 0.0, -P / H ** 2)))
        j, k = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
        d = -u[3 * m.node_id(NX, j.ravel(), k.ravel()) + 2].mean()
        assert d > prev
        prev = d
        out.append(d)
    assert abs(out[-1] / d_ref - 1) < 0.03
    assert (d_ref - out[1]) / (d_ref - out[2]) > 2.5
