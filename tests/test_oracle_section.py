"""Pins of the oracle on the curved C-section spar: general hexahedra, per-element
ply frames, the end-face load and subdomain problems on curved geometry.

What fixes each value: the covariance of elasticity under a rigid rotation of
the body together with its material, the rigid-body null space, the exact
energy of a constant strain over an extruded element (volume from the
shoelace area of its cross-section), the resultant and first moment of a
uniform traction (polygon area and centroid formulas), the patch test, and
the uniform-compression solution of a prismatic bar (Saint-Venant) away from
the clamped end.
"""
import numpy as np
import pytest

from oracle.assemble import assemble_global, make_cache
from oracle.element import CORNERS, hex_stiffness
from oracle.fine import solve_fine
from oracle.local import local_eigs_dense, local_problem
from oracle.material import isotropic_constants, rotated_tensor
from oracle.mesh import HexMesh, make_mesh
from oracle.partition import partition_of_unity, subdomains
from workloads import element_angles, get_config
from workloads.section import SectionConfig

E_PLY = get_config("c1").material


def random_rotation(rng):
    Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def distorted_hex(rng):
    X = (CORNERS + 1.0) / 2.0 * np.array([2.0, 1.5, 0.5])
    return X + 0.15 * rng.standard_normal(X.shape)


def shoelace(P):
    """Signed area and first moments (int y dA, int z dA) of a polygon P (n x 2)."""
    y, z = P[:, 0], P[:, 1]
    y1, z1 = np.roll(y, -1), np.roll(z, -1)
    cr = y * z1 - y1 * z
    A = 0.5 * cr.sum()
    return A, ((y + y1) * cr).sum() / 6.0, ((z + z1) * cr).sum() / 6.0


def test_frame_identity_is_the_beam_rotation():
    for th in (0.0, 30.0, -45.0, 90.0):
        assert np.allclose(rotated_tensor(E_PLY, th, np.eye(3)), rotated_tensor(E_PLY, th), atol=1e-9)


def test_rotation_covariance_of_element_stiffness():
    """Rotating the element and its ply frame by G maps K to G K G^T per node."""
    rng = np.random.default_rng(0)
    for _ in range(3):
        X = distorted_hex(rng)
        F = random_rotation(rng).T          # rows: an arbitrary right-handed frame
        th = rng.uniform(-90, 90)
        G = random_rotation(rng)
        K1 = hex_stiffness(X, rotated_tensor(E_PLY, th, F))
        K2 = hex_stiffness(X @ G.T, rotated_tensor(E_PLY, th, F @ G.T))
        Gb = np.kron(np.eye(8), G)
        assert np.allclose(K2, Gb @ K1 @ Gb.T, rtol=0, atol=1e-9 * np.abs(K1).max())


def test_frame_axes_fix_the_fibre_direction():
    """The fibre modulus lies along cos(t) a0 + sin(t) a1 of the element's frame."""
    rng = np.random.default_rng(1)
    F = random_rotation(rng).T
    for th in (0.0, 35.0, 90.0):
        C = rotated_tensor(E_PLY, th, F)
        f = np.cos(np.deg2rad(th)) * F[0] + np.sin(np.deg2rad(th)) * F[1]
        # uniaxial strain along f: the normal stress along f is C_ffff = 1/S11 of the ply
        eps = np.outer(f, f)
        sig = np.einsum("ijkl,kl->ij", C, eps)
        S = np.linalg.inv(np.array([[1 / 162000.0, -0.35 / 162000.0, -0.35 / 162000.0],
                                    [-0.35 / 162000.0, 1 / 10000.0, -0.5 / 10000.0],
                                    [-0.35 / 162000.0, -0.5 / 10000.0, 1 / 10000.0]]))
        assert np.isclose(f @ sig @ f, S[0, 0], rtol=1e-12)


@pytest.mark.parametrize("j", [4, 7, 12])
def test_curved_element_null_space(j):
    """An element on a corner arc has exactly the six rigid modes as null space."""
    cfg = get_config("s1")
    m = make_mesh(cfg)
    X = m.element_corners(1, j, 1)
    K = hex_stiffness(X, rotated_tensor(E_PLY, 45.0, m.frames[1, j, 1]))
    w = np.linalg.eigvalsh(K)
    assert np.all(w[:6] < 1e-10 * w[-1]) and w[6] > 1e-6 * w[-1]
    c = X.mean(0)
    R = [np.tile(np.eye(3)[a], 8) for a in range(3)] + [np.cross(e, X - c).ravel() for e in np.eye(3)]
    for r in R:
        assert np.abs(K @ r).max() < 1e-9 * np.abs(K).max()


@pytest.mark.parametrize("j", [1, 5, 10])
def test_constant_strain_energy_is_volume_times_density(j):
    """u = eps x on an extruded element: u^T K u = V eps:C:eps, V = h_x * cross-section area."""
    cfg = get_config("s1")
    m = make_mesh(cfg)
    X = m.element_corners(2, j, 2)
    F = m.frames[2, j, 2]
    C = rotated_tensor(E_PLY, 30.0, F)
    K = hex_stiffness(X, C)
    rng = np.random.default_rng(j)
    eps = rng.standard_normal((3, 3))
    eps = 0.5 * (eps + eps.T)
    u = (X @ eps.T).ravel()
    face = X[[0, 3, 7, 4]][:, 1:]           # the corners at the low x end, in cyclic order
    A, _, _ = shoelace(face)
    V = abs(A) * (X[1, 0] - X[0, 0])
    assert np.isclose(u @ K @ u, V * np.einsum("ij,ijkl,kl->", eps, C, eps), rtol=1e-11)


def test_section_face_load_resultant_and_moment():
    cfg = get_config("s1")
    m = make_mesh(cfg)
    b = m.compression_load(1.0)
    A = Sy = Sz = 0.0
    for j in range(m.NY):
        for k in range(m.NZ):
            P = np.array([m.xyz[m.NX, j, k], m.xyz[m.NX, j + 1, k], m.xyz[m.NX, j + 1, k + 1],
                          m.xyz[m.NX, j, k + 1]])[:, 1:]
            a, sy, sz = shoelace(P)
            sgn = np.sign(a)
            A, Sy, Sz = A + sgn * a, Sy + sgn * sy, Sz + sgn * sz
    bx = b[0::3]
    X = m.coords(np.arange(m.n_nodes))
    assert np.isclose(bx.sum(), -A, rtol=1e-12)
    assert np.isclose((bx * X[:, 1]).sum(), -Sy, rtol=1e-12)
    assert abs((bx * X[:, 2]).sum() + Sz) < 1e-10 * A * cfg.web
    assert np.abs(b[1::3]).max() == 0.0 and np.abs(b[2::3]).max() == 0.0


def test_section_patch_test():
    """A linear displacement field leaves no force on nodes inside the curved mesh
    (homogeneous material: an isotropic tensor is the same in every ply frame)."""
    cfg = get_config("s1")
    m = make_mesh(cfg)
    E = isotropic_constants(70000.0, 0.3)
    A = assemble_global(m, element_angles(cfg), E, cache=make_cache(m, E))
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, 3))
    X = m.coords(np.arange(m.n_nodes))
    u = (X @ G.T + rng.standard_normal(3)).ravel()
    f = (A @ u).reshape(-1, 3)
    i, j, k = m.node_ijk(np.arange(m.n_nodes))
    inner = (i > 0) & (i < m.NX) & (j > 0) & (j < m.NY) & (k > 0) & (k < m.NZ)
    assert inner.sum() > 50
    assert np.abs(f[inner]).max() < 1e-10 * np.abs(f).max()


@pytest.mark.parametrize("material,theta", [("iso", 0.0), ("ply", 0.0)])
def test_section_uniform_compression_mid_span(material, theta):
    """A prismatic bar under uniform end compression: away from the clamped end the
    mean axial strain over the section is eps_xx = -p / E_x (the clamp's restraint
    of the lateral contraction is self-equilibrated; on this thin open section it
    still bends the bar slightly at mid-span, so only the axial strain is pinned)."""
    cfg = SectionConfig("cs", length=400.0, web=40.0, flange=20.0, radius=4.0, n_plies=2, t=1.0,
                        h_len=10.0, h_arc=4.0, h_corner=2.0, xparts=(40,), sparts=(24,))
    assert cfg.NY == 24
    E = isotropic_constants(70000.0, 0.3) if material == "iso" else E_PLY
    Ex = 70000.0 if material == "iso" else E_PLY[0]
    m = HexMesh.from_config(cfg)
    ang = np.full((cfg.NX, cfg.NY, cfg.NZ), theta)
    A = assemble_global(m, ang, E, cache=make_cache(m, E))
    p = 2.0
    u = solve_fine(m, A, m.compression_load(p)).reshape(-1, 3)
    X = m.coords(np.arange(m.n_nodes))
    i, _, _ = m.node_ijk(np.arange(m.n_nodes))
    a, b = i == 18, i == 22
    exx = (u[b, 0].mean() - u[a, 0].mean()) / (X[b, 0].mean() - X[a, 0].mean())
    assert abs(exx / (-p / Ex) - 1.0) < 1e-3


def test_floating_curved_subdomain_has_rigid_null_modes():
    """A floating oversampling domain over a curved corner: six zero eigenvalues
    whose span holds the rigid modes of the curved geometry (Sec. 5.2)."""
    cfg = get_config("s2")
    m = make_mesh(cfg)
    ang = element_angles(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    b = m.compression_load(cfg.traction)
    cache = make_cache(m, cfg.material)
    s = subs[5]          # second x part, second arc part: floating, spans a corner
    assert s.star[0] > 0 and s.star[2] < 11 < s.star[3]
    lp = local_problem(m, ang, cfg.material, s, mus[s.index], b, cache)
    lam, phi = local_eigs_dense(lp, 8)
    top = abs(lam[7])
    assert np.all(np.abs(lam[:6]) < 1e-8 * top) and lam[6] > 1e-4 * top
    X = m.coords(lp.nodes)
    c = X.mean(0)
    R = np.array([np.tile(np.eye(3)[a], len(X)) for a in range(3)] +
                 [np.cross(e, X - c).ravel() for e in np.eye(3)]).T
    Q, _ = np.linalg.qr(phi[:, :6])
    resid = R - Q @ (Q.T @ R)
    assert np.linalg.norm(resid) < 1e-6 * np.linalg.norm(R)


def test_general_mesh_reduces_to_the_box_beam():
    """A HexMesh given the box beam's node coordinates and identity frames assembles
    the same stiffness and load as the box-beam path (whose pins are the beam tests)."""
    from oracle.assemble import assemble_global
    from oracle.mesh import BeamMesh
    cfg = get_config("t2")
    box = BeamMesh.from_config(cfg)
    i, j, k = np.meshgrid(np.arange(cfg.NX + 1), np.arange(cfg.NY + 1), np.arange(cfg.NZ + 1), indexing="ij")
    xyz = np.stack([i * cfg.hx, j * cfg.hy, k * cfg.t], axis=-1).astype(np.float64)
    frames = np.broadcast_to(np.eye(3), (cfg.NX, cfg.NY, cfg.NZ, 3, 3)).copy()
    gen = HexMesh(xyz, frames)
    ang = element_angles(cfg)
    Ab = assemble_global(box, ang, cfg.material)
    Ag = assemble_global(gen, ang, cfg.material, cache=make_cache(gen, cfg.material))
    assert abs(Ab - Ag).max() <= 1e-10 * abs(Ab).max()
    assert np.allclose(gen.compression_load(1.0), box.compression_load(1.0), rtol=0, atol=1e-12)
