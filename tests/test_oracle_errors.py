"""Pins of the L2 error oracle (oracle/errors.py, Sec. 5.4's e_d and e_eps):
closed-form integrals of linear fields on the box beam (moments of the box)
and on the curved C-section (volume = shoelace area of the cross-section x
length; a linear field has the constant strain sym(G)), zero strain of an
infinitesimal rigid motion, and the ratios' special cases."""
import numpy as np
import pytest

from oracle.errors import field_norms, l2_errors
from oracle.mesh import make_mesh
from workloads import get_config


def _linear_field(mesh, G, c):
    X = mesh.coords(np.arange(mesh.n_nodes))
    return (X @ G.T + c).reshape(-1)


def _shoelace_area(P):
    y, z = P[:, 0], P[:, 1]
    return 0.5 * abs((y * np.roll(z, -1) - np.roll(y, -1) * z).sum())


def _volume(mesh, cfg):
    if getattr(mesh, "general", False):
        outline = np.concatenate([mesh.xyz[0, :, 0, 1:], mesh.xyz[0, ::-1, mesh.NZ, 1:]])
        return _shoelace_area(outline) * (mesh.xyz[mesh.NX, 0, 0, 0] - mesh.xyz[0, 0, 0, 0])
    return cfg.NX * cfg.hx * cfg.NY * cfg.hy * cfg.NZ * cfg.t


@pytest.mark.parametrize("name", ["t2", "s1"])
def test_linear_field_strain_and_constant_field(name):
    cfg = get_config(name)
    mesh = make_mesh(cfg)
    V = _volume(mesh, cfg)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    sym = 0.5 * (G + G.T)
    _, s = field_norms(mesh, _linear_field(mesh, G, c))
    assert np.isclose(s, V * (sym * sym).sum(), rtol=1e-12)
    d, s0 = field_norms(mesh, _linear_field(mesh, np.zeros((3, 3)), c))
    assert np.isclose(d, V * c @ c, rtol=1e-12) and s0 < 1e-24 * d


def test_linear_field_displacement_on_the_box():
    """int_box |G x + c|^2 dx = V (tr(G^T G M) + c^T G L + |c|^2) with the box's
    second moments M_ii = L_i^2 / 3, M_ij = L_i L_j / 4 and first moments L / 2."""
    cfg = get_config("t2")
    mesh = make_mesh(cfg)
    L = np.array([cfg.NX * cfg.hx, cfg.NY * cfg.hy, cfg.NZ * cfg.t])
    V = L.prod()
    M = np.outer(L, L) / 4.0
    np.fill_diagonal(M, L * L / 3.0)
    rng = np.random.default_rng(1)
    for _ in range(3):
        G = rng.standard_normal((3, 3))
        c = rng.standard_normal(3)
        d, _ = field_norms(mesh, _linear_field(mesh, G, c))
        exact = V * (np.trace(G.T @ G @ M) + c @ G @ L + c @ c)
        assert np.isclose(d, exact, rtol=1e-12)


@pytest.mark.parametrize("name", ["t2", "s1"])
def test_rigid_motion_has_no_strain(name):
    cfg = get_config(name)
    mesh = make_mesh(cfg)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(3)
    W = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])   # x -> w x x
    ref = rng.standard_normal(mesh.n_dof)
    rigid = _linear_field(mesh, W, rng.standard_normal(3))
    e_d, e_eps = l2_errors(mesh, ref, ref - rigid)
    assert e_d > 0.1 and e_eps < 1e-13


def test_error_ratios_special_cases():
    cfg = get_config("t2")
    mesh = make_mesh(cfg)
    ref = np.random.default_rng(3).standard_normal(mesh.n_dof)
    assert l2_errors(mesh, ref, ref) == (0.0, 0.0)
    assert np.allclose(l2_errors(mesh, ref, np.zeros_like(ref)), (1.0, 1.0), rtol=1e-14)
    assert np.allclose(l2_errors(mesh, ref, 0.75 * ref), (0.25, 0.25), rtol=1e-13)
    # the norms are those of the fields, not of the DoF vectors: refining the
    # mesh with the same linear field leaves them unchanged
    G = np.diag([1.0, 2.0, 3.0])
    fine = make_mesh(cfg.with_(NX=2 * cfg.NX, hx=cfg.hx / 2))
    a = field_norms(mesh, _linear_field(mesh, G, np.ones(3)))
    b = field_norms(fine, _linear_field(fine, G, np.ones(3)))
    assert np.allclose(a, b, rtol=1e-12)
