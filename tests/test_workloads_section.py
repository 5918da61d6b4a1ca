"""The C-section workload as specified: its geometry (web, flanges, corner radius,
length, plies), mesh sizes, the subdomain boxes tiling the mesh, the range of the
oversampling-domain sizes, and ply frames that are orthonormal, right-handed and
tangent to the cross-section."""
import numpy as np

from workloads import get_config
from workloads.section import omega_star_sizes, section_frames, section_nodes


def test_c4_mesh_and_partition():
    cfg = get_config("c4")
    assert (cfg.NX, cfg.NY, cfg.NZ) == (250, 110, 32)
    assert cfg.n_dof == 2_758_239
    assert cfg.n_sub == 256
    cover = np.zeros((cfg.NX, cfg.NY), dtype=int)
    for x0, x1, y0, y1 in cfg.boxes:
        cover[x0:x1, y0:y1] += 1
    assert (cover == 1).all()
    s = omega_star_sizes(cfg)
    assert s.min() == 4455 and s.max() == 41580


def test_c4_geometry():
    cfg = get_config("c4")
    X = section_nodes(cfg)
    inner = X[0, :, 0, 1:]                   # inner surface at x = 0
    outer = X[0, :, -1, 1:]
    # flange tips at y = 60 (inner face), web inner face at y = 0, flanges 200 mm apart
    assert np.allclose(inner[0], [60.0, -100.0]) and np.allclose(inner[-1], [60.0, 100.0])
    assert np.isclose(inner[:, 0].min(), 0.0)
    # laminate 8 mm thick everywhere: outer minus inner surface has length 8
    assert np.allclose(np.linalg.norm(outer - inner, axis=1), 8.0)
    assert np.isclose(X[-1, 0, 0, 0], 1000.0)
    # corner nodes on the arc of radius 8 about (8, -92) and (8, 92)
    nf, nc = cfg.segments[0], cfg.segments[1]
    c1 = inner[nf:nf + nc + 1]
    assert np.allclose(np.linalg.norm(c1 - [8.0, -92.0], axis=1), 8.0)


def test_section_frames_orthonormal_and_tangent():
    cfg = get_config("s2")
    F = section_frames(cfg)[0, :, 0]
    X = section_nodes(cfg)[0, :, 0, 1:]
    for j in range(cfg.NY):
        R = F[j]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.isclose(np.linalg.det(R), 1.0)
        chord = X[j + 1] - X[j]
        assert np.allclose(R[1, 1:], chord / np.linalg.norm(chord))
        assert np.allclose(R[0], [1.0, 0.0, 0.0])


def test_per_subdomain_eigenpair_counts():
    """c4: 16 eigenpairs on the smallest oversampling domain, 31 on the largest,
    never fewer on a larger domain; a section without n_loc_max keeps one count."""
    from workloads.section import n_loc_per_subdomain, omega_star_sizes
    cfg = get_config("c4")
    n = n_loc_per_subdomain(cfg)
    d = omega_star_sizes(cfg)
    assert n.shape == (256,) and n.dtype == np.int32
    assert n[np.argmin(d)] == 16 and n[np.argmax(d)] == 31 and n.min() == 16 and n.max() == 31
    order = np.argsort(d, kind="stable")
    assert np.all(np.diff(n[order]) >= 0)
    s = get_config("s2")
    assert np.all(n_loc_per_subdomain(s) == s.n_loc)
