"""Hexahedron-list versions of the structured test meshes (test helper, no
method arithmetic): node and element numberings shuffled by a seeded
permutation, elements in the standard local node order (nodes 0-3
counterclockwise on the bottom face, 4-7 above), per-node clamp flags on the
x = 0 face and an element -> part map for a box partition."""
import numpy as np

# local node a of the standard order -> (di, dj, dk)
HEX_OFF = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])


def structured_xyz(cfg):
    """Node coordinates [n_nodes, 3] in the structured order (box beam or section)."""
    if getattr(cfg, "kind", "beam") == "section":
        from workloads.section import section_nodes
        return section_nodes(cfg).reshape(-1, 3)
    i, j, k = np.meshgrid(np.arange(cfg.NX + 1), np.arange(cfg.NY + 1), np.arange(cfg.NZ + 1), indexing="ij")
    return np.stack([i * cfg.hx, j * cfg.hy, k * cfg.t], axis=-1).reshape(-1, 3).astype(np.float64)


def hex_list(cfg, seed=0):
    """(xyz [n_nodes, 3], hex8 [n_elems, 8], node_of_user, elem_of_user): the
    mesh with user node u = structured node node_of_user[u] and user element e
    = structured element elem_of_user[e]."""
    NX, NY, NZ = cfg.NX, cfg.NY, cfg.NZ
    nn, ne = (NX + 1) * (NY + 1) * (NZ + 1), NX * NY * NZ
    rng = np.random.default_rng(seed)
    node_of_user = rng.permutation(nn)
    elem_of_user = rng.permutation(ne)
    user_of_node = np.argsort(node_of_user)
    xyz = structured_xyz(cfg)[node_of_user]
    hex8 = np.zeros((ne, 8), dtype=np.int64)
    for e in range(ne):
        s = elem_of_user[e]
        i, j, k = s // (NY * NZ), (s // NZ) % NY, s % NZ
        for a in range(8):
            di, dj, dk = HEX_OFF[a]
            hex8[e, a] = user_of_node[((i + di) * (NY + 1) + j + dj) * (NZ + 1) + k + dk]
    return xyz, hex8, node_of_user, elem_of_user


def clamp_flags(cfg, node_of_user):
    NY, NZ = cfg.NY, cfg.NZ
    return (node_of_user < (NY + 1) * (NZ + 1)).astype(np.uint8)


def box_parts(cfg):
    """Element -> part map (structured element order) of the sx x sy box partition or the explicit boxes."""
    NX, NY, NZ = cfg.NX, cfg.NY, cfg.NZ
    part = np.zeros((NX, NY, NZ), dtype=np.int32)
    boxes = getattr(cfg, "boxes", None)
    if boxes:
        for p, (x0, x1, y0, y1) in enumerate(boxes):
            part[x0:x1, y0:y1, :] = p
    else:
        for a in range(cfg.sx):
            for b in range(cfg.sy):
                part[a * NX // cfg.sx:(a + 1) * NX // cfg.sx, b * NY // cfg.sy:(b + 1) * NY // cfg.sy, :] = a * cfg.sy + b
    return part.reshape(-1)
