"""Domain decomposition, DoF classes and the partition of unity.

Sec. 3.1: non-overlapping subdomains hat-Omega_j are extended by o element
layers to Omega_j; Sec. 3.3: Omega_j is extended further to the oversampling
domain Omega*_j (o* layers counted from hat-Omega_j, Sec. 4.2).  The
non-overlapping subdomains here are element boxes in (x, y) spanning the full
thickness: a regular sx x sy partition (subdomain (a, b) has index
j = a sy + b) or a list of boxes given by the workload.

DoF classes on Omega*_j (Sec. 4.3): B3 = nodes on the clamped face, B2 =
nodes on the closure of the cut boundary dOmega*_j inside Omega (minus B3),
B1 = all other nodes.  An FE function that vanishes on the open cut face
vanishes at its corner nodes too, so the closure is used.

Partition of unity (Sec. 4.2): on Omega_j, w_p starts at 0 on the closure of
the cut boundary dOmega_j inside Omega and at 2o elsewhere, then
w_p <- min(w_p, min_q (w_q + 1), 2o) over the nodes q sharing an element with
p, repeated 2o - 1 times (Jacobi sweeps); mu_{j,p} = w_{j,p} / sum_i w_{i,p};
mu_j = 0 on Omega*_j \\ Omega_j.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Subdomain:
    index: int
    hat: tuple      # element box (x0, x1, y0, y1) of hat-Omega_j
    omega: tuple    # element box of Omega_j
    star: tuple     # element box of Omega*_j


def _split(n, parts, a):
    return (a * n) // parts, ((a + 1) * n) // parts


def subdomains(cfg):
    """Subdomains of a workload: the regular sx x sy box partition, or the
    explicit non-overlapping element boxes of ``cfg.boxes`` (C-section)."""
    boxes = getattr(cfg, "boxes", None)
    if boxes is not None:
        out = []
        for idx, (x0, x1, y0, y1) in enumerate(boxes):
            def grow(m, x0=x0, x1=x1, y0=y0, y1=y1):
                return (max(0, x0 - m), min(cfg.NX, x1 + m), max(0, y0 - m), min(cfg.NY, y1 + m))
            out.append(Subdomain(idx, (x0, x1, y0, y1), grow(cfg.overlap), grow(cfg.oversampling)))
        return out
    out = []
    for a in range(cfg.sx):
        for b in range(cfg.sy):
            x0, x1 = _split(cfg.NX, cfg.sx, a)
            y0, y1 = _split(cfg.NY, cfg.sy, b)

            def grow(m):
                return (max(0, x0 - m), min(cfg.NX, x1 + m), max(0, y0 - m), min(cfg.NY, y1 + m))
            out.append(Subdomain(a * cfg.sy + b, (x0, x1, y0, y1), grow(cfg.overlap), grow(cfg.oversampling)))
    return out


def box_nodes(mesh, box):
    """Global node ids of an element box (full thickness), in (i, j, k) lexicographic order."""
    x0, x1, y0, y1 = box
    i, j, k = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1), np.arange(mesh.NZ + 1), indexing="ij")
    return mesh.node_id(i.ravel(), j.ravel(), k.ravel())


def on_cut_boundary(mesh, box, nodes):
    """True for nodes on the closure of the part of the box boundary inside Omega."""
    x0, x1, y0, y1 = box
    i, j, _ = mesh.node_ijk(nodes)
    return (((i == x0) & (x0 > 0)) | ((i == x1) & (x1 < mesh.NX)) |
            ((j == y0) & (y0 > 0)) | ((j == y1) & (y1 < mesh.NY)))


def dof_classes(mesh, sub):
    """Node lists of B1, B2, B3 on Omega*_j, in the order of ``box_nodes``."""
    nodes = box_nodes(mesh, sub.star)
    i, _, _ = mesh.node_ijk(nodes)
    b3 = i == 0
    b2 = on_cut_boundary(mesh, sub.star, nodes) & ~b3
    b1 = ~(b2 | b3)
    return nodes, b1, b2, b3


def pou_weights(mesh, sub, o):
    """Relaxed weights w_j on the nodes of Omega_j (array over its node box)."""
    x0, x1, y0, y1 = sub.omega
    nodes = box_nodes(mesh, sub.omega)
    shape = (x1 - x0 + 1, y1 - y0 + 1, mesh.NZ + 1)
    w = np.where(on_cut_boundary(mesh, sub.omega, nodes), 0.0, 2.0 * o).reshape(shape)
    for _ in range(2 * o - 1):
        padded = np.pad(w, 1, constant_values=np.inf)
        best = np.full(shape, np.inf)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    if di == dj == dk == 0:
                        continue
                    best = np.minimum(best, padded[1 + di:1 + di + shape[0], 1 + dj:1 + dj + shape[1],
                                                   1 + dk:1 + dk + shape[2]])
        w = np.minimum(np.minimum(w, best + 1.0), 2.0 * o)
    return nodes, w.ravel()


def partition_of_unity(mesh, subs, o):
    """mu_j as global node arrays (zero outside Omega_j), one per subdomain."""
    ws = []
    total = np.zeros(mesh.n_nodes)
    for s in subs:
        nodes, w = pou_weights(mesh, s, o)
        g = np.zeros(mesh.n_nodes)
        g[nodes] = w
        ws.append(g)
        total += g
    if (total <= 0).any():
        raise ValueError("partition of unity: a node has zero total weight")
    return [g / total for g in ws]
