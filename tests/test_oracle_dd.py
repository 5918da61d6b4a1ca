"""Pins of the oracle's decomposition: boxes, DoF classes and the partition
of unity (Secs. 3.1, 4.2, 4.3 of the paper)."""
import numpy as np
import pytest

from oracle.mesh import BeamMesh
from oracle.partition import (box_nodes, dof_classes, on_cut_boundary,
                              partition_of_unity, pou_weights, subdomains)
from workloads import get_config


@pytest.mark.parametrize("name", ["t1", "t2", "t3", "t4", "c1", "c2"])
def test_pou_sums_to_one(name):
    """sum_j R_j^T Xi_j v = v for any v (Eq. PoU): the weights add to one."""
    cfg = get_config(name)
    m = BeamMesh.from_config(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(m, subs, cfg.overlap)
    total = np.sum(mus, axis=0)
    assert np.abs(total - 1.0).max() < 1e-14
    rng = np.random.default_rng(0)
    v = rng.standard_normal(m.n_nodes)
    assert np.allclose(sum(mu * v for mu in mus), v, rtol=0, atol=1e-14)
    for s, mu in zip(subs, mus):
        assert mu.min() >= 0 and mu.max() <= 1
        inside = np.zeros(m.n_nodes, dtype=bool)
        nodes = box_nodes(m, s.omega)
        inside[nodes] = True
        assert (mu[~inside] == 0).all()
        assert (mu[nodes[on_cut_boundary(m, s.omega, nodes)]] == 0).all()


@pytest.mark.parametrize("name", ["t2", "t4", "c2"])
def test_pou_weights_are_clipped_distance(name):
    """After 2o - 1 relaxation sweeps the weight is min(2o, Chebyshev (i, j)
    distance to the cut boundary of Omega_j): the closed form on a box."""
    cfg = get_config(name)
    m = BeamMesh.from_config(cfg)
    o = cfg.overlap
    for s in subdomains(cfg):
        nodes, w = pou_weights(m, s, o)
        x0, x1, y0, y1 = s.omega
        i, j, _ = m.node_ijk(nodes)
        d = np.full(len(nodes), np.inf)
        if x0 > 0:
            d = np.minimum(d, i - x0)
        if x1 < m.NX:
            d = np.minimum(d, x1 - i)
        if y0 > 0:
            d = np.minimum(d, j - y0)
        if y1 < m.NY:
            d = np.minimum(d, y1 - j)
        assert np.array_equal(w, np.minimum(d, 2 * o))


def test_pou_linear_across_a_two_subdomain_overlap():
    """In a 2 x 1 split the two weights add to 2o inside the overlap, so mu is
    linear in x there (the smooth transition of Sec. 4.2)."""
    cfg = get_config("c1")
    m = BeamMesh.from_config(cfg)
    mus = partition_of_unity(m, subdomains(cfg), cfg.overlap)
    xs = np.arange(10, 15)
    vals = mus[0][m.node_id(xs, 2, 5)]
    assert np.allclose(vals, [1.0, 1.0, 0.5, 0.0, 0.0])


def class_counts(cfg):
    m = BeamMesh.from_config(cfg)
    return [tuple(3 * int(c.sum()) for c in dof_classes(m, s)[1:]) for s in subdomains(cfg)]


def test_dof_classes_c1():
    """C1: the clamped subdomain has its end face in B3, the other is floating."""
    assert class_counts(get_config("c1")) == [(2535, 195, 195), (2730, 195, 0)]


def test_dof_classes_c2_interior():
    counts = class_counts(get_config("c2"))
    assert counts[5] == (22800, 4920, 0)
    # the two subdomains at x = 0 each clamp an 11 x 40 node face
    assert sum(c[2] for c in counts) == 2 * 3 * 11 * 40


def test_boxes_cover_and_nest():
    cfg = get_config("c2")
    subs = subdomains(cfg)
    cover = np.zeros((cfg.NX, cfg.NY), dtype=int)
    for s in subs:
        x0, x1, y0, y1 = s.hat
        cover[x0:x1, y0:y1] += 1
        for inner, outer in ((s.hat, s.omega), (s.omega, s.star)):
            assert outer[0] <= inner[0] and outer[1] >= inner[1]
            assert outer[2] <= inner[2] and outer[3] >= inner[3]
    assert (cover == 1).all()
