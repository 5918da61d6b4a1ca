"""The library's host-side set-up (setup.cpp, run on the CPU through the host
harness) against the oracle: DoF classes B1/B2/B3 (Sec. 4.3), the partition of
unity (Sec. 4.2), the consistent end-face load (Eq. up_r's right-hand side),
and the 3-2-1 pins of floating subdomains (they must fix all six rigid
motions, Sec. 5.1's floating local problems), on box beams and curved
C-sections, plus the validation of explicit partition boxes, the grouping
of subdomains into memory-bounded waves and the element types that share one
element matrix."""
import numpy as np
import pytest

from tests.host import hostcheck as hc

pytestmark = pytest.mark.skipif(hc.cuda_include() is None, reason="host harness needs the CUDA headers")

CONFIGS = ("t1", "t2", "c1", "s1", "s2")


def _cfg(name):
    from workloads import get_config
    return get_config(name)


def _oracle(cfg):
    from oracle.mesh import make_mesh
    from oracle.partition import dof_classes, partition_of_unity, subdomains
    mesh = make_mesh(cfg)
    subs = subdomains(cfg)
    mus = partition_of_unity(mesh, subs, cfg.overlap)
    load = mesh.compression_load(cfg.traction)
    return mesh, subs, mus, load, dof_classes


def _local_nodes(mesh, s):
    """Global node ids of Omega*_j in the library's local order n = k npl + q."""
    i = np.arange(s["I0"], s["I1"] + 1)
    j = np.arange(s["J0"], s["J1"] + 1)
    k = np.arange(mesh.NZ + 1)
    kk, ii, jj = np.meshgrid(k, i, j, indexing="ij")
    return mesh.node_id(ii.ravel(), jj.ravel(), kk.ravel())


@pytest.mark.parametrize("name", CONFIGS)
def test_classes_pou_and_load_match_oracle(name):
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg)
    assert hs.status == 0, hs.error
    mesh, subs, mus, load, dof_classes = _oracle(cfg)
    assert hs.N == len(subs)
    for j, sub in enumerate(subs):
        s = hs.sub(j)
        a = hs.arrays(j)
        x0, x1, y0, y1 = sub.star
        assert (s["I0"], s["I1"], s["J0"], s["J1"]) == (x0, x1, y0, y1)
        assert (s["oI0"], s["oI1"], s["oJ0"], s["oJ1"]) == tuple(sub.omega)
        nodes = _local_nodes(mesh, s)
        # classes of the in-layer nodes (the same in every layer)
        onodes, b1, b2, b3 = dof_classes(mesh, sub)
        cls_o = np.where(b3, 3, np.where(b2, 2, 1))
        lookup = dict(zip(onodes.tolist(), cls_o.tolist()))
        assert [lookup[n] for n in nodes[:s["npl"]]] == a["cls"].tolist()
        assert (s["n1"], s["n2"], s["n3"]) == (3 * b1.sum(), 3 * b2.sum(), 3 * b3.sum())
        assert s["floating"] == int(not b3.any())
        # partition of unity on the Omega* nodes (zero outside Omega_j)
        np.testing.assert_allclose(a["mu"], mus[j][nodes], rtol=0, atol=1e-15)
        # consistent nodal load of the end-face traction
        ref = load.reshape(-1, 3)[nodes].reshape(-1)
        np.testing.assert_allclose(a["load"], ref, rtol=1e-13, atol=1e-13 * np.abs(load).max())
        # compact layer numberings: K keeps B1 + B2, A11 keeps B1, in layer order
        keepK = [3 * q + c for q in range(s["npl"]) for c in range(3) if a["cls"][q] != 3]
        keepA = [3 * q + c for q in range(s["npl"]) for c in range(3) if a["cls"][q] == 1]
        assert a["mapK"][:s["nK"]].tolist() == keepK and (a["mapK"][s["nK"]:] == -1).all()
        assert a["mapA"][:s["nA"]].tolist() == keepA and (a["mapA"][s["nA"]:] == -1).all()
        assert s["bK"] % hc.TILE == 0 and s["bK"] >= s["nK"] and s["bA"] % hc.TILE == 0 and s["bA"] >= s["nA"]
    hs.close()


def _rigid_modes(X):
    """The six rigid motions at points X (n x 3), as 3n x 6 (translations, rotations)."""
    n = len(X)
    R = np.zeros((3 * n, 6))
    for c in range(3):
        R[c::3, c] = 1.0
    Xc = X - X.mean(axis=0)
    for r, axis in enumerate(np.eye(3)):
        R[:, 3 + r] = np.cross(axis, Xc).reshape(-1)
    return R


@pytest.mark.parametrize("name", CONFIGS + ("c4",))
def test_pins_fix_all_rigid_motions(name):
    """A floating subdomain's K is pinned at six DoFs: the pinned rows of the rigid
    modes must be nonsingular (the pins remove every rigid motion), all pins
    distinct DoFs of B1 or B2 on the bottom layer; a clamped one has none."""
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg)
    assert hs.status == 0, hs.error
    from oracle.mesh import make_mesh
    mesh = make_mesh(cfg)
    nfloat = 0
    for j in range(hs.N):
        s = hs.sub(j)
        pins = s["pins"]
        if not s["floating"]:
            assert pins == [-1] * 6
            continue
        nfloat += 1
        assert len(set(pins)) == 6 and min(pins) >= 0
        a = hs.arrays(j)
        for p in pins:
            q = p // 3
            assert q < s["npl"] and a["cls"][q] != 3          # bottom layer, a kept DoF of K
        nodes = _local_nodes(mesh, s)
        R = _rigid_modes(mesh.coords(nodes))
        sv = np.linalg.svd(R[pins], compute_uv=False)
        assert sv[-1] > 1e-3 * sv[0], (j, sv)
    assert nfloat > 0
    hs.close()


def test_batched_instances_repeat_the_partition():
    cfg = _cfg("t2")
    one = hc.HostSetup(cfg)
    three = hc.HostSetup(cfg, instances=3)
    assert three.N == 3 * one.N
    for j in range(three.N):
        assert three.sub(j) == one.sub(j % one.N)
        a, b = three.arrays(j), one.arrays(j % one.N)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("boxes, why", [
    ([[0, 6, 0, 4], [5, 12, 0, 4]], "tile"),          # overlapping
    ([[0, 6, 0, 4], [7, 12, 0, 4]], "tile"),          # a gap
    ([[0, 6, 0, 4], [6, 13, 0, 4]], "outside"),       # beyond the mesh
    ([[0, 12, 0, 4], [3, 3, 0, 4]], "empty"),         # empty box
])
def test_explicit_boxes_are_validated(boxes, why):
    cfg = _cfg("t2")
    hs = hc.HostSetup(cfg, boxes=np.array(boxes))
    assert hs.status == 1 and why in hs.error, hs.error


def test_explicit_boxes_equal_the_regular_partition():
    cfg = _cfg("t2")
    reg = hc.HostSetup(cfg)
    boxes = [[a * cfg.NX // cfg.sx, (a + 1) * cfg.NX // cfg.sx, b * cfg.NY // cfg.sy, (b + 1) * cfg.NY // cfg.sy]
             for a in range(cfg.sx) for b in range(cfg.sy)]
    exp = hc.HostSetup(cfg, boxes=np.array(boxes))
    assert exp.status == 0 and exp.N == reg.N
    for j in range(reg.N):
        assert exp.sub(j) == reg.sub(j)
        np.testing.assert_array_equal(exp.arrays(j)["mu"], reg.arrays(j)["mu"])


@pytest.mark.parametrize("mixed", [False, True])
def test_waves_fit_the_budget(mixed):
    """Every subdomain in exactly one wave, members ascending, every wave within
    the budget, waves filled largest first; one wave when everything fits; a
    subdomain larger than the budget is refused (ENOMEM)."""
    cfg = _cfg("s2")
    hs = hc.HostSetup(cfg, mixed=mixed)
    sizes = np.array([hs.sub_bytes(j) for j in range(hs.N)])
    assert (sizes % 256 == 0).all() and (sizes > 0).all()
    assert hs.plan_waves(sizes.sum()) == 1
    assert hs.members(0) == list(range(hs.N)) and hs.pool_bytes == sizes.sum()
    for budget in (sizes.max(), 2 * sizes.max(), sizes.sum() // 3, sizes.sum() - 1):
        nw = hs.plan_waves(budget)
        assert nw >= 2
        seen = []
        fills = []
        for w in range(nw):
            m = hs.members(w)
            assert m == sorted(m) and len(m) > 0
            assert sizes[m].sum() <= budget
            fills.append(sizes[m].sum())
            seen += m
        assert sorted(seen) == list(range(hs.N))
        assert hs.pool_bytes == max(fills)
        # largest first: the first wave holds the largest subdomain
        assert int(np.argmax(sizes)) in hs.members(0)
    assert hs.plan_waves(sizes.max() - 1) == -2          # ENOMEM
    assert "wave budget" in hs.L.hc_error(hs.h).decode()
    # the FP32 factors of the mixed path need about half the bytes
    if mixed:
        ref = hc.HostSetup(cfg, mixed=False)
        r = np.array([ref.sub_bytes(j) for j in range(ref.N)])
        assert (sizes < 0.6 * r).all()


@pytest.mark.parametrize("name", ["s1", "s2"])
def test_curved_element_types_share_one_stiffness(name):
    """On a curved mesh, elements the library gives one type have the same oracle
    element matrix (Eq. element_stiffness with their own corners, frame and
    angle); elements of different types differ in shape, frame or angle; the
    types are exactly the distinct (relative corners, frame, angle) keys."""
    from oracle.element import hex_stiffness
    from oracle.material import rotated_tensor
    from oracle.mesh import make_mesh
    from workloads import element_angles
    cfg = _cfg(name)
    mesh = make_mesh(cfg)
    ang = element_angles(cfg)
    hs = hc.HostSetup(cfg)
    layered, types, etype, trep = hs.element_types(ang, mesh.frames)
    assert not layered and etype.min() == 0 and etype.max() == len(types) - 1
    nel = cfg.NX * cfg.NY * cfg.NZ
    ii, jj, kk = np.unravel_index(np.arange(nel), (cfg.NX, cfg.NY, cfg.NZ))
    keys = {}
    for e in range(nel):
        X = mesh.element_corners(ii[e], jj[e], kk[e])
        key = ((X - X[0]).tobytes(), mesh.frames[ii[e], jj[e], kk[e]].tobytes(), float(ang.reshape(-1)[e]))
        keys.setdefault(key, set()).add(int(etype[e]))
    assert all(len(v) == 1 for v in keys.values())               # one type per key
    assert len(keys) == len(types)                               # and one key per type
    assert (etype[trep] == np.arange(len(types))).all()          # a type's first element carries it
    assert np.array_equal(types, ang.reshape(-1)[trep])
    assert len(types) < nel                                      # the curved mesh still repeats shapes
    E = cfg.material
    rng = np.random.default_rng(0)
    for t in rng.choice(len(types), size=min(12, len(types)), replace=False):
        members = np.nonzero(etype == t)[0]
        r = trep[t]
        Kr = hex_stiffness(mesh.element_corners(ii[r], jj[r], kk[r]),
                           rotated_tensor(E, float(types[t]), mesh.frames[ii[r], jj[r], kk[r]]))
        for e in members[:: max(1, len(members) // 5)]:
            Ke = hex_stiffness(mesh.element_corners(ii[e], jj[e], kk[e]),
                               rotated_tensor(E, float(ang.reshape(-1)[e]), mesh.frames[ii[e], jj[e], kk[e]]))
            assert np.abs(Ke - Kr).max() <= 1e-12 * np.abs(Kr).max()


def test_box_beam_element_types():
    """Box beam: an angle field that depends on the ply only gives one type per
    ply and instance (layered); one element off its ply's angle gives one type
    per element; ply frames make the mesh curved-typed (shape, frame, angle)."""
    from workloads import element_angles
    cfg = _cfg("t2")
    nel = cfg.NX * cfg.NY * cfg.NZ
    ang = element_angles(cfg).reshape(-1)
    hs = hc.HostSetup(cfg, instances=2)
    two = np.concatenate([ang, ang + 15.0])
    layered, types, etype, trep = hs.element_types(two)
    assert layered and np.array_equal(types, np.concatenate([ang[:cfg.NZ], ang[:cfg.NZ] + 15.0]))
    bad = two.copy()
    bad[nel + 7] += 1.0
    layered, types, _, _ = hs.element_types(bad)
    assert not layered and np.array_equal(types, bad)
    frames = np.broadcast_to(np.eye(3), (nel, 3, 3))
    one = hc.HostSetup(cfg)
    layered, types, etype, trep = one.element_types(ang, frames)
    assert not layered and len(types) == len(np.unique(ang[:cfg.NZ]))   # congruent bricks: one type per angle
    assert np.array_equal(types[etype[:nel]], ang)


@pytest.mark.parametrize("name", ["t2", "c1", "s1", "s2"])
def test_coarse_pairs_cover_every_coupling(name):
    """A^H_{st} = V_s^T A V_t couples nodes p with mu_s(p) > 0 to nodes q with
    mu_t(q) > 0 that share an element with p (oracle partition of unity).  Every
    such (s, t) must be a coarse pair of the library, and all such nodes p must
    lie in the pair's node box, over which the block is accumulated."""
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg)
    mesh, subs, mus, _, _ = _oracle(cfg)
    pairs = {(int(r[0]), int(r[1])): r[2:] for r in hs.pairs()}
    shape = (cfg.NX + 1, cfg.NY + 1, cfg.NZ + 1)
    pos = [(mu > 0).reshape(shape) for mu in mus]
    for t, pt in enumerate(pos):
        # nodes sharing an element with the support of mu_t (index-space neighbours)
        near = np.zeros(shape, dtype=bool)
        padded = np.pad(pt, 1)
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    near |= padded[1 + di:1 + di + shape[0], 1 + dj:1 + dj + shape[1], 1 + dk:1 + dk + shape[2]]
        for s, ps in enumerate(pos):
            I, J, _ = np.nonzero(ps & near)
            if len(I) == 0:
                continue
            assert (s, t) in pairs, (s, t)
            x0, x1, y0, y1 = pairs[s, t]
            assert I.min() >= x0 and I.max() <= x1 and J.min() >= y0 and J.max() <= y1, (s, t)


@pytest.mark.parametrize("name", ["t2", "s1"])
def test_nodal_loads_reach_every_subdomain(name):
    """Given nodal forces replace the end-face traction: each subdomain holds
    their restriction to its Omega* nodes, and gets a particular function
    exactly when they are non-zero on one of its B1 DoFs."""
    cfg = _cfg(name)
    mesh, subs, _, _, _ = _oracle(cfg)
    rng = np.random.default_rng(4)
    load = np.zeros((cfg.NX + 1, cfg.NY + 1, cfg.NZ + 1, 3))
    load[cfg.NX, :2] = rng.standard_normal((2, cfg.NZ + 1, 3))        # a corner of the free end
    hs = hc.HostSetup(cfg, load=load)
    assert hs.status == 0, hs.error
    flat = load.reshape(-1, 3)
    seen = set()
    for j in range(hs.N):
        s = hs.sub(j)
        a = hs.arrays(j)
        nodes = _local_nodes(mesh, s)
        np.testing.assert_array_equal(a["load"], flat[nodes].reshape(-1))
        b1 = np.repeat(np.tile(a["cls"], s["nzn"]) == 1, 3)
        seen.add(bool(s["loaded"]))
        assert s["loaded"] == int(np.any(a["load"][b1] != 0.0))
    assert seen == {True, False}
    # without the array: the traction's particular function on Omega* touching x = L
    ref = hc.HostSetup(cfg)
    for j in range(ref.N):
        s = ref.sub(j)
        assert s["loaded"] == int(s["I1"] == cfg.NX)
