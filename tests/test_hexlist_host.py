"""General mesh input on the host (no GPU): a hexahedron list in any node and
element order, per-node clamp flags and an element -> part map (Sec. 3.1,
Sec. 4.1) are mapped onto the structured problem the local stage needs.
Checked through msgfem_plan, which runs the same decomposition as
msgfem_setup without a handle: the shuffled list plans exactly like the
structured mesh, and meshes the layer-block factorisation cannot take are
refused (EINVAL): an element with another local orientation, a part that is
not a box through the thickness, missing elements."""
import ctypes as C

import numpy as np
import pytest

from hexlist import box_parts, hex_list
from workloads import get_config


@pytest.fixture(scope="module")
def lib():
    from paper_2211_13893_gb300.build import build
    build()
    from paper_2211_13893_gb300 import msgfem
    return msgfem


def _plan(ms, cfg, xyz=None, hex8=None, elem_part=None, structured=False):
    info = ms.PlanInfo()
    opt = ms.Options()
    if structured:
        mesh = ms.Mesh(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t, cfg.traction, None, None)
    else:
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        hex8 = np.ascontiguousarray(hex8, dtype=np.int32)
        mesh = ms.Mesh(0, 0, 0, 0.0, 0.0, 0.0, cfg.traction, None, None, 1, len(xyz), len(hex8), xyz.ctypes.data,
                       hex8.ctypes.data, None)
    ep = None if elem_part is None else np.ascontiguousarray(elem_part, dtype=np.int32)
    part = ms.Partition(cfg.sx, cfg.sy, 0, None, None if ep is None else ep.ctypes.data)
    st = ms.load_library().msgfem_plan(C.byref(mesh), C.byref(part), cfg.overlap, cfg.oversampling, C.byref(opt),
                                       C.byref(info))
    return st, {k: getattr(info, k) for k, _ in ms.PlanInfo._fields_}


@pytest.mark.parametrize("name", ["t2", "t4", "c1"])
def test_shuffled_hex_list_plans_like_the_structured_mesh(lib, name):
    cfg = get_config(name)
    st0, ref = _plan(lib, cfg, structured=True)
    assert st0 == 0
    for seed in (0, 1):
        xyz, hex8, _, elem_of_user = hex_list(cfg, seed)
        st, got = _plan(lib, cfg, xyz, hex8)
        assert st == 0 and got == ref
        ep = box_parts(cfg)[elem_of_user]           # the box partition in the list's element order
        st, got = _plan(lib, cfg, xyz, hex8, elem_part=ep)
        assert st == 0 and got == ref


def test_refused_hex_lists(lib):
    cfg = get_config("t2")
    xyz, hex8, _, elem_of_user = hex_list(cfg, 3)
    # one element listed with another local orientation (rotated about its zeta axis)
    bad = hex8.copy()
    bad[5] = bad[5][[1, 2, 3, 0, 5, 6, 7, 4]]
    assert _plan(lib, cfg, xyz, bad)[0] == 1
    # an element missing
    assert _plan(lib, cfg, xyz, hex8[:-1])[0] == 1
    # a node id out of range
    bad = hex8.copy()
    bad[0, 0] = len(xyz)
    assert _plan(lib, cfg, xyz, bad)[0] == 1
    # a part that is not a box through the thickness
    ep = box_parts(cfg).copy()
    ep[0] = 1                                      # the bottom ply of one column moved to another part
    assert _plan(lib, cfg, xyz, hex8, elem_part=ep[elem_of_user])[0] == 1
    # part ids with a gap
    ep = box_parts(cfg) * 2
    assert _plan(lib, cfg, xyz, hex8, elem_part=ep[elem_of_user])[0] == 1
