"""General mesh input on the GPU (msgfem_mesh.kind = 1, dirichlet_node,
msgfem_partition.elem_part; Sec. 3.1, Sec. 4.1): a structured test mesh given
as a hexahedron list with shuffled node and element numbers, explicit clamp
flags and an element -> part map equal to its box partition is the same
problem, so every result is bit-identical to the structured run's once the
permutation is undone (against the structured mesh given by the same node
coordinates; the box of bricks computes its element matrices from the brick
size and agrees to rounding): eigenvalues, the coarse solution (returned in the
list's node order), the energy error against a reference in that order, the
allocation-free energy error on device vectors in that order."""
import ctypes as C

import numpy as np
import pytest

from hexlist import box_parts, clamp_flags, hex_list, structured_xyz
from parity_util import assert_eigs
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def _pair(name, seed=2):
    """The structured handle (with explicit node coordinates, the same element
    path as a hexahedron list) and the hexahedron-list handle."""
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    ang = element_angles(cfg).reshape(-1)
    ref = MSGFEM.from_config(cfg, ang, seed=7, xyz=structured_xyz(cfg))
    xyz, hex8, node_of_user, elem_of_user = hex_list(cfg, seed)
    kw = {}
    if getattr(cfg, "kind", "beam") == "section":
        from workloads.section import section_frames
        kw["frames"] = section_frames(cfg).reshape(-1, 9)[elem_of_user]
    m = MSGFEM(0, 0, 0, 0.0, 0.0, 0.0, cfg.traction, cfg.material, ang[elem_of_user], 0, 0, cfg.overlap,
               cfg.oversampling, seed=7, xyz=xyz, hex8=hex8, dirichlet=clamp_flags(cfg, node_of_user),
               elem_part=box_parts(cfg)[elem_of_user], **kw)
    return cfg, ang, ref, m, node_of_user, elem_of_user


@pytest.mark.parametrize("name", ["t2", "s1"])
def test_hex_list_is_bit_identical_to_the_structured_mesh(name):
    import torch
    from oracle.coarse import run_msgfem
    cfg, ang, ref, m, node_of_user, elem_of_user = _pair(name)
    dims, nodes, elems = m.numbering()
    assert dims == (cfg.NX, cfg.NY, cfg.NZ)
    assert np.array_equal(nodes, node_of_user) and np.array_equal(elems, elem_of_user)
    assert m.N == ref.N
    la = ref.local_spaces(cfg.n_loc)
    lb = m.local_spaces(cfg.n_loc)
    assert np.array_equal(la, lb)
    if getattr(cfg, "kind", "beam") == "beam":
        # the box of bricks (element matrices from hx, hy, hz) agrees to rounding
        from paper_2211_13893_gb300 import MSGFEM
        box = MSGFEM.from_config(cfg, ang, seed=7)
        lbox = box.local_spaces(cfg.n_loc)
        box.close()
        for j in range(m.N):
            assert_eigs(lb[j], lbox[j], 1e-10, j)
    assert ref.coarse_assemble() == m.coarse_assemble()
    uh = run_msgfem(cfg, angles=element_angles(cfg)).uh                  # structured order
    ua, ea = ref.solve(u_ref=uh)
    uh_user = uh.reshape(-1, 3)[node_of_user].reshape(-1)
    ub, eb = m.solve(u_ref=uh_user)
    assert np.array_equal(ub.reshape(-1, 3), ua.reshape(-1, 3)[node_of_user])
    assert ea == eb
    # allocation-free energy error on device vectors in the list's order
    du = torch.tensor(ub, device="cuda")
    dr = torch.tensor(uh_user, device="cuda")
    e = C.c_double(-1.0)
    assert m.lib.msgfem_energy_error_noalloc(m.h, du.data_ptr(), dr.data_ptr(), C.addressof(e)) == 0
    assert abs(e.value - eb) <= 1e-12 * eb
    # angles updated in the list's element order
    ang2 = ang + 1.5
    ref.update_angles(ang2)
    m.update_angles(ang2[elem_of_user])
    assert np.array_equal(ref.local_spaces(cfg.n_loc), m.local_spaces(cfg.n_loc))
    ref.close()
    m.close()


def test_clamp_flags_elsewhere_are_refused():
    from paper_2211_13893_gb300 import MSGFEM, MsgfemError
    cfg = get_config("t2")
    ang = element_angles(cfg).reshape(-1)
    xyz, hex8, node_of_user, elem_of_user = hex_list(cfg, 4)
    flags = clamp_flags(cfg, node_of_user)
    flags[np.argmax(flags == 0)] = 1                      # one more node clamped
    with pytest.raises(MsgfemError) as err:
        MSGFEM(0, 0, 0, 0.0, 0.0, 0.0, cfg.traction, cfg.material, ang[elem_of_user], 0, 0, cfg.overlap,
               cfg.oversampling, xyz=xyz, hex8=hex8, dirichlet=flags)
    assert err.value.code == 1 and "dirichlet_node" in str(err.value)
