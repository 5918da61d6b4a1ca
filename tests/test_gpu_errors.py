"""GPU parity of the relative L2 errors of the coarse solution (Sec. 5.4, e_d
and e_eps; msgfem_solution_errors) against the oracle's (oracle/errors.py) on
the same coarse solution, for the box beam and the curved C-section; the
special cases u_ref = u^G (zero) and a device reference; ESTATE before a
solve."""
import ctypes as C

import numpy as np
import pytest

from oracle.coarse import run_msgfem
from oracle.errors import l2_errors
from oracle.mesh import make_mesh
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["t2", "s1"])
def test_solution_errors_match_oracle(name):
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    ang = element_angles(cfg)
    m = MSGFEM.from_config(cfg, ang, seed=1)
    out = (C.c_double * 2)()
    ref = run_msgfem(cfg, angles=ang)
    assert m.lib.msgfem_solution_errors(m.h, ref.uh.ctypes.data, out) == 6          # ESTATE
    m.local_spaces(cfg.n_loc)
    m.coarse_assemble()
    assert m.lib.msgfem_solution_errors(m.h, ref.uh.ctypes.data, out) == 6
    uG, _ = m.solve()
    e_d, e_eps = m.solution_errors(ref.uh)
    o_d, o_eps = l2_errors(make_mesh(cfg), ref.uh, uG)
    assert 0.0 < o_d < 1.0 and 0.0 < o_eps < 1.0
    assert abs(e_d - o_d) <= 1e-10 * o_d and abs(e_eps - o_eps) <= 1e-10 * o_eps, (e_d, o_d, e_eps, o_eps)
    assert m.solution_errors(uG) == (0.0, 0.0)
    dev = torch.tensor(ref.uh, dtype=torch.float64, device="cuda")
    assert m.solution_errors(dev) == (e_d, e_eps)
    m.close()
