"""msgfem_energy_error_noalloc: the energy error of caller-owned device vectors
computed with a fixed device array instead of allocated scratch memory.

Callers whose device memory is committed elsewhere, or that must not enter
the driver's allocator, use this entry point; it must give the same number as
the energy error that msgfem_solve reports for the same vectors.  This file is
collected last so that a failure here does not hide the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from oracle.coarse import run_msgfem
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def test_noalloc_energy_error_matches_solve_twice():
    import torch
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t2")
    ang = element_angles(cfg)
    ref = run_msgfem(cfg, angles=ang)
    m = MSGFEM.from_config(cfg, ang, seed=5)
    m.local_spaces(cfg.n_loc)
    m.coarse_assemble()
    dev = torch.device("cuda", 0)
    u_dev = torch.zeros(m.n_dof, dtype=torch.float64, device=dev)
    uref_dev = torch.tensor(ref.uh, dtype=torch.float64, device=dev)
    _, err_solve = m.solve(u_ref=ref.uh, u_out=u_dev)
    torch.cuda.synchronize()
    out = []
    for _ in range(2):
        e = C.c_double(-1.0)
        st = m.lib.msgfem_energy_error_noalloc(m.h, u_dev.data_ptr(), uref_dev.data_ptr(), C.addressof(e))
        assert st == 0, m.lib.msgfem_last_error(m.h)
        out.append(e.value)
    # device output pointer as well
    e_dev = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    assert m.lib.msgfem_energy_error_noalloc(m.h, u_dev.data_ptr(), uref_dev.data_ptr(), e_dev.data_ptr()) == 0
    torch.cuda.synchronize()
    out.append(float(e_dev.item()))
    for v in out:
        assert v > 0
        assert abs(v - err_solve) <= 1e-12 * err_solve, (v, err_solve)
    assert out[0] == out[1]
    # host vectors are rejected with a message
    e = C.c_double(-1.0)
    uh = np.ascontiguousarray(ref.uh)
    assert m.lib.msgfem_energy_error_noalloc(m.h, uh.ctypes.data, uref_dev.data_ptr(), C.addressof(e)) == 1
    assert b"device pointers" in m.lib.msgfem_last_error(m.h)
    m.close()
