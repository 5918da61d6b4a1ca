"""Call order of the C ABI: setup -> local_spaces -> coarse_assemble -> solve,
with ESTATE for a call out of order; repeating a step discards the later ones
once the repeated call has accepted its arguments; a call whose arguments are
refused leaves the handle as it was."""
import ctypes as C

import numpy as np
import pytest

from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu

EINVAL, ESTATE = 1, 6


def test_call_order_and_repeats():
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("t1")
    m = MSGFEM.from_config(cfg, element_angles(cfg), seed=3)
    nc = C.c_int()
    u = np.zeros(m.n_dof)
    err = C.c_double()
    solve = lambda: m.lib.msgfem_solve(m.h, u.ctypes.data, None, C.byref(err))   # noqa: E731
    assert m.lib.msgfem_coarse_assemble(m.h, C.byref(nc)) == ESTATE
    assert solve() == ESTATE
    lam1 = m.local_spaces(cfg.n_loc).copy()
    assert solve() == ESTATE
    m.coarse_assemble()
    assert solve() == 0
    u1 = u.copy()
    assert np.abs(u1).max() > 0
    assert solve() == 0 and np.array_equal(u, u1)
    # refused arguments: nothing changes
    assert m.lib.msgfem_local_spaces(m.h, 0, None) == EINVAL
    assert m.lib.msgfem_coarse_assemble_threshold(m.h, -1.0, C.byref(nc)) == EINVAL
    assert solve() == 0 and np.array_equal(u, u1)
    # a repeated local stage discards the coarse problem and the solution
    lam2 = m.local_spaces(cfg.n_loc).copy()
    assert np.allclose(lam2, lam1, rtol=1e-10, atol=1e-12 * np.abs(lam1).max())
    assert solve() == ESTATE
    m.coarse_assemble()
    assert solve() == 0
    np.testing.assert_allclose(u, u1, rtol=0, atol=1e-10 * np.abs(u1).max())
    # a repeated coarse assembly needs a new solve only for its own result
    m.coarse_assemble(threshold=1e-6)
    assert solve() == 0
    m.close()
