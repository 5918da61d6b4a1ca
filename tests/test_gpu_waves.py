"""Memory-bounded waves and explicit subdomain boxes.

A handle whose layer-block storage is capped (msgfem_options.wave_mb) runs the
local stage in waves of subdomains that share one factor pool; every
subdomain's eigenproblem is independent of the others, so the eigenvalues and
the coarse solution must equal those of the one-wave run.  A box beam given
its regular partition as an explicit list of boxes must give the same result
as the sx x sy description."""
import numpy as np
import pytest

from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def _run(cfg, ang, **kw):
    from paper_2211_13893_gb300 import MSGFEM
    m = MSGFEM.from_config(cfg, ang, seed=7, **kw)
    lam = m.local_spaces(cfg.n_loc)
    m.coarse_assemble()
    u, _ = m.solve()
    prof = m.profile()
    m.close()
    return lam, u, prof


@pytest.mark.parametrize("name,precision,tol", [("t4", 0, 1e-10), ("s2", 1, 1e-8)])
def test_waves_match_one_wave(name, precision, tol):
    cfg = get_config(name)
    ang = element_angles(cfg)
    la, ua, pa = _run(cfg, ang, precision=precision)
    assert pa["waves"] == 1
    lb, ub, pb = _run(cfg, ang, precision=precision, wave_mb=pa["pool_mb"] / 3.0)
    assert pb["waves"] >= 3 and pb["pool_mb"] <= pa["pool_mb"] / 3.0 + 1e-9
    scale = np.abs(la).max(axis=1, keepdims=True)
    assert (np.abs(la - lb) / scale).max() <= tol
    assert np.abs(ua - ub).max() <= tol * np.abs(ua).max()


def test_wave_budget_below_one_subdomain_is_rejected():
    from paper_2211_13893_gb300 import MSGFEM
    from paper_2211_13893_gb300.msgfem import MsgfemError
    cfg = get_config("t2")
    with pytest.raises(MsgfemError) as e:
        MSGFEM.from_config(cfg, element_angles(cfg), wave_mb=1e-3)
    assert e.value.code == 2


def test_explicit_boxes_equal_regular_partition():
    cfg = get_config("t3")
    ang = element_angles(cfg)
    boxes = [((a * cfg.NX) // cfg.sx, ((a + 1) * cfg.NX) // cfg.sx, (b * cfg.NY) // cfg.sy, ((b + 1) * cfg.NY) // cfg.sy)
             for a in range(cfg.sx) for b in range(cfg.sy)]
    la, ua, _ = _run(cfg, ang)
    lb, ub, _ = _run(cfg, ang, boxes=np.array(boxes))
    assert np.array_equal(la, lb) and np.array_equal(ua, ub)


def test_boxes_that_do_not_tile_are_rejected():
    from paper_2211_13893_gb300 import MSGFEM
    from paper_2211_13893_gb300.msgfem import MsgfemError
    cfg = get_config("t2")
    boxes = np.array([(0, 6, 0, 4), (5, 12, 0, 4)])       # element column 5 covered twice
    with pytest.raises(MsgfemError) as e:
        MSGFEM.from_config(cfg, element_angles(cfg), boxes=boxes)
    assert e.value.code == 1
