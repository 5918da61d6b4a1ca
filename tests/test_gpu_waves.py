"""Memory-bounded waves, explicit subdomain boxes, the block-solve kernels and
the autotuner.

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


@pytest.mark.parametrize("name,precision,tol,kernel", [("t4", 0, 1e-10, 0), ("s2", 1, 1e-8, 0), ("s2", 1, 1e-8, 4)])
def test_waves_match_one_wave(name, precision, tol, kernel):
    cfg = get_config(name)
    ang = element_angles(cfg)
    la, ua, pa = _run(cfg, ang, precision=precision, solve_kernel=kernel)
    assert pa["waves"] == 1
    lb, ub, pb = _run(cfg, ang, precision=precision, wave_mb=pa["pool_mb"] / 3.0, solve_kernel=kernel)
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


@pytest.mark.parametrize("name,precision,kernel", [("t4", 0, 2), ("t4", 0, 3), ("t4", 0, 4), ("s2", 1, 1),
                                                   ("s2", 1, 2), ("s2", 1, 3), ("s2", 1, 4), ("t2", 1, 4),
                                                   ("c1", 1, 4)])
def test_solve_kernels_parity(name, precision, kernel):
    """Every block-solve kernel the autotuner may choose gives oracle parity
    (kernel 4, the TMA-filled ring, is FP32 only: with FP64 the default runs)."""
    from test_gpu_local import run_case
    tol = (1e-8, 1e-5) if precision == 0 else (1e-5, 1e-4)
    run_case(name, precision=precision, tol_lam=tol[0], tol_angle=tol[1], solve_kernel=kernel)


def test_autotune_keeps_results_and_adopts_choice():
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("s2")
    ang = element_angles(cfg)
    m = MSGFEM.from_config(cfg, ang, seed=7, precision=1)
    la = m.local_spaces(cfg.n_loc)
    t = m.autotune()
    assert t["streams"] in (4, 8, 16, 32) and t["solve_kernel"] in (1, 2, 3, 4) and t["best_ms"] > 0
    assert t["factor_schedule"] in (0, 1) and t["factor_streams"] in (16, 32)
    assert min(x for row in t["factor_ms"] for x in row if x > 0) > 0
    assert min(x for row in t["solve_ms"] for x in row if x > 0) == pytest.approx(t["best_ms"])
    assert any(row[3] > 0 for row in t["solve_ms"])            # the TMA ring was timed
    lb = m.local_spaces(cfg.n_loc)
    m.close()
    scale = np.abs(la).max(axis=1, keepdims=True)
    assert (np.abs(la - lb) / scale).max() <= 1e-6


@pytest.mark.parametrize("name,precision", [("t4", 0), ("s2", 1), ("c1", 1)])
def test_left_looking_factorisation_parity(name, precision):
    """The left-looking factorisation schedule gives oracle parity."""
    from test_gpu_local import run_case
    tol = (1e-8, 1e-5) if precision == 0 else (1e-5, 1e-4)
    run_case(name, precision=precision, tol_lam=tol[0], tol_angle=tol[1], factor_schedule=1)


@pytest.mark.parametrize("name", ["t4", "s2", "c1"])
def test_persistent_factorisation_is_bit_identical(name):
    """msgfem_options.factor_persistent = 1: the FP32 factorisation as one
    cooperative launch whose CTAs take the tasks in a topological order (one
    dependency group per chain) gives the step schedule's factors bit for bit,
    hence the same eigenvalues and coarse solution, also over memory-bounded
    waves (s2)."""
    cfg = get_config(name)
    ang = element_angles(cfg)
    la, ua, pa = _run(cfg, ang, precision=1)
    lb, ub, _ = _run(cfg, ang, precision=1, factor_persistent=1)
    assert np.array_equal(la, lb) and np.array_equal(ua, ub)
    if name == "s2":
        lc, uc, pc = _run(cfg, ang, precision=1, factor_persistent=1, wave_mb=pa["pool_mb"] / 3.0)
        assert pc["waves"] >= 3
        assert np.array_equal(la, lc) and np.array_equal(ua, uc)


def test_autotune_times_the_persistent_factorisation():
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("c1")
    m = MSGFEM.from_config(cfg, element_angles(cfg), seed=7, precision=1)
    la = m.local_spaces(cfg.n_loc).copy()
    t = m.autotune()
    lb = m.local_spaces(cfg.n_loc)
    m.close()
    assert all(x > 0 for x in t["factor_ms_persistent"]), t
    assert t["factor_persistent"] in (0, 1)
    if t["factor_persistent"]:
        assert t["factor_kernel"] == 0
    assert np.array_equal(la, lb) or (np.abs(la - lb) / np.abs(la).max(axis=1, keepdims=True)).max() <= 1e-6
