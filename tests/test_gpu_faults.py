"""Failures made on the host and reported by a status code (nothing traps or
hangs the GPU: every kernel loop is bounded and the tile Cholesky records a
non-positive pivot instead of stopping): an indefinite material (negative
fibre modulus) gives ENOTSPD naming the subdomain; non-finite angles are
refused; a step cap of one gives ENOCONV; a start block that cannot converge
falls back to the cold start."""
import pytest

from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def _handle(cfg, ang, E=None, **kw):
    from paper_2211_13893_gb300 import MSGFEM
    E = cfg.material if E is None else E
    return MSGFEM(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t, cfg.traction, E, ang, cfg.sx, cfg.sy,
                  cfg.overlap, cfg.oversampling, **kw)


def test_indefinite_material_is_reported():
    from paper_2211_13893_gb300.msgfem import MsgfemError
    cfg = get_config("t1")
    E = list(cfg.material)
    E[0] = -E[0]
    m = _handle(cfg, element_angles(cfg), E)
    with pytest.raises(MsgfemError) as err:
        m.local_spaces(cfg.n_loc)
    assert err.value.code == 4 and "subdomain" in str(err.value)
    m.close()


def test_non_finite_angles_are_refused():
    """A NaN fibre angle is refused at set-up and by msgfem_update_angles (EINVAL)."""
    import numpy as np
    from paper_2211_13893_gb300.msgfem import MsgfemError
    cfg = get_config("t1")
    ang = element_angles(cfg).copy()
    bad = ang.copy()
    bad.reshape(-1)[5] = np.nan
    with pytest.raises(MsgfemError) as err:
        _handle(cfg, bad)
    assert err.value.code == 1 and "angle" in str(err.value)
    m = _handle(cfg, ang)
    with pytest.raises(MsgfemError) as err:
        m.update_angles(bad)
    assert err.value.code == 1
    m.local_spaces(cfg.n_loc)          # the handle is still usable with its previous angles
    m.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_step_cap_gives_enoconv(solver):
    """max_iter = 1 stops the eigensolver (block Krylov or subspace iteration)
    before convergence: ENOCONV with the last Rayleigh-Ritz pairs, finite and
    ascending, a residual above the tolerance reported per subdomain; the same
    handle converges with the default cap."""
    import numpy as np
    from paper_2211_13893_gb300.msgfem import MsgfemError
    cfg = get_config("t2")
    ang = element_angles(cfg)
    m = _handle(cfg, ang, max_iter=1, solver=solver, seed=3)
    with pytest.raises(MsgfemError) as err:
        m.local_spaces(cfg.n_loc)
    assert err.value.code == 5
    lam = m.local_spaces(cfg.n_loc, allow_noconv=True)
    assert np.all(np.isfinite(lam)) and np.all(np.diff(lam, axis=1) >= -1e-12 * np.abs(lam).max())
    res = [m.info(j)["residual"] for j in range(m.N)]
    assert max(res) > 1e-7
    m.close()
    m = _handle(cfg, ang, solver=solver, seed=3)
    m.local_spaces(cfg.n_loc)
    assert max(m.info(j)["residual"] for j in range(m.N)) <= 1e-5
    m.close()


@pytest.mark.parametrize("kind", ["nan", "zero"])
def test_bad_warm_start_falls_back_to_cold_start(kind):
    """Start blocks that cannot lead anywhere fall back to the cold start, the
    warm start's fallback: a block with NaN entries (a network that produced
    NaN) is refused before use; an all-zero block (finite, rank 0) makes the
    block Krylov basis break down, the subdomain reaches the step cap
    unconverged and is solved again from the cold start.  Eigenvalues equal
    those of a cold run (1e-8 per eigenvalue) and msgfem_subinfo.cold_restart
    marks the subdomains."""
    import numpy as np
    import torch
    from parity_util import assert_eigs
    cfg = get_config("t2")
    ang = element_angles(cfg)
    cold = _handle(cfg, ang, seed=3)
    lam_cold = cold.local_spaces(cfg.n_loc)
    cold.close()
    m = _handle(cfg, ang, seed=3)
    m.local_spaces(cfg.n_loc)
    blocks = {}
    for j in range(m.N):
        n2, nw = m.warm_sizes(j, cfg.n_loc)
        if nw <= 0:
            continue
        fill = float("nan") if kind == "nan" else 0.0
        blocks[j] = torch.full((n2, 8), fill, dtype=torch.float32, device="cuda")
        m.set_start_block(j, blocks[j], 8, 8)
    assert blocks
    lam = m.local_spaces(cfg.n_loc)
    for j in range(m.N):
        assert m.info(j)["cold_restart"] == (1 if j in blocks else 0), j
        assert_eigs(lam[j], lam_cold[j], 1e-8, j)
    assert max(m.info(j)["residual"] for j in range(m.N)) <= 1e-5
    m.close()
