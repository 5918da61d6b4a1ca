"""A failure made on the host and reported by a status code (nothing traps
or hangs the GPU: every kernel loop is bounded and the tile Cholesky records
a non-positive pivot instead of stopping): an indefinite material (negative
fibre modulus) gives ENOTSPD naming the subdomain."""
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
