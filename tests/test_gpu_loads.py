"""Nodal loads in place of the end-face traction (msgfem_mesh.load): GPU parity
with the oracle run on the same right-hand side (eigenvalues unchanged to 1e-8,
energy error and e_d within 1 % of the oracle's at equal n_loc), for a load
spread over the whole beam and for one on a corner of the free end, where only
some subdomains get a particular function."""
import numpy as np
import pytest

from oracle.coarse import run_msgfem
from oracle.errors import l2_errors
from oracle.mesh import make_mesh
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def _loads(cfg, kind):
    rng = np.random.default_rng(11)
    load = np.zeros((cfg.NX + 1, cfg.NY + 1, cfg.NZ + 1, 3))
    if kind == "spread":
        load[1:] = rng.standard_normal(load[1:].shape)
    else:
        load[cfg.NX, :2] = rng.standard_normal((2, cfg.NZ + 1, 3))
    return load.reshape(-1)


@pytest.mark.parametrize("name", ["t2", "s1"])
@pytest.mark.parametrize("kind", ["spread", "corner"])
def test_nodal_loads_parity(name, kind):
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    ang = element_angles(cfg)
    load = _loads(cfg, kind)
    ref = run_msgfem(cfg, angles=ang, load=load)
    m = MSGFEM.from_config(cfg, ang, seed=2, load=load)
    lam = m.local_spaces(cfg.n_loc)
    m.coarse_assemble()
    uG, err = m.solve(u_ref=ref.uh)
    lo = np.array(ref.lam)
    assert np.abs(lam - lo).max() <= 1e-8 * np.abs(lo).max()
    assert abs(err - ref.energy_error) <= 0.01 * ref.energy_error, (err, ref.energy_error)
    e_d, _ = m.solution_errors(ref.uh)
    o_d, _ = l2_errors(make_mesh(cfg), ref.uh, ref.uG)
    assert abs(e_d - o_d) <= 0.01 * o_d + 1e-12, (e_d, o_d)
    m.close()
