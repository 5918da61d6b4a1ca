"""Two-level additive Schwarz PCG on the GPU (msgfem_schwarz_solve; Sec. 2.3,
Eq. condition_bound; the paper's reference solver of Sec. 5.3-5.4) against the
oracle of oracle/schwarz.py.

The local Dirichlet solves are the A11 factors of a handle whose oversampling
equals its overlap; the coarse space is an MS-GFEM handle's (or a GenEO
handle's) after coarse assembly.  Checked: the PCG solution equals the
oracle's direct u_h to 1e-9 in the energy norm, the iteration counts equal the
oracle's PCG with the same preconditioner (within one), the CG-Lanczos
estimates of the condition number agree with the oracle's (2 %), starting from
u^G saves iterations, more GenEO modes lower the condition number, the
library's own load vector equals the oracle's, and the coarse handle's own
solve is unchanged afterwards."""
from dataclasses import replace

import numpy as np
import pytest

from oracle.coarse import run_msgfem
from oracle.geneo import geneo_basis
from oracle.mesh import make_mesh
from oracle.partition import subdomains
from oracle.schwarz import TwoLevelSchwarz, pcg
from parity_util import energy_rel
from workloads import element_angles, get_config

pytestmark = pytest.mark.gpu


def _local(cfg, ang, **kw):
    from paper_2211_13893_gb300 import MSGFEM
    return MSGFEM.from_config(replace(cfg, oversampling=cfg.overlap), ang, seed=7, **kw)


@pytest.mark.parametrize("name", ["c1", "t3"])
def test_schwarz_with_msgfem_coarse_space(name):
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config(name)
    ang = element_angles(cfg)
    ref = run_msgfem(cfg, angles=ang)
    mesh = make_mesh(cfg)
    prec = TwoLevelSchwarz(mesh, ref.A, subdomains(cfg), ref.V)
    cold = pcg(mesh, ref.A, ref.b, prec)
    warm = pcg(mesh, ref.A, ref.b, prec, x0=ref.uG)
    hc = MSGFEM.from_config(cfg, ang, seed=7)
    hc.local_spaces(cfg.n_loc)
    hc.coarse_assemble()
    uG, _ = hc.solve()
    hl = _local(cfg, ang)
    u, inf = hl.schwarz_solve(hc, b=ref.b, rtol=1e-10)
    assert energy_rel(ref.A, u, ref.uh) <= 1e-9, energy_rel(ref.A, u, ref.uh)
    assert inf["residual"] <= 1e-10
    assert abs(inf["iterations"] - cold.iterations) <= 1, (inf, cold.iterations)
    assert abs(inf["kappa"] - cold.kappa) <= 0.02 * cold.kappa, (inf["kappa"], cold.kappa)
    # the library's own load (b = NULL) and the start from u^G
    u2, inf2 = hl.schwarz_solve(hc, u0=uG, rtol=1e-10)
    assert energy_rel(ref.A, u2, ref.uh) <= 1e-9
    assert inf2["iterations"] < inf["iterations"]
    assert abs(inf2["iterations"] - warm.iterations) <= 1, (inf2, warm.iterations)
    uG2, _ = hc.solve()
    assert np.array_equal(uG, uG2)
    # one level: a worse condition number than with the coarse space
    one = pcg(mesh, ref.A, ref.b, TwoLevelSchwarz(mesh, ref.A, subdomains(cfg)))
    u1, inf1 = hl.schwarz_solve(None, b=ref.b, rtol=1e-10)
    assert energy_rel(ref.A, u1, ref.uh) <= 1e-9
    assert abs(inf1["kappa"] - one.kappa) <= 0.02 * one.kappa, (inf1["kappa"], one.kappa)
    assert inf1["kappa"] > 2.0 * inf["kappa"]
    hl.close()
    hc.close()


def test_schwarz_with_geneo_coarse_spaces():
    """t3: GenEO handles with 8, 12 and 16 modes per subdomain serve as their
    own local solvers and coarse spaces; the condition number falls with the
    number of modes, as the oracle's does, and matches it."""
    cfg = get_config("t3")
    ang = element_angles(cfg)
    mesh = make_mesh(cfg)
    kap = []
    for n in (8, 12, 16):
        V, _, _, A, b = geneo_basis(cfg, angles=ang, n_loc=n)
        orc = pcg(mesh, A, b, TwoLevelSchwarz(mesh, A, subdomains(cfg), V))
        g = _local(cfg, ang, method=1)
        g.local_spaces(n)
        g.coarse_assemble()
        u, inf = g.schwarz_solve(g, b=b, rtol=1e-10)
        g.close()
        assert inf["residual"] <= 1e-10
        assert abs(inf["kappa"] - orc.kappa) <= 0.02 * orc.kappa, (n, inf["kappa"], orc.kappa)
        assert abs(inf["iterations"] - orc.iterations) <= 1, (n, inf, orc.iterations)
        kap.append(inf["kappa"])
    assert kap[0] > kap[1] > kap[2]


def test_schwarz_mixed_precision_local_solves():
    """FP32 local factors as the Dirichlet solvers: PCG still reaches u_h (FP64
    products and recurrences)."""
    from paper_2211_13893_gb300 import MSGFEM
    cfg = get_config("c1")
    ang = element_angles(cfg)
    ref = run_msgfem(cfg, angles=ang)
    hc = MSGFEM.from_config(cfg, ang, seed=7, precision=1)
    hc.local_spaces(cfg.n_loc)
    hc.coarse_assemble()
    hl = _local(cfg, ang, precision=1)
    u, inf = hl.schwarz_solve(hc, b=ref.b, rtol=1e-10)
    assert energy_rel(ref.A, u, ref.uh) <= 1e-9
    hl.close()
    hc.close()


def test_schwarz_refuses_oversampled_local_handle():
    from paper_2211_13893_gb300 import MSGFEM, MsgfemError
    cfg = get_config("t2")
    ang = element_angles(cfg)
    m = MSGFEM.from_config(cfg, ang)          # oversampling 2 > overlap 1
    with pytest.raises(MsgfemError) as err:
        m.schwarz_solve(None)
    assert err.value.code == 1
    m.close()
